"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer.

`oracle_sanitize_driver.c` compiles the oracle into one process with both
sanitizers and calls every entry point on small and degenerate inputs (one-
to three-cell lines, the shortest periodic lines, one-cell-wide 2D grids,
boundary sides with moving splits, every order), with buffers of exactly the
sizes the entry points' contracts name.  Any out-of-bounds access, leak or
undefined integer arithmetic aborts it.  A case it found: reflective sides
on lines shorter than g read past the line; the oracle now rejects them, as
the C ABI does.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_oracle_under_address_and_ub_sanitizers(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    exe = str(tmp_path / "oracle_sanitize")
    build = subprocess.run(
        ["gcc", "-std=c99", "-O1", "-g", "-fsanitize=address,undefined",
         "-fno-sanitize-recover=all", "-fno-omit-frame-pointer", "-ffp-contract=off",
         "-I", ROOT, os.path.join(HERE, "oracle_sanitize_driver.c"), "-lm", "-o", exe],
        capture_output=True, text=True)
    if build.returncode != 0:
        pytest.skip("gcc cannot build with the sanitizers here: " + build.stderr[-300:])
    run = subprocess.run([exe], capture_output=True, text=True, timeout=900)
    assert run.returncode == 0, run.stderr[-3000:]
    assert run.stdout.strip().endswith("ok")


@pytest.mark.parametrize("R", [7, 17])
def test_reflective_side_needs_g_cells(R):
    g = (R + 1) // 2
    U = np.zeros((4, 20, g - 1))
    U[0] = 1.0
    U[3] = 2.5
    wall = oracle.side(oracle.SIDE_REFLECTIVE)
    with pytest.raises(oracle.OracleError):
        oracle.rhs_euler2d_ext(U, 0.1, 0.1, R, sides=(wall, None, None, None))
    # the same grid with a wall on the long (y) sides is accepted
    out = oracle.rhs_euler2d_ext(U, 0.1, 0.1, R, sides=(None, None, wall, wall))
    assert np.isfinite(out["rhs"]).all()
