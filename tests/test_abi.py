"""Host-side checks of the C ABI (no GPU needed).

The library must load, export every symbol include/enomr.h declares, and
reject bad arguments on the host before touching the device.  The CUDA-side
coefficient header must be the exact-rational tables, rounded once.
"""
import ctypes
import os
import re
import subprocess
import sys
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "enomr.h")
CSRC = os.path.join(ROOT, "paper_2311_15504_gb300", "csrc")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build_cuda()
    from paper_2311_15504_gb300 import enomr
    return enomr


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"ENOMR_API\s+[\w\s\*]+?\b(enomr_\w+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 10
    so = ctypes.CDLL(lib.LIB_PATH)
    for n in names:
        assert hasattr(so, n), n
    assert sorted(lib.EXPORTED) == names


def test_host_side_argument_checks(lib):
    L = lib._lib
    ctx = ctypes.c_void_p()
    P = ctypes.c_void_p
    bad = [
        (0, 1, 100, 1, 0.1, 0.1, 6, 1.4, 0, 1.0),    # even order
        (0, 1, 100, 1, 0.1, 0.1, 19, 1.4, 0, 1.0),   # order too high
        (0, 2, 100, 100, 0.1, 0.1, 5, 1.4, 0, 1.0),  # advection is 1D
        (1, 1, 100, 1, -0.1, 0.1, 5, 1.4, 0, 1.0),   # dx <= 0
        (1, 1, 100, 1, 0.1, 0.1, 5, 1.0, 0, 1.0),    # gamma <= 1
        (1, 1, 5, 1, 0.1, 0.1, 5, 1.4, 0, 1.0),      # periodic needs nx >= 2g
        (1, 2, 64, 4, 0.1, 0.1, 9, 1.4, 0, 1.0),     # periodic needs ny >= 2g
        (1, 1, 100, 1, 0.1, 0.1, 5, 1.4, 7, 1.0),    # unknown bc
        (3, 1, 100, 1, 0.1, 0.1, 5, 1.4, 0, 1.0),    # unknown equation
        (2, 2, 100, 100, 0.1, 0.1, 5, 1.4, 0, 1.0),  # Burgers is 1D
        (0, 1, 0, 1, 0.1, 0.1, 5, 1.4, 1, 1.0),      # empty line
        (1, 2, 0, 64, 0.1, 0.1, 5, 1.4, 1, 1.0),     # empty grid
    ]
    for args in bad:
        st = L.enomr_init(ctypes.byref(ctx), *args, P(0))
        assert st == 1, args
        assert not ctx.value
    assert L.enomr_rhs(None, None, None) == 1
    assert L.enomr_step(None, None, 0.0, 0.5, None) == 1
    assert L.enomr_get_status(None) == 1
    assert L.enomr_set_staging(None, 0) == 1
    assert L.enomr_set_occupancy(None, 0) == 1
    L.enomr_free(None)


def test_status_strings_and_tested_counts(lib):
    assert lib._lib.enomr_strerror(0) == b"ok"
    assert b"non-physical" in lib._lib.enomr_strerror(4)
    import oracle
    for R in lib.ORDERS:
        assert lib.num_tested(R) == oracle.num_tested(R)
    assert lib.num_tested(4) == -1


def test_generated_coefficients_are_fresh_and_exact():
    r = subprocess.run([sys.executable, os.path.join(CSRC, "gen_coeffs.py"), "--check"])
    assert r.returncode == 0
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from test_oracle_tables import exact_weights, golden_candidates
    text = open(os.path.join(CSRC, "enomr_coeffs.h")).read()
    for R in (5, 7, 9, 11, 13, 15, 17):
        g = (R + 1) // 2
        W = 2 * g - 1
        tested = [(m, n) for (m, n) in golden_candidates() if 1 <= m <= g - 1 and 1 <= n <= g - 1]
        for name, which in (("kB", 1), ("kA", 0)):
            body = re.search(rf"{name}{R}\[\d+\] = \{{(.*?)\}};", text, re.S).group(1)
            vals = [float.fromhex(x) if "0x" in x else float(x)
                    for x in re.findall(r"-?0x[0-9a-fp.+-]+|-?\d+\.\d+", body)]
            assert len(vals) == len(tested) * W
            for t, (m, n) in enumerate(tested):
                w = exact_weights(m, n)[which]
                row = vals[t * W:(t + 1) * W]
                want = [0.0] * W
                for s, x in enumerate(w):
                    want[s - m + g - 1] = float(Fraction(x))
                assert row == want, (R, t, name)


def test_batch_host_side_argument_checks(lib):
    import numpy as np
    L = lib._lib
    ctx = ctypes.c_void_p()
    P = ctypes.c_void_p
    n = np.array([100, 0, 50], dtype=np.int64)
    dx = np.array([0.1, 0.1, 0.1])
    assert L.enomr_batch_init(ctypes.byref(ctx), 3, n.ctypes.data_as(P), dx.ctypes.data_as(P),
                              9, 1.4, 1, P(0)) == 1
    n[1] = 5
    assert L.enomr_batch_init(ctypes.byref(ctx), 3, n.ctypes.data_as(P), dx.ctypes.data_as(P),
                              9, 1.4, 0, P(0)) == 1  # periodic needs n >= 2g
    dx[2] = 0.0
    assert L.enomr_batch_init(ctypes.byref(ctx), 3, n.ctypes.data_as(P), dx.ctypes.data_as(P),
                              9, 1.4, 1, P(0)) == 1
    assert L.enomr_batch_step(None, None, 0.5) == 1
    assert L.enomr_batch_total_cells(None) == -1
    L.enomr_batch_free(None)
