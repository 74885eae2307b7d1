"""Batched 1D Euler problems (one persistent launch per RK stage).

Each problem's result must be bitwise that of enomr_step on the problem
alone (same arithmetic), for every tile size the autotuner may pick, and
match the oracle like the single-problem path does.
"""
import numpy as np
import pytest

import oracle
from paper_2311_15504_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build_cuda()
    from paper_2311_15504_gb300 import enomr
    return enomr


@pytest.mark.parametrize("R,bc", [(9, 1), (5, 1), (17, 1), (9, 0)])
def test_batch_bitwise_equals_single_problems(E, R, bc):
    import torch
    sizes, Us, hs = wl.riemann_batch(37, seed=R, nmin=20 if bc else 2 * R, nmax=900)
    B = E.Batch(sizes, hs, order=R, bc=bc)
    Ub = B.pack(Us)
    singles = [E.Solver(E.EULER, int(n), order=R, dx=float(h), bc=bc) for n, h in zip(sizes, hs)]
    Uref = Ub.clone()
    views = [B.view(Uref, p) for p in range(len(sizes))]
    for step in range(6):
        if step == 3:
            B.autotune(Ub, reps=1)  # a different tile size / grid must not change results
        B.step(Ub, 0.5)
        for sp, v in zip(singles, views):
            sp.step(v, 0.0, 0.5)
    torch.cuda.synchronize()
    for p in range(len(sizes)):
        assert torch.equal(B.view(Ub, p), B.view(Uref, p)), p
    B.check_status()


@pytest.mark.parametrize("tile_reps", [1])
def test_batch_matches_oracle(E, tile_reps):
    sizes, Us, hs = wl.riemann_batch(9, seed=3, nmin=64, nmax=700)
    B = E.Batch(sizes, hs, order=9, bc=1)
    Ub = B.pack(Us)
    B.step(Ub, 0.5)
    for p in range(len(sizes)):
        P = oracle.Problem(oracle.EQ_EULER1D, 9, int(sizes[p]), dx=float(hs[p]),
                           bc=oracle.BC_TRANSMISSIVE)
        ref = P.step_ssprk3(Us[p], P.cfl_dt(Us[p], 0.5))
        got = B.view(Ub, p).cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max(), p
