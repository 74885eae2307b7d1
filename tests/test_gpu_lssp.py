"""Linear SSP-RK(m, m-1) on the GPU (Eq. lSSPRK): one step against the
oracle, and the paper's printed advection errors (Tables 5-7) reproduced by
the CUDA path itself."""
import numpy as np
import pytest

import oracle
from conftest import read_golden
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


@pytest.mark.parametrize("R,m", [(5, 6), (9, 10), (17, 18), (9, 3)])
def test_lssp_step_matches_oracle(E, R, m):
    import torch
    u, h = wl.advection_sine(130, power=3)
    s = E.Solver(E.ADVECTION, 130, order=R, dx=h, bc=E.PERIODIC)
    ud = torch.from_numpy(u).cuda()
    s.step_lssp(ud, h, m)
    P = oracle.Problem(oracle.EQ_ADVECTION, R, 130, dx=h, bc=oracle.BC_PERIODIC)
    ref = P.step_lssp(u, h, m)
    assert np.abs(ud.cpu().numpy() - ref).max() <= 1e-13


@pytest.mark.parametrize("row", read_golden("advection_errors_tables_5_7.txt"))
def test_paper_advection_errors_on_gpu(E, row):
    import torch
    parts = row.split()
    R, N, power = int(parts[0]), int(parts[1]), int(parts[2])
    lam, l1p, lip = float(parts[3]), float(parts[4]), float(parts[5])
    u0, h = wl.advection_sine(N, power, lam)
    s = E.Solver(E.ADVECTION, N, order=R, dx=h, bc=E.PERIODIC)
    ud = torch.from_numpy(u0).cuda()
    for _ in range(int(round(2.0 / h))):
        s.step_lssp(ud, h, R + 1)
    e = np.abs(ud.cpu().numpy() - u0)
    l1 = (e.sum() + e[0]) / (N + 1)   # the paper's N+1 nodes
    li = e.max()
    tol = 0.006 if l1p / lam > 1e-11 else 0.01
    assert abs(l1 - l1p) <= tol * l1p, (l1, l1p)
    assert abs(li - lip) <= tol * lip, (li, lip)
