"""GPU parity for the inviscid Burgers equation (Sec. 4.2) through the C ABI.

- RHS against the oracle at every order in the three flux treatments
  (u > 0: f^+ = f; u < 0: f^- = f; mixed signs: global Lax-Friedrichs),
  periodic and transmissive, sizes spanning several 255-cell tiles with a
  ragged tail; selections equal except at near-ties, values against the
  oracle re-run on the GPU's selections.
- Table 8 on the GPU: the SSP-RK3 runs of the accuracy test land on the
  oracle's final states (smooth: L1 <= 1e-10) and on the printed errors.
- The shock case (t = 2/lam, CFL 0.3): final state within the oracle's own
  rounding envelope.
- Edge cases: u = 0 (RHS 0, CFL step 0), NaN input (status word).
"""
import numpy as np
import pytest

import oracle
from burgers_exact import dt_schedule, errors
from conftest import read_golden
from parity import assert_selection, assert_values, shock_gate
from paper_2311_15504_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
ORDERS = [5, 7, 9, 11, 13, 15, 17]


@pytest.fixture(scope="module")
def E():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build_cuda()
    from paper_2311_15504_gb300 import enomr
    return enomr


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _field(kind, N, R):
    rng = np.random.Generator(np.random.PCG64(7 * N + R))
    x = np.arange(N) / N
    base = np.sin(2 * np.pi * x) + 0.3 * np.sin(6 * np.pi * x + 1.0)
    base += 0.4 * (np.abs(x - 0.6) < 0.1)  # a plateau with two jumps
    if kind == "positive":
        return 1.5 + base + 0.05 * rng.random(N)
    if kind == "negative":
        return -(1.5 + base + 0.05 * rng.random(N))
    return base + 0.05 * rng.standard_normal(N)


@pytest.mark.parametrize("R", ORDERS)
@pytest.mark.parametrize("kind", ["positive", "negative", "mixed"])
@pytest.mark.parametrize("N,bc", [(1000, 0), (531, 1)])
def test_burgers_rhs(E, R, kind, N, bc):
    u = _field(kind, N, R)
    h = 1.0 / N
    s = E.Solver(E.BURGERS, N, order=R, dx=h, bc=bc)
    ud = dev(u)
    sel = s.selection(ud).cpu().numpy().reshape(2, N + 1)
    ref = oracle.rhs_burgers(u, h, R, bc=bc, want_sel=True, want_win=True)
    assert_selection(R, sel, ref["sel"], ref["win"], f"burgers R={R} {kind}")
    T = oracle.num_tested(R)
    if kind == "positive":
        assert (sel[1] == T + 2).all()  # f^- = 0
    if kind == "negative":
        assert (sel[0] == T + 2).all()  # f^+ = 0
    forced = oracle.rhs_burgers(u, h, R, bc=bc, forced=sel.reshape(-1))
    got = s.rhs(ud).cpu().numpy()
    assert_values(got, forced["rhs"], 0.5 * np.abs(u).max() ** 2 / h, f"burgers R={R} {kind}")
    s.check_status()


TABLE8 = [r for r in read_golden("burgers_errors_table_8.txt") if 64 <= int(r.split()[1]) <= 128]


@pytest.mark.parametrize("row", TABLE8)
def test_burgers_table_8_on_gpu(E, row):
    p = row.split()
    R, hinv, l1p, lip = int(p[0]), int(p[1]), float(p[2]), float(p[3])
    n = 2 * hinv
    u0, h = wl.burgers_sine3(n)
    t = 0.1
    steps = dt_schedule(R, h, t)
    P = oracle.Problem(oracle.EQ_BURGERS, R, n, dx=h, bc=oracle.BC_PERIODIC)
    ref = u0.copy()
    for dt in steps:
        ref = P.step_ssprk3(ref, dt)
    s = E.Solver(E.BURGERS, n, order=R, dx=h, bc=E.PERIODIC)
    ud = dev(u0)
    for dt in steps:
        s.step(ud, dt=dt)
    got = ud.cpu().numpy()
    s.check_status()
    assert np.abs(got - ref).mean() <= 1e-10
    l1, li = errors(got, h, t)
    print(f"GPU R={R} h=1/{hinv}: L1 {l1:.3e} (paper {l1p:.2e}), Linf {li:.3e} (paper {lip:.2e})")
    assert abs(l1 / l1p - 1.0) <= 0.02 and abs(li / lip - 1.0) <= 0.02


@pytest.mark.parametrize("R", [5, 9, 13, 17])
def test_burgers_shock_final_state(E, R):
    """Sec. 4.2's second run: h = 1/64, CFL 0.3, to t = 2 (a shock at the
    centre); the dt sequence of the oracle's own CFL run on both sides."""
    n = 128
    u0, h = wl.burgers_sine3(n)
    P = oracle.Problem(oracle.EQ_BURGERS, R, n, dx=h, bc=oracle.BC_PERIODIC)
    steps, ref, t = [], u0.copy(), 0.0
    while t < 2.0:
        dt = min(P.cfl_dt(ref, 0.3), 2.0 - t)
        ref = P.step_ssprk3(ref, dt)
        steps.append(dt)
        t += dt
    ref2, tol, env = shock_gate(P.step_ssprk3, u0, steps, seeds=(1,))
    assert np.array_equal(ref, ref2)
    s = E.Solver(E.BURGERS, n, order=R, dx=h, bc=E.PERIODIC)
    ud = dev(u0)
    for dt in steps:
        s.step(ud, dt=dt)
    got = ud.cpu().numpy()
    l1 = np.abs(got - ref).mean()
    print(f"burgers shock R={R}: L1(gpu-oracle) = {l1:.3e}, oracle envelope {env:.3e}")
    assert l1 <= tol
    # no new extrema across the shock beyond the initial range (ENO)
    assert got.max() <= u0.max() + 1e-3 and got.min() >= u0.min() - 1e-3
    s.check_status()


def test_burgers_cfl_step_matches_oracle(E):
    u0, h = wl.burgers_sine3(300)
    P = oracle.Problem(oracle.EQ_BURGERS, 9, 300, dx=h, bc=oracle.BC_PERIODIC)
    s = E.Solver(E.BURGERS, 300, order=9, dx=h, bc=E.PERIODIC)
    ud = dev(u0)
    dt = s.step(ud, 0.0, 0.5, return_dt=True)
    assert dt == pytest.approx(P.cfl_dt(u0, 0.5), rel=1e-15)
    ref = P.step_ssprk3(u0, dt)
    assert np.abs(ud.cpu().numpy() - ref).max() <= 1e-13
    s.check_status()


def test_burgers_zero_and_nan(E):
    import torch
    s = E.Solver(E.BURGERS, 400, order=7, dx=0.01, bc=E.PERIODIC)
    z = torch.zeros(400, dtype=torch.float64, device="cuda")
    assert torch.count_nonzero(s.rhs(z)) == 0
    assert s.step(z, 0.0, 0.5, return_dt=True) == 0.0
    assert torch.count_nonzero(z) == 0
    s.check_status()
    bad = torch.ones(400, dtype=torch.float64, device="cuda")
    bad[123] = float("nan")
    s.rhs(bad)
    with pytest.raises(E.EnomrError):
        s.check_status()


def test_burgers_rejects_adjoint_and_2d(E):
    import torch
    s = E.Solver(E.BURGERS, 64, order=5, dx=0.1, bc=E.PERIODIC)
    u = torch.ones(64, dtype=torch.float64, device="cuda")
    with pytest.raises(E.EnomrError):
        s.rhs_vjp(u, u.clone())
    with pytest.raises(E.EnomrError):
        E.Solver(E.BURGERS, (32, 32), order=5, dx=0.1)
