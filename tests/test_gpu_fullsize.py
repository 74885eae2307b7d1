"""Parity at the full sizes the benchmark runs, in the benchmark's launch
configuration (the public API with the library's fixed tile shapes).

The oracle evaluates every output here (its OpenMP loops make a 4096^2 RHS
take seconds); values are compared with the oracle re-run on the CUDA
path's selections, and every selection flip is classified as a near-tie
(tests/parity.py) and counted.
"""
import numpy as np
import pytest

import oracle
from parity import (assert_selection, assert_values, classify_euler2d_flips, euler_flux_scale,
                    euler_scale_fn)
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


def test_riemann2d_4096_order9(E):
    """The benchmark workload: four-quadrant Riemann problem, 4096^2,
    order 9, transmissive; checked after two CFL steps (smeared fronts)."""
    import torch
    n, R = 4096, 9
    U0, dx, dy = wl.riemann2d(n, n, seed=0)
    s = E.Solver(E.EULER, (n, n), order=R, dx=dx, dy=dy, bc=E.TRANSMISSIVE)
    Ud = torch.from_numpy(U0).cuda()
    for _ in range(2):
        s.step(Ud, 0.0, 0.5)
    U = Ud.cpu().numpy()
    sel = s.selection(Ud).cpu().numpy()
    got = s.rhs(Ud).cpu().numpy()
    s.check_status()
    ref_sel = oracle.rhs_euler2d(U, dx, dy, R, bc=oracle.BC_TRANSMISSIVE, want_sel=True)["sel"]
    n_fl, n_tie, worst = classify_euler2d_flips(U, dx, dy, R, oracle.BC_TRANSMISSIVE, sel,
                                                ref_sel)
    print(f"4096^2: selection flips {n_fl} of {sel.size}, {n_tie} near-ties "
          f"(worst relative distance {worst:.2e})")
    assert n_fl == n_tie, f"{n_fl - n_tie} flips that are not near-ties (worst {worst:.2e})"
    assert n_fl <= 1e-3 * sel.size
    forced = oracle.rhs_euler2d(U, dx, dy, R, bc=oracle.BC_TRANSMISSIVE, forced=sel)["rhs"]
    assert_values(got, forced, euler_flux_scale(U) / dx, "4096^2 riemann")


@pytest.mark.parametrize("R", [5, 9, 17])
def test_advection_2p24(E, R):
    import torch
    N = 1 << 24
    u, h = wl.advection_sine(N)
    u = u + 0.5 * (np.abs(np.arange(N) - N // 3) < N // 7)  # add two jumps
    s = E.Solver(E.ADVECTION, N, order=R, dx=h, bc=E.PERIODIC)
    ud = torch.from_numpy(u).cuda()
    sel = s.selection(ud).cpu().numpy()
    got = s.rhs(ud).cpu().numpy()
    ref = oracle.rhs_advection(u, h, R, want_sel=True)
    rs = ref["sel"].reshape(-1)
    flips = np.nonzero(rs != sel)[0]
    print(f"advection 2^24 R={R}: {flips.size} flips")
    assert flips.size <= 1e-6 * sel.size
    if flips.size:
        # a = 1 > 0: f^+ = u, f^- = 0; the f^+ window of interface k (entry k
        # of side 0) is u at cells k-1+l, so the f^- windows cannot flip
        assert (flips < N + 1).all()
        g = (R + 1) // 2
        cells = (flips[:, None] - 1 + np.arange(-(g - 1), g)[None, :]) % N
        assert_selection(R, sel[flips], rs[flips], u[cells], f"advection 2^24 R={R}")
    forced = oracle.rhs_advection(u, h, R, forced=sel)["rhs"]
    assert_values(got, forced, np.abs(u).max() / h, f"advection 2^24 R={R}")


@pytest.mark.parametrize("R", [5, 9, 17])
def test_burgers_2p24(E, R):
    """Burgers at the throughput size (N = 2^24, [0, 2] periodic,
    u0 = 1 + 0.5 sin^3(pi x) advanced 3 CFL steps).  u' has double zeros at
    x = 0 and 1, where the indicators of hundreds of cells are at rounding
    level; every flip is classified as a near-tie on its window (u > 0, so
    the f^+ windows are f = u^2/2 at consecutive cells, as the oracle forms
    them)."""
    import torch
    N = 1 << 24
    u, h = wl.burgers_sine3(N)
    s = E.Solver(E.BURGERS, N, order=R, dx=h, bc=E.PERIODIC)
    ud = torch.from_numpy(u).cuda()
    for _ in range(3):
        s.step(ud, 0.0, 0.5)
    u = ud.cpu().numpy()
    assert u.min() > 0
    sel = s.selection(ud).cpu().numpy()
    got = s.rhs(ud).cpu().numpy()
    s.check_status()
    ref = oracle.rhs_burgers(u, h, R, want_sel=True)
    rs = ref["sel"].reshape(-1)
    flips = np.nonzero(rs != sel)[0]
    print(f"burgers 2^24 R={R}: {flips.size} flips")
    assert flips.size <= 1e-3 * sel.size
    assert (flips < N + 1).all()  # f^- = 0: its windows cannot flip
    if flips.size:
        g = (R + 1) // 2
        f = 0.5 * (u * u)
        cells = (flips[:, None] - 1 + np.arange(-(g - 1), g)[None, :]) % N
        assert_selection(R, sel[flips], rs[flips], f[cells], f"burgers 2^24 R={R}")
    forced = oracle.rhs_burgers(u, h, R, forced=sel)["rhs"]
    assert_values(got, forced, 0.5 * np.abs(u).max() ** 2 / h, f"burgers 2^24 R={R}")


@pytest.mark.parametrize("R", [5, 17])
def test_euler1d_6400(E, R):
    import torch
    U, h = wl.shock_entropy(6400)
    s = E.Solver(E.EULER, 6400, order=R, dx=h, bc=E.TRANSMISSIVE)
    Ud = torch.from_numpy(U).cuda()
    for _ in range(3):
        s.step(Ud, 0.0, 0.5)
    U = Ud.cpu().numpy()
    sel = s.selection(Ud).cpu().numpy()
    got = s.rhs(Ud).cpu().numpy()
    ref = oracle.rhs_euler1d(U, h, R, want_sel=True, want_win=True)
    fn = euler_scale_fn(lambda line: U.T.copy(), 1, 6400, R, 1, lambda line: ref["alpha"])
    nflip = assert_selection(R, sel, ref["sel"], ref["win"], f"euler1d 6400 R={R}", fn)
    print(f"euler1d 6400 R={R}: {nflip} flips, all near-ties")
    forced = oracle.rhs_euler1d(U, h, R, forced=sel)["rhs"]
    assert_values(got, forced, euler_flux_scale(U) / h, f"euler1d 6400 R={R}")


def test_batch_4096_sample_vs_oracle(E):
    """The batched workload (4096 problems, sizes log-uniform in
    [128, 8192], order 9): one persistent-kernel step; 24 problems spread
    over the size range against the oracle."""
    import torch
    sizes, Us, hs = wl.riemann_batch(4096, seed=0)
    B = E.Batch(sizes, hs, order=9, bc=E.TRANSMISSIVE)
    Ub = B.pack(Us)
    B.autotune(Ub, reps=1)
    B.step(Ub, 0.5)
    B.check_status()
    order = np.argsort(sizes)
    for p in order[np.linspace(0, len(sizes) - 1, 24).astype(int)]:
        P = oracle.Problem(oracle.EQ_EULER1D, 9, int(sizes[p]), dx=float(hs[p]),
                           bc=oracle.BC_TRANSMISSIVE)
        ref = P.step_ssprk3(Us[p], P.cfl_dt(Us[p], 0.5))
        got = B.view(Ub, p).cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max(), int(p)


def test_adjoint_vortex_512_vs_frozen_oracle(E):
    """The adjoint workload's grid (512^2 isentropic vortex, order 9, moved
    off the grid's symmetry axes): RHS transpose product against the
    frozen-choice oracle."""
    import torch
    n, R = 512, 9
    U, h, _ = wl.isentropic_vortex(n, centre=(5.0 + 0.37 * 10 / n, 5.0 - 0.21 * 10 / n))
    s = E.Solver(E.EULER, (n, n), order=R, dx=h, dy=h, bc=E.PERIODIC)
    Ud = torch.from_numpy(U).cuda()
    sel = s.selection(Ud).cpu().numpy()
    _, am = oracle.rhs_euler2d_frozen(U, h, h, R, sel, bc=0)
    rng = np.random.Generator(np.random.PCG64(3))
    d = rng.standard_normal(U.shape) * (np.abs(U) + 0.1)
    v = rng.standard_normal(U.shape)
    eps = 1e-6
    jd = (oracle.rhs_euler2d_frozen(U + eps * d, h, h, R, sel, amax=am, bc=0)
          - oracle.rhs_euler2d_frozen(U - eps * d, h, h, R, sel, amax=am, bc=0)) / (2 * eps)
    lhs = float((v * jd).sum())
    rhs = float((s.rhs_vjp(Ud, torch.from_numpy(v).cuda()).cpu().numpy() * d).sum())
    assert abs(lhs - rhs) <= 1e-7 * float(np.abs(v * jd).sum()), (lhs, rhs)
