"""Edge cases of the CUDA path against the oracle: the smallest periodic
lines (N = 2g: every window wraps around the line), one- to three-cell
transmissive lines (windows made of clamped ghosts), and 2D grids one
cell wide in either direction."""
import numpy as np
import pytest

import oracle
from parity import assert_selection, assert_values, euler_flux_scale
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


@pytest.mark.parametrize("R", ORDERS)
def test_smallest_periodic_lines(E, R):
    g = (R + 1) // 2
    N = 2 * g
    rng = np.random.Generator(np.random.PCG64(R))
    h = 1.0 / N
    # advection and Burgers
    u = 1.0 + 0.5 * rng.random(N)
    for eq, ref_fn in ((E.ADVECTION, lambda w, **k: oracle.rhs_advection(w, h, R, **k)),
                       (E.BURGERS, lambda w, **k: oracle.rhs_burgers(w, h, R, **k))):
        s = E.Solver(eq, N, order=R, dx=h, bc=E.PERIODIC)
        ud = dev(u)
        sel = s.selection(ud).cpu().numpy()
        ref = ref_fn(u, want_sel=True, want_win=True)
        assert_selection(R, sel.reshape(2, N + 1), ref["sel"], ref["win"], f"N=2g R={R}")
        got = s.rhs(ud).cpu().numpy()
        assert_values(got, ref_fn(u, forced=sel)["rhs"], np.abs(u).max() ** 2 / h, f"N=2g R={R}")
        s.check_status()
    # 1D Euler: a density wave on the shortest line
    U, _ = wl.density_wave_1d(N)
    s = E.Solver(E.EULER, N, order=R, dx=h, bc=E.PERIODIC)
    Ud = dev(U)
    sel = s.selection(Ud).cpu().numpy()
    got = s.rhs(Ud).cpu().numpy()
    forced = oracle.rhs_euler1d(U, h, R, bc=oracle.BC_PERIODIC, forced=sel)["rhs"]
    assert_values(got, forced, euler_flux_scale(U) / h, f"euler1d N=2g R={R}")
    s.check_status()


@pytest.mark.parametrize("R", [5, 9, 17])
@pytest.mark.parametrize("N", [1, 2, 3])
def test_tiny_transmissive_lines(E, R, N):
    h = 0.1
    rng = np.random.Generator(np.random.PCG64(10 * R + N))
    U = wl.conserved_1d(rng.uniform(0.5, 1.5, N), rng.uniform(-0.5, 0.5, N),
                        rng.uniform(0.5, 1.5, N))
    s = E.Solver(E.EULER, N, order=R, dx=h, bc=E.TRANSMISSIVE)
    Ud = dev(U)
    sel = s.selection(Ud).cpu().numpy()
    ref = oracle.rhs_euler1d(U, h, R, bc=oracle.BC_TRANSMISSIVE, want_sel=True)
    assert np.array_equal(sel.reshape(ref["sel"].shape), ref["sel"])
    got = s.rhs(Ud).cpu().numpy()
    assert_values(got, ref["rhs"], euler_flux_scale(U) / h, f"euler1d N={N}")
    if N == 1:
        assert np.count_nonzero(got) == 0  # a single cell with clamped ghosts is steady
    u = np.linspace(1.0, 2.0, N)
    sa = E.Solver(E.ADVECTION, N, order=R, dx=h, bc=E.TRANSMISSIVE)
    ra = oracle.rhs_advection(u, h, R, bc=oracle.BC_TRANSMISSIVE)["rhs"]
    assert_values(sa.rhs(dev(u)).cpu().numpy(), ra, 2.0 / h, f"advection N={N}")
    s.check_status()
    sa.check_status()


@pytest.mark.parametrize("shape", [(1, 37), (37, 1), (2, 130), (130, 3)])
def test_one_cell_wide_2d_grids(E, shape):
    ny, nx = shape
    R = 9
    U, dx, dy = wl.riemann2d(nx, ny, seed=3, xc=0.5, yc=0.5)
    s = E.Solver(E.EULER, (ny, nx), order=R, dx=dx, dy=dy, bc=E.TRANSMISSIVE)
    Ud = dev(U)
    sel = s.selection(Ud).cpu().numpy()
    ref = oracle.rhs_euler2d(U, dx, dy, R, bc=oracle.BC_TRANSMISSIVE, want_sel=True)
    assert np.array_equal(sel, ref["sel"].reshape(-1))
    got = s.rhs(Ud).cpu().numpy()
    forced = oracle.rhs_euler2d(U, dx, dy, R, bc=oracle.BC_TRANSMISSIVE, forced=sel)["rhs"]
    assert_values(got, forced, euler_flux_scale(U) / min(dx, dy), f"2d {shape}")
    s.check_status()


@pytest.mark.parametrize("R", [5, 9, 17])
@pytest.mark.parametrize("bc", [0, 1])
def test_uniform_state_is_steady(E, R, bc):
    """A uniform state is a steady solution.  Every interface is flat with
    equal centre states, both sides take S(0,0) and the flux R (f^+ + f^-)
    is F(U) (exactly so on the GPU, which takes the cell's own flux there),
    so the RHS is exactly zero on the GPU and zero up to rounding in the
    oracle; one step keeps the state to within an ulp (the SSP-RK3 weights
    round)."""
    import torch
    g = (R + 1) // 2
    for ndim in (1, 2):
        if ndim == 1:
            N = max(3 * g, 40)
            U = wl.conserved_1d(np.full(N, 1.3), np.full(N, 0.4), np.full(N, 2.1))
            s = E.Solver(E.EULER, N, order=R, dx=0.1, bc=bc)
            ref = oracle.rhs_euler1d(U, 0.1, R, bc=bc, want_sel=True)
        else:
            ny, nx = 70, 130
            U = wl.conserved_2d(np.full((ny, nx), 1.3), 0.4, -0.7, 2.1)
            s = E.Solver(E.EULER, (ny, nx), order=R, dx=0.1, dy=0.2, bc=bc)
            ref = oracle.rhs_euler2d(U, 0.1, 0.2, R, bc=bc, want_sel=True)
        Ud = dev(U)
        sel = s.selection(Ud).cpu().numpy()
        T = oracle.num_tested(R)
        assert (sel == T + 2).all() and (ref["sel"] == T + 2).all()
        rhs = s.rhs(Ud)
        assert torch.count_nonzero(rhs) == 0
        assert_values(rhs.cpu().numpy(), ref["rhs"], euler_flux_scale(U) / 0.1, "uniform")
        s.step(Ud, dt=0.01)
        assert np.abs(Ud.cpu().numpy() - U).max() <= 2e-16 * np.abs(U).max()
        s.check_status()
