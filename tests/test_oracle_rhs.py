"""Pins for the oracle's right-hand sides and time integrators.

- Values printed in the paper: Tables 5-7 (advection errors, Sec. 4.1).
- Scale invariance of the whole scheme (Sec. 4.1: lam = 1e6 errors are the
  lam = 1 errors times 1e6).
- Designed order on smooth periodic data, SSP-RK3 with dt ~ h^(R/3).
- Discrete conservation of Eq. (1DWENOFD); constant states are steady.
- Euler eigen-system: L R = I and the Roe property
  R diag(lambda) L (U_R - U_L) = F(U_R) - F(U_L).
- 2D -> 1D reduction for data constant in y.
- SSP-RK3 and linear SSP-RK reproduce their stability polynomials.
"""
import math

import numpy as np
import pytest

import oracle
from conftest import read_golden
from paper_2311_15504_gb300 import workloads as wl

ORDERS = [5, 7, 9, 11, 13, 15, 17]


def advect_lssp(R, N, power, lam):
    u0, h = wl.advection_sine(N, power, lam)
    P = oracle.Problem(oracle.EQ_ADVECTION, R, N, dx=h, bc=oracle.BC_PERIODIC, a=1.0)
    u = u0.copy()
    for _ in range(int(round(2.0 / h))):
        u = P.step_lssp(u, h, R + 1)
    e = np.abs(u - u0)
    # nodes x_j, j = 1..N+1 of Sec. 2.1: the periodic endpoint counted twice
    return (e.sum() + e[0]) / (N + 1), e.max()


@pytest.mark.parametrize("row", read_golden("advection_errors_tables_5_7.txt"))
def test_paper_advection_errors(row):
    parts = row.split()
    R, N, power = int(parts[0]), int(parts[1]), int(parts[2])
    lam, l1p, lip = float(parts[3]), float(parts[4]), float(parts[5])
    l1, li = advect_lssp(R, N, power, lam)
    # three printed digits; errors near 1e-12 also carry FP64 round-off
    tol = 0.006 if l1p / lam > 1e-11 else 0.01
    assert abs(l1 - l1p) <= tol * l1p, (l1, l1p)
    assert abs(li - lip) <= tol * lip, (li, lip)


def test_scale_invariance_of_scheme():
    for R, N in [(5, 200), (9, 100), (17, 30)]:
        a = advect_lssp(R, N, 4, 1.0)
        b = advect_lssp(R, N, 4, 1e6)
        assert b[0] == pytest.approx(1e6 * a[0], rel=1e-7)
        assert b[1] == pytest.approx(1e6 * a[1], rel=1e-7)


@pytest.mark.parametrize("R,Ns", [(5, [25, 50, 100]), (7, [25, 50, 100]), (9, [20, 40])])
def test_ssprk3_convergence_order(R, Ns):
    """Smooth sin(pi x), SSP-RK3 with dt = 0.5 h (h/h0)^(R/3-1): the time
    error O(dt^3) matches the space error O(h^R)."""
    errs = []
    h0 = 2.0 / Ns[0]
    for N in Ns:
        u0, h = wl.advection_sine(N)
        dt = 0.5 * h * (h / h0) ** (R / 3.0 - 1.0)
        P = oracle.Problem(oracle.EQ_ADVECTION, R, N, dx=h, bc=oracle.BC_PERIODIC)
        nsteps = int(math.ceil(2.0 / dt - 1e-9))
        dt = 2.0 / nsteps
        u = u0.copy()
        for _ in range(nsteps):
            u = P.step_ssprk3(u, dt)
        errs.append(np.abs(u - u0).mean())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert min(orders) > R - 0.6, orders


@pytest.mark.parametrize("R", ORDERS)
def test_advection_conservation_and_constant(R):
    rng = np.random.Generator(np.random.PCG64(R))
    N = 64
    u = rng.standard_normal(N)
    r = oracle.rhs_advection(u, 0.1, R)["rhs"]
    assert abs(r.sum()) <= N * 1e-14 * np.abs(u).max() / 0.1 * 50
    assert np.all(oracle.rhs_advection(np.full(N, 2.5), 0.1, R)["rhs"] == 0)
    # negative speed: the mirrored f^- path carries the flux
    r1 = oracle.rhs_advection(u, 0.1, R, a=-1.0)["rhs"]
    r2 = oracle.rhs_advection(u[::-1].copy(), 0.1, R, a=1.0)["rhs"]
    assert np.array_equal(r1, r2[::-1])


def _rand_state(rng, c):
    rho = rng.uniform(0.1, 2.0)
    u = rng.uniform(-1, 1, size=c - 2)
    p = rng.uniform(0.1, 5.0)
    if c == 3:
        return wl.conserved_1d(np.array([rho]), u[0], p)[:, 0]
    return wl.conserved_2d(np.array([rho]), u[0], u[1], p)[:, 0]


def _flux(U, gamma=1.4):
    c = U.shape[0]
    rho, un = U[0], U[1] / U[0]
    ut = U[2] / U[0] if c == 4 else 0.0
    p = (gamma - 1) * (U[-1] - 0.5 * rho * (un * un + ut * ut))
    F = [U[1], U[1] * un + p] + ([U[2] * un] if c == 4 else []) + [(U[-1] + p) * un]
    return np.array(F)


@pytest.mark.parametrize("c", [3, 4])
def test_roe_eigensystem(c):
    rng = np.random.Generator(np.random.PCG64(7 + c))
    for _ in range(50):
        UL, UR = _rand_state(rng, c), _rand_state(rng, c)
        Rm, Lm, lam = oracle.euler_eigen(UL, UR)
        assert np.abs(Lm @ Rm - np.eye(c)).max() < 1e-12
        lhs = Rm @ np.diag(lam) @ Lm @ (UR - UL)
        rhs = _flux(UR) - _flux(UL)
        assert np.abs(lhs - rhs).max() <= 1e-11 * (1 + np.abs(rhs).max())
        # consistency: at UL == UR the Roe matrix is the flux Jacobian
        Rm2, Lm2, lam2 = oracle.euler_eigen(UL, UL)
        eps = 1e-7 * (1 + np.abs(UL).max())
        J = np.stack([(_flux(UL + eps * e) - _flux(UL - eps * e)) / (2 * eps)
                      for e in np.eye(c)], axis=1)
        assert np.abs(Rm2 @ np.diag(lam2) @ Lm2 - J).max() < 1e-6 * (1 + np.abs(J).max())


@pytest.mark.parametrize("R", [5, 9, 17])
def test_euler_constant_state_is_steady(R):
    U1 = wl.conserved_1d(np.full(40, 0.7), 0.3, 1.2)
    for bc in (oracle.BC_PERIODIC, oracle.BC_TRANSMISSIVE):
        assert np.all(oracle.rhs_euler1d(U1, 0.05, R, bc=bc)["rhs"] == 0)
    U2 = wl.conserved_2d(np.full((24, 20), 0.7), 0.3, -0.2, 1.2)
    assert np.all(oracle.rhs_euler2d(U2, 0.05, 0.04, R, bc=oracle.BC_TRANSMISSIVE)["rhs"] == 0)


@pytest.mark.parametrize("R", [5, 9, 13, 17])
def test_euler_conservation_periodic(R):
    U, h = wl.density_wave_1d(64)
    U = U + 0.05 * np.random.Generator(np.random.PCG64(R)).standard_normal(U.shape) * np.array(
        [[1], [0], [1]])
    r = oracle.rhs_euler1d(U, h, R, bc=oracle.BC_PERIODIC)["rhs"]
    assert np.abs(r.sum(axis=1)).max() <= 1e-11 / h
    U2 = wl.smooth_random_euler2d(36, 40, seed=R)
    r2 = oracle.rhs_euler2d(U2, 0.1, 0.1, R, bc=oracle.BC_PERIODIC)["rhs"]
    assert np.abs(r2.sum(axis=(1, 2))).max() <= 1e-10 / 0.1


@pytest.mark.parametrize("R", [5, 9, 17])
def test_2d_reduces_to_1d(R):
    """Data constant in y with v = 0: the y sweep sees constant columns,
    so IS_0 = 0 everywhere, minmod returns f_j and the y flux differences
    vanish exactly; the x sweep is the 1D scheme with a passive
    component."""
    U1, h = wl.shock_entropy(80)
    ny = 2 * ((R + 1) // 2) + 1
    U2 = np.zeros((4, ny, 80))
    U2[0], U2[1], U2[3] = U1[0], U1[1], U1[2]
    r1 = oracle.rhs_euler1d(U1, h, R, bc=oracle.BC_TRANSMISSIVE, want_sel=True)
    r2 = oracle.rhs_euler2d(U2, h, 0.1, R, bc=oracle.BC_TRANSMISSIVE, want_sel=True)
    scale = np.abs(r1["rhs"]).max()
    for q1, q2 in ((0, 0), (1, 1), (2, 3)):
        assert np.abs(r2["rhs"][q2] - r1["rhs"][q1][None, :]).max() <= 1e-12 * scale
    assert np.abs(r2["rhs"][2]).max() <= 1e-12 * scale
    T = oracle.num_tested(R)
    assert np.all(r2["sel_y"] == T + 2)
    # acoustic/entropy fields of the x sweep select like the 1D scheme
    for fx, f1 in ((0, 0), (1, 1), (3, 2)):
        same = (r2["sel_x"][:, fx] == r1["sel"][:, f1][:, None, :]).mean()
        assert same > 0.99


@pytest.mark.parametrize("R", [5, 9])
def test_euler_density_wave_order(R):
    errs = []
    Ns = [24, 48] if R == 9 else [32, 64, 128]
    for N in Ns:
        U0, h = wl.density_wave_1d(N)
        P = oracle.Problem(oracle.EQ_EULER1D, R, N, dx=h, bc=oracle.BC_PERIODIC)
        t_end = 0.5
        dt = 0.2 * h * (h / (2.0 / Ns[0])) ** (R / 3.0 - 1.0)
        n = int(math.ceil(t_end / dt))
        dt = t_end / n
        U = U0.copy()
        for _ in range(n):
            U = P.step_ssprk3(U, dt)
        x, _ = wl.periodic_grid(-1.0, 1.0, N)
        errs.append(np.abs(U[0] - (1 + 0.2 * np.sin(np.pi * (x - t_end)))).mean())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert min(orders) > R - 0.8, (errs, orders)


def test_forced_selection_reproduces_rhs():
    u, h = wl.advection_step(64)
    o = oracle.rhs_advection(u, h, 9, want_sel=True)
    f = oracle.rhs_advection(u, h, 9, forced=o["sel"])
    assert np.array_equal(o["rhs"], f["rhs"])
    U, h = wl.shock_entropy(60)
    o = oracle.rhs_euler1d(U, h, 13, want_sel=True)
    f = oracle.rhs_euler1d(U, h, 13, forced=o["sel"])
    assert np.array_equal(o["rhs"], f["rhs"])
    U2, dx, dy = wl.riemann2d(20, 18, seed=3)
    o = oracle.rhs_euler2d(U2, dx, dy, 9, want_sel=True)
    f = oracle.rhs_euler2d(U2, dx, dy, 9, forced=o["sel"])
    assert np.array_equal(o["rhs"], f["rhs"])
    # forcing a different (valid) stencil changes the result
    g = o["sel"].copy()
    g[:] = 0
    assert not np.array_equal(oracle.rhs_euler2d(U2, dx, dy, 9, forced=g)["rhs"], o["rhs"])


def test_nonphysical_state_raises():
    U = wl.conserved_1d(np.full(20, 1.0), 0.0, 1.0)
    U[0, 5] = -1.0
    with pytest.raises(oracle.OracleError):
        oracle.rhs_euler1d(U, 0.1, 5)


def test_ssprk3_is_third_order_taylor_on_linear_operator():
    """For data where every stage keeps the top stencil the advection RHS
    is a fixed matrix M; one SSP-RK3 step must equal
    (I + dt M + dt^2 M^2/2 + dt^3 M^3/6) u (Eq. TVD3rdRK)."""
    R, N = 5, 32
    u, h = wl.advection_sine(N)
    sel = oracle.rhs_advection(u, h, R, want_sel=True)["sel"]
    assert np.all(sel[0] == 0)
    forced = np.zeros(2 * (N + 1), dtype=np.uint8)
    M = np.stack([oracle.rhs_advection(e, h, R, forced=forced)["rhs"] for e in np.eye(N)], axis=1)
    dt = 0.4 * h
    P = oracle.Problem(oracle.EQ_ADVECTION, R, N, dx=h, bc=oracle.BC_PERIODIC)
    got = P.step_ssprk3(u, dt)
    A = dt * M
    want = u + A @ u + A @ (A @ u) / 2 + A @ (A @ (A @ u)) / 6
    assert np.abs(got - want).max() < 1e-13


@pytest.mark.parametrize("m", list(range(2, 19)))
def test_lssp_stability_polynomial(m):
    """Eq. (lSSPRK): u^{n+1} = [sum_{k<m-1} a_k (1+z/2)^k + a_{m-1}(1+z/2)^m] u^n
    must agree with exp(z) through z^{m-1}."""
    a = oracle.lssp_coeffs(m)
    assert abs(a.sum() - 1.0) < 1e-14 and np.all(a >= -1e-15)
    poly = np.zeros(m + 1)
    for k in range(m):
        p = k if k < m - 1 else m
        for i in range(p + 1):
            poly[i] += a[k] * math.comb(p, i) * 0.5 ** i
    for i in range(m):
        assert poly[i] == pytest.approx(1.0 / math.factorial(i), rel=1e-12), (m, i)


def test_lssp_coefficients_small_m_exact():
    """alpha_{3,*} = (1/3, 0, 2/3); alpha_{4,*} = (0, 2/3, 0, 1/3)."""
    assert oracle.lssp_coeffs(3) == pytest.approx([1 / 3, 0, 2 / 3], abs=3e-16)
    assert oracle.lssp_coeffs(4) == pytest.approx([0, 2 / 3, 0, 1 / 3], abs=3e-16)
    assert oracle.lssp_coeffs(2).tolist() == [0.0, 1.0]


@pytest.mark.parametrize("R", [5, 13])
def test_euler2d_transpose_symmetry(R):
    """Exchanging x and y (transposing the grid, swapping the momenta and the
    spacings) transposes the right-hand side with its momenta swapped: the y
    sweep is the x sweep of the transposed problem.  Bit for bit, since the
    oracle takes the same operations on either axis; a wrong index or
    component in one sweep breaks it."""
    rng = np.random.Generator(np.random.PCG64(R))
    ny, nx = 23, 31
    U = wl.conserved_2d(0.5 + rng.random((ny, nx)), rng.uniform(-1, 1, (ny, nx)),
                        rng.uniform(-1, 1, (ny, nx)), 0.5 + rng.random((ny, nx)))
    U[:, 5:9, :] = U[:, 5:6, :]  # some flat windows too
    for bc in (oracle.BC_TRANSMISSIVE, oracle.BC_PERIODIC):
        a = oracle.rhs_euler2d(U, 0.1, 0.07, R, bc=bc, want_sel=True)
        V = U.transpose(0, 2, 1)[[0, 2, 1, 3]].copy()
        b = oracle.rhs_euler2d(V, 0.07, 0.1, R, bc=bc, want_sel=True)
        assert np.array_equal(b["rhs"], a["rhs"].transpose(0, 2, 1)[[0, 2, 1, 3]])
        assert np.array_equal(b["sel_x"], a["sel_y"]) and np.array_equal(b["sel_y"], a["sel_x"])


def test_rp1_rows_far_from_the_centre_evolve_as_the_1d_riemann_problem():
    """The paper's first 2D Riemann configuration (Sec. 4.4): away from the
    centre, each half-line interface is a 1D Riemann problem.  For y = 0.7 the
    states either side of x = 0, (0.5323, 1.206, 0, 0.3) | (1.5, 0, 0, 1.5),
    have v = 0.  The exact solution is a single left-moving shock (p* = 1.5
    and u* = 0 to 1e-5: the right state is the shocked left state), and
    nothing from y = 0 reaches the row in 20 short steps, so the 2D oracle's
    row follows its 1D scheme on the same data, step for step (same dt), to
    rounding, with its shock where the exact speed puts it."""
    from riemann_exact import star_state
    ps, us = star_state((0.5323, 1.206, 0.3), (1.5, 0.0, 1.5))
    assert abs(ps - 1.5) < 1e-5 and abs(us) < 1e-5
    n, R = 101, 9
    U, h, _ = wl.riemann2d_rp1(n)
    y = -1.0 + h * (np.arange(n) + 0.5)
    j = int(np.argmin(np.abs(y - 0.7)))
    row = U[:, j, :]
    U1 = np.stack([row[0], row[1], row[3]])
    dt, steps = 0.1 * h, 20
    P2 = oracle.Problem(oracle.EQ_EULER2D, R, n, n, dx=h, dy=h, bc=oracle.BC_TRANSMISSIVE)
    P1 = oracle.Problem(oracle.EQ_EULER1D, R, n, dx=h, bc=oracle.BC_TRANSMISSIVE)
    for _ in range(steps):
        U = P2.step_ssprk3(U, dt)
        U1 = P1.step_ssprk3(U1, dt)
    scale = np.abs(U1).max()
    assert np.abs(U[0, j] - U1[0]).max() <= 1e-12 * scale
    assert np.abs(U[1, j] - U1[1]).max() <= 1e-12 * scale
    assert np.abs(U[3, j] - U1[2]).max() <= 1e-12 * scale
    assert np.abs(U[2, j]).max() <= 1e-12 * scale
    # the shock: the largest density jump of the row, within a cell of
    # x = S t with the exact left-shock speed
    rl, ul, pl = 0.5323, 1.206, 0.3
    S = ul - np.sqrt(1.4 * pl / rl) * np.sqrt(2.4 / 2.8 * ps / pl + 0.4 / 2.8)
    x = -1.0 + h * (np.arange(n) + 0.5)
    k = int(np.argmax(np.abs(np.diff(U1[0]))))
    assert abs(0.5 * (x[k] + x[k + 1]) - S * steps * dt) <= h
