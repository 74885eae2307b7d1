"""Pins for the oracle's boundary sides and body force (the 2D problems of
Sec. 4.4: double Mach reflection, Rayleigh-Taylor).

- Reflective sides: the right-hand side on [0, L] equals, bit for bit, the
  restriction of the right-hand side of the mirror-extended problem on
  [-L, L] with periodic boundaries (mirror image: rho, E and the tangential
  momentum even, the normal momentum odd).
- Inflow sides, with a split moving along the side: equal, bit for bit, to
  the transmissive problem on a grid extended by g columns (rows) that hold
  the inflow states, on the original cells (the inflow states are chosen
  slower than the interior, so each line's alpha is attained inside).
- Transmissive sides given explicitly reproduce the plain scheme.
- Body force: on a constant state the right-hand side is exactly
  S = (0, rho gx, rho gy, rho u gx + rho v gy); on any state it adds S to
  rounding.
"""
import numpy as np
import pytest

import oracle
from paper_2311_15504_gb300 import workloads as wl

T, RF, IN = oracle.SIDE_TRANSMISSIVE, oracle.SIDE_REFLECTIVE, oracle.SIDE_INFLOW


def field(nx, ny, seed):
    U = wl.smooth_random_euler2d(nx, ny, seed=seed, amp=0.2)
    U = U + 0.02 * np.random.Generator(np.random.PCG64(seed)).standard_normal(U.shape) * [[[1.0]], [[0.3]], [[0.3]], [[1.0]]]
    return np.ascontiguousarray(U)


def mirror_x(V):
    """The mirror image about x = 0 of a state (normal momentum negated)."""
    M = V[:, :, ::-1].copy()
    M[1] *= -1.0
    return M


def mirror_y(V):
    M = V[:, ::-1, :].copy()
    M[2] *= -1.0
    return M


@pytest.mark.parametrize("R", [5, 9, 17])
def test_reflective_sides_are_a_mirror_extension(R):
    """The per-field alpha of a line is not invariant under a mirror image
    (|u - c| and |u + c| trade places), so the field is made mirror
    symmetric within the domain: then every line of the doubled domain has
    the alphas of the original line.  A wrong ghost index or a missing sign
    flip of the normal momentum fails the comparison."""
    g = (R + 1) // 2
    nx, ny = 2 * g + 3, 2 * g + 4
    V = field(nx, ny, R)
    U = np.concatenate([mirror_x(V), V], axis=2)            # symmetric about the x mid-line
    U = np.ascontiguousarray(np.concatenate([mirror_y(U), U], axis=1))  # and the y mid-line
    _, NY, NX = U.shape
    dx, dy = 0.013, 0.011
    rr = oracle.rhs_euler2d_ext(U, dx, dy, R, sides=(oracle.side(RF),) * 4)["rhs"]
    Q = np.concatenate([mirror_x(U), U], axis=2)
    Q = np.ascontiguousarray(np.concatenate([mirror_y(Q), Q], axis=1))
    full = oracle.rhs_euler2d(Q, dx, dy, R, bc=oracle.BC_PERIODIC)["rhs"]
    assert np.array_equal(rr, full[:, NY:, NX:])
    # reflective in x only (transmissive in y): a state constant in y, so
    # that the transmissive y sweep contributes nothing on either side
    Vy = np.ascontiguousarray(np.broadcast_to(U[:, :1, :], U.shape))
    a = oracle.rhs_euler2d_ext(Vy, dx, dy, R, sides=(oracle.side(RF), oracle.side(RF), None, None))["rhs"]
    Qy = np.ascontiguousarray(np.concatenate([mirror_x(Vy), Vy], axis=2))
    b = oracle.rhs_euler2d(Qy, dx, dy, R, bc=oracle.BC_PERIODIC)["rhs"]
    assert np.array_equal(a, b[:, :, NX:])


@pytest.mark.parametrize("R", [5, 9])
@pytest.mark.parametrize("t", [0.0, 0.37])
def test_inflow_sides_are_an_extended_grid(R, t):
    g = (R + 1) // 2
    nx, ny = 3 * g + 4, 2 * g + 6
    dx, dy = 0.02, 0.03
    rng = np.random.Generator(np.random.PCG64(3))
    # interior: c ~ 2.6 and |u|, |v| up to 0.1; inflow: c ~ 0.6 and |u|, |v| <= 0.05,
    # so every line's alpha is attained at an interior cell
    U = wl.conserved_2d(1.0 + 0.2 * rng.random((ny, nx)), 0.2 * rng.random((ny, nx)) - 0.1,
                        0.2 * rng.random((ny, nx)) - 0.1, 5.0 + 0.5 * rng.random((ny, nx)))
    U[1, 0, 0] = 0.1 * U[0, 0, 0]
    U[2, 0, 0] = -0.1 * U[0, 0, 0]
    A = wl.conserved_2d(np.array([2.0]), 0.05, 0.03, 0.5)[:, 0]
    B = wl.conserved_2d(np.array([1.8]), -0.04, 0.05, 0.45)[:, 0]
    y0, rate = 0.2, 0.5        # split along the left side at y = y0 + rate t
    x0, xrate = 0.15, -0.1     # split along the bottom at x = x0 + xrate t
    sides = (oracle.side(IN, A, IN, B, y0, rate), None,
             oracle.side(IN, B, IN, A, x0, xrate), None)
    r = oracle.rhs_euler2d_ext(U, dx, dy, R, sides=sides, t=t)["rhs"]
    # extended grid: g columns left (x < 0) and g rows below (y < 0)
    E = np.zeros((4, ny + g, nx + g))
    E[:, g:, g:] = U
    yc = (np.arange(ny) + 0.5) * dy
    xc = (np.arange(nx) + 0.5) * dx
    for j in range(ny):
        E[:, g + j, :g] = (A if yc[j] < y0 + rate * t else B)[:, None]
    for i in range(nx):
        E[:, :g, g + i] = (B if xc[i] < x0 + xrate * t else A)[:, None]
    E[:, :g, :g] = A[:, None, None]  # corner: never inside a window of the original cells
    e = oracle.rhs_euler2d(np.ascontiguousarray(E), dx, dy, R, bc=oracle.BC_TRANSMISSIVE)["rhs"]
    assert np.array_equal(r, e[:, g:, g:])


def test_explicit_transmissive_sides_and_zero_force_are_the_plain_scheme():
    U, dx, dy = wl.riemann2d(37, 23, seed=4)
    a = oracle.rhs_euler2d(U, dx, dy, 9)["rhs"]
    b = oracle.rhs_euler2d_ext(U, dx, dy, 9, sides=(oracle.side(T),) * 4, gravity=(0.0, 0.0))["rhs"]
    assert np.array_equal(a, b)


def test_body_force():
    gx, gy = 0.3, 1.0
    U = np.ascontiguousarray(np.broadcast_to(wl.conserved_2d(np.array([1.3]), 0.2, -0.4, 2.0)[:, 0][:, None, None],
                                             (4, 20, 24)))
    r = oracle.rhs_euler2d_ext(U, 0.1, 0.1, 9, gravity=(gx, gy))["rhs"]
    rho, mx, my = U[0], U[1], U[2]
    assert not r[0].any()
    assert np.array_equal(r[1], rho * gx)
    assert np.array_equal(r[2], rho * gy)
    assert np.array_equal(r[3], my * gy + mx * gx)
    V = field(30, 26, 9)
    d = (oracle.rhs_euler2d_ext(V, 0.1, 0.1, 9, gravity=(gx, gy))["rhs"]
         - oracle.rhs_euler2d_ext(V, 0.1, 0.1, 9)["rhs"])
    S = np.stack([0 * V[0], V[0] * gx, V[0] * gy, V[2] * gy + V[1] * gx])
    assert np.allclose(d, S, rtol=0, atol=1e-12 * 100)


def test_paper_2d_problem_setups():
    U, dx, dy, sides = wl.double_mach(120, 30)
    assert U.shape == (4, 30, 120) and abs(dx - 1 / 30) < 1e-15 and abs(dy - 1 / 30) < 1e-15
    assert sides[2][4] == pytest.approx(1 / 6)
    V, hx, hy, _ = wl.rayleigh_taylor(16, 64)
    assert V.shape == (4, 64, 16) and abs(hx - hy) < 1e-15


def test_double_mach_incident_shock_where_the_exact_solution_puts_it():
    """The double Mach reflection (Sec. 4.4) on 120 x 30 cells at CFL 0.1 to
    t = 0.05: away from the wall (y >= 0.3) the Mach 10 incident shock is
    the exact straight shock x = 1/6 + (y + 20 t)/sqrt(3), which the top
    side's moving split also follows.  The oracle's shock (the crossing of
    the mid density between the post- and pre-shock states) sits within one
    cell of it in every row, the gas well ahead of it is the pre-shock state
    and density and pressure stay positive."""
    kinds = {"transmissive": oracle.SIDE_TRANSMISSIVE, "reflective": oracle.SIDE_REFLECTIVE,
             "inflow": oracle.SIDE_INFLOW}
    nx, ny, R, T = 120, 30, 9, 0.05
    U, dx, dy, sides = wl.double_mach(nx, ny)
    pre = U[:, -1, -1].copy()
    sd = tuple(oracle.side(kinds[k0], s0, kinds[k1], s1, a, b) for k0, s0, k1, s1, a, b in sides)
    P = oracle.Problem(oracle.EQ_EULER2D, R, nx, ny, dx=dx, dy=dy, bc=oracle.BC_TRANSMISSIVE)
    t, n = 0.0, 0
    while t < T and n < 5000:
        dt = min(P.cfl_dt(U, 0.1), T - t)
        assert dt > 0.0
        U = oracle.step_euler2d_ext(U, dx, dy, R, dt, sides=sd, t=t)
        t += dt
        n += 1
    rho = U[0]
    p = 0.4 * (U[3] - 0.5 * (U[1] ** 2 + U[2] ** 2) / rho)
    assert rho.min() > 0 and p.min() > 0
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dy
    mid = 0.5 * (8.0 + 1.4)
    for j in np.nonzero(y >= 0.3)[0]:
        xs = 1.0 / 6.0 + (y[j] + 20.0 * T) / np.sqrt(3.0)
        i = np.nonzero(rho[j] > mid)[0].max()
        x_num = x[i] + dx * (rho[j, i] - mid) / (rho[j, i] - rho[j, i + 1])
        assert abs(x_num - xs) <= dx, (y[j], x_num, xs)
        # the captured shock is a few cells wide; its precursor decays by
        # about a decade per cell and is below 1e-9 twelve cells ahead
        ahead = x > xs + 12 * dx
        assert np.allclose(U[:, j, ahead], pre[:, None], rtol=0, atol=1e-8)


@pytest.mark.parametrize("R", [5, 9, 17])
def test_rayleigh_taylor_rest_state_is_hydrostatic(R):
    """The Rayleigh-Taylor set-up without its velocity perturbation is at
    rest in hydrostatic balance: p is linear in y with dp/dy = rho g, and
    the scheme reproduces linear data, so the pressure gradient cancels the
    body force (0, rho g) to rounding in every cell more than g + 1 cells
    from the density jump at y = 0.5 and from the inflow sides; the
    x-momentum right-hand side is exactly zero.  With the force's sign
    flipped the y-momentum right-hand side is 2 rho g there."""
    kinds = {"transmissive": oracle.SIDE_TRANSMISSIVE, "reflective": oracle.SIDE_REFLECTIVE,
             "inflow": oracle.SIDE_INFLOW}
    gamma = 5.0 / 3.0
    _, dx, dy, sides = wl.rayleigh_taylor(16, 128)
    sd = tuple(oracle.side(kinds[k0], s0, kinds[k1], s1, a, b) for k0, s0, k1, s1, a, b in sides)
    y = (np.arange(128) + 0.5) * dy
    rho = np.repeat(np.where(y < 0.5, 2.0, 1.0)[:, None], 16, axis=1)
    p = np.repeat(np.where(y < 0.5, 2.0 * y + 1.0, y + 1.5)[:, None], 16, axis=1)
    U = wl.conserved_2d(rho, 0.0, 0.0, p, gamma)
    g = (R + 1) // 2
    far = (np.abs(y - 0.5) > (g + 1) * dy) & (y > (g + 1) * dy) & (y < 1.0 - (g + 1) * dy)
    r = oracle.rhs_euler2d_ext(U, dx, dy, R, sides=sd, gravity=(0.0, 1.0), gamma=gamma)["rhs"]
    assert np.abs(r[:, far]).max() <= 1e-12 * p.max() / dy
    assert not np.any(r[1])
    flipped = oracle.rhs_euler2d_ext(U, dx, dy, R, sides=sd, gravity=(0.0, -1.0),
                                     gamma=gamma)["rhs"]
    assert np.allclose(flipped[2, far], -2.0 * rho[far], rtol=1e-12)
