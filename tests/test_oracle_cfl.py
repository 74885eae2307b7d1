"""Pins for the oracle's CFL step (orc_cfl_dt) and the last-step clip.

The step sizes are checked against hand-computed values on states chosen so
that every sound speed is a small exact number (gamma = 1.4, rho = 1.4 p
gives c = 1; rho = 0.35 p gives c = 2):

- 1D Euler: dt = CFL h / max_i(|u_i| + c_i) (Sec. 4.3 runs at a CFL number;
  the speed is the largest characteristic speed |u| + c of Sec. 4).
- 2D Euler: dt = CFL / max_i((|u_i| + c_i)/dx + (|v_i| + c_i)/dy), one
  maximum of the per-cell sum.  The cells are chosen so that the plausible
  other forms give other numbers: the sum of the two directional maxima
  (7/CFL here instead of 5), CFL min(dx, dy) / max(|u| + c, |v| + c), and
  the larger of the two one-dimensional steps.
- Advection dt = CFL h / |a|; Burgers dt = CFL h / max|u| (f'(u) = u, Sec. 4.2).
- The march to t_final clips its last step so that it lands on t_final.
"""
import numpy as np
import pytest

import oracle

GAMMA = 1.4


def euler2d_cells(prims):
    """Conserved [4, 1, n] from (rho, u, v, p) per cell."""
    U = np.zeros((4, 1, len(prims)))
    for i, (r, u, v, p) in enumerate(prims):
        U[:, 0, i] = [r, r * u, r * v, p / (GAMMA - 1) + 0.5 * r * (u * u + v * v)]
    return U


def euler1d_cells(prims):
    U = np.zeros((3, len(prims)))
    for i, (r, u, p) in enumerate(prims):
        U[:, i] = [r, r * u, p / (GAMMA - 1) + 0.5 * r * u * u]
    return U


@pytest.mark.parametrize("cfl", [0.5, 0.3])
def test_cfl_dt_euler1d_hand_values(cfl):
    # c = 1 in both cells: |u| + c = 4 and 3
    U = euler1d_cells([(1.4, -3.0, 1.0), (1.4, 2.0, 1.0), (1.4, 0.5, 1.0)])
    h = 0.125
    P = oracle.Problem(oracle.EQ_EULER1D, 5, 3, dx=h, bc=oracle.BC_TRANSMISSIVE)
    assert P.cfl_dt(U, cfl) == pytest.approx(cfl * h / 4.0, rel=1e-14)
    # a faster sound speed (c = 2 at u = 2.5) decides it
    U2 = euler1d_cells([(1.4, -3.0, 1.0), (0.35, 2.5, 1.0)])
    P2 = oracle.Problem(oracle.EQ_EULER1D, 5, 2, dx=h, bc=oracle.BC_TRANSMISSIVE)
    assert P2.cfl_dt(U2, cfl) == pytest.approx(cfl * h / 4.5, rel=1e-14)


def test_cfl_dt_euler2d_is_max_of_sums():
    # cell A: |u|+c = 3, |v|+c = 1; cell B: |u|+c = 1, |v|+c = 4 (c = 1 in both)
    U = euler2d_cells([(1.4, 2.0, 0.0, 1.0), (1.4, 0.0, -3.0, 1.0)])
    for dx, dy, want in [(1.0, 1.0, 5.0),          # max(3+1, 1+4)
                         (0.5, 0.25, 18.0),        # max(6+4, 2+16)
                         (0.25, 1.0, 13.0)]:       # max(12+1, 4+4)
        P = oracle.Problem(oracle.EQ_EULER2D, 5, 2, 1, dx=dx, dy=dy, bc=oracle.BC_TRANSMISSIVE)
        dt = P.cfl_dt(U, 0.5)
        assert dt == pytest.approx(0.5 / want, rel=1e-14), (dx, dy, dt)
        # the plausible misreadings give other steps on these cells
        sum_of_maxes = 0.5 / (max(3 / dx, 1 / dx) + max(1 / dy, 4 / dy))
        min_h = 0.5 * min(dx, dy) / 4.0
        one_d = min(0.5 * dx / 3.0, 0.5 * dy / 4.0)
        for wrong in (sum_of_maxes, min_h, one_d):
            assert abs(dt - wrong) > 1e-3 * dt


def test_cfl_dt_euler2d_sound_speed_counts_in_both_directions():
    # c = 2 (rho = 0.35, p = 1) at rest: (0+2)/dx + (0+2)/dy
    U = euler2d_cells([(0.35, 0.0, 0.0, 1.0), (1.4, 0.5, 0.5, 1.0)])
    P = oracle.Problem(oracle.EQ_EULER2D, 5, 2, 1, dx=0.5, dy=0.25, bc=oracle.BC_TRANSMISSIVE)
    assert P.cfl_dt(U, 0.4) == pytest.approx(0.4 / (4.0 + 8.0), rel=1e-14)


def test_cfl_dt_scalar_equations():
    h = 0.01
    P = oracle.Problem(oracle.EQ_ADVECTION, 5, 8, dx=h, bc=oracle.BC_PERIODIC, a=-2.0)
    assert P.cfl_dt(np.zeros(8), 0.5) == 0.5 * h / 2.0
    u = np.array([0.5, -3.0, 2.0, 1.0, 0.0, 0.25, -1.0, 2.5])
    B = oracle.Problem(oracle.EQ_BURGERS, 5, 8, dx=h, bc=oracle.BC_PERIODIC)
    assert B.cfl_dt(u, 0.5) == 0.5 * h / 3.0


def test_cfl_dt_rejects_non_physical_states():
    U = euler2d_cells([(1.4, 0.0, 0.0, 1.0), (1.4, 0.0, 0.0, 1.0)])
    U[3, 0, 1] = 0.0  # p < 0
    P = oracle.Problem(oracle.EQ_EULER2D, 5, 2, 1, dx=1.0, dy=1.0, bc=oracle.BC_TRANSMISSIVE)
    with pytest.raises(oracle.OracleError):
        P.cfl_dt(U, 0.5)


def test_march_clips_the_last_step_to_t_final():
    """run_ssprk3 takes CFL steps and shortens the last one to land on
    t_final: with dt = CFL h / |a| and t_final = 2.5 dt the march is
    step(dt), step(dt), step(dt / 2), bit for bit."""
    N = 32
    h = 2.0 / N
    x = -1.0 + h * np.arange(N)
    u0 = np.sin(np.pi * x) + 0.3 * (np.abs(x) < 0.4)
    P = oracle.Problem(oracle.EQ_ADVECTION, 5, N, dx=h, bc=oracle.BC_PERIODIC, a=1.0)
    dt = P.cfl_dt(u0, 0.5)
    assert dt == 0.5 * h
    U, n = P.run_ssprk3(u0, 2.5 * dt, 0.5)
    assert n == 3
    ref = P.step_ssprk3(P.step_ssprk3(P.step_ssprk3(u0, dt), dt), 2.5 * dt - 2 * dt)
    assert np.array_equal(U, ref)
    # an exact multiple of dt takes no extra step
    _, n2 = P.run_ssprk3(u0, 4 * dt, 0.5)
    assert n2 == 4
