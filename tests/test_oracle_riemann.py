"""The oracle's 1D Euler scheme on the paper's Lax shock tube (Sec. 4.3:
[0, 2], (0.445, 0.698, 3.528) | (0.5, 0, 0.571), non-reflecting ends,
t = 0.26, h = 1/100), pinned to the exact Riemann solution:
- the exact solution itself is checked against the jump conditions across
  its shock and the isentropic relations across its rarefaction;
- density errors at the grid points: first-order convergence under
  refinement (the solution has a shock and a contact), a bound at the
  paper's h, and no new extrema beyond 1 % of the density range (the ENO
  property the paper states for every order);
- the shock where the exact solution puts it, to two cells;
- conservation: with the waves inside the domain, the totals change by
  exactly t (F(U_L) - F(U_R)), the boundary fluxes.
Planted in the oracle, a dropped pressure term of the energy flux fails five
of these tests and halving the split's dissipation fails the no-new-extrema
bound.  A wrong eigenvector or Roe average still gives a consistent,
conservative scheme and passes here; the eigensystem pins of
test_oracle_rhs.py catch those."""
import math

import numpy as np
import pytest

import oracle
from riemann_exact import sample, star_state
from paper_2311_15504_gb300 import workloads as wl

LEFT, RIGHT = (0.445, 0.698, 3.528), (0.5, 0.0, 0.571)
T_END, X0, G = 0.26, 1.0, 1.4


def _flux(rho, u, p):
    E = p / (G - 1.0) + 0.5 * rho * u * u
    return np.array([rho * u, rho * u * u + p, (E + p) * u]), np.array([rho, rho * u, E])


def _run(N, R, cfl=0.5):
    U, h = wl.lax_tube(N)
    P = oracle.Problem(oracle.EQ_EULER1D, R, N, dx=h, bc=oracle.BC_TRANSMISSIVE)
    U0, t, n = U.copy(), 0.0, 0
    while t < T_END and n < 10000:
        dt = min(P.cfl_dt(U, cfl), T_END - t)
        assert dt > 0.0
        U = P.step_ssprk3(U, dt)
        t += dt
        n += 1
    assert t == T_END
    return U0, U, h


def _exact_rho(N, h):
    x = h * (np.arange(N) + 0.5)
    return sample(LEFT, RIGHT, (x - X0) / T_END)[0], x


def test_exact_solution_satisfies_jump_and_isentropic_relations():
    ps, us = star_state(LEFT, RIGHT)
    rl, ul, pl = LEFT
    rr, ur, pr = RIGHT
    # right-moving shock into the right state: mass, momentum, energy fluxes
    # relative to the shock are continuous
    S = ur + math.sqrt(G * pr / rr) * math.sqrt((G + 1) / (2 * G) * ps / pr + (G - 1) / (2 * G))
    rs = sample(LEFT, RIGHT, [0.5 * (us + S)])[0, 0]
    Fa, Ua = _flux(rr, ur, pr)
    Fb, Ub = _flux(rs, us, ps)
    assert np.allclose(Fa - S * Ua, Fb - S * Ub, rtol=1e-12, atol=1e-12)
    # left rarefaction: p / rho^gamma and u + 2c/(gamma-1) as on the left
    cl = math.sqrt(G * pl / rl)
    xi = np.linspace(ul - cl, us - 1e-9, 7)
    r, u, p = sample(LEFT, RIGHT, xi)
    assert np.allclose(p / r ** G, pl / rl ** G, rtol=1e-12)
    assert np.allclose(u + 2 * np.sqrt(G * p / r) / (G - 1), ul + 2 * cl / (G - 1), rtol=1e-12)
    # the contact: pressure and velocity continuous across it
    a, b = sample(LEFT, RIGHT, [us - 1e-9, us + 1e-9])[:, :].T
    assert abs(a[1] - b[1]) < 1e-12 and abs(a[2] - b[2]) < 1e-12 and a[0] != b[0]


@pytest.mark.parametrize("R", [5, 9, 13, 17])
def test_lax_tube_against_exact_solution(R):
    N = 200  # h = 1/100, the paper's grid
    U0, U, h = _run(N, R)
    ex, x = _exact_rho(N, h)
    rho = U[0]
    assert np.abs(rho - ex).mean() < 1.2e-2
    span = ex.max() - ex.min()
    assert rho.max() <= ex.max() + 0.01 * span and rho.min() >= ex.min() - 0.01 * span
    # the shock: the steepest density drop right of the contact
    ps, us = star_state(LEFT, RIGHT)
    cr = math.sqrt(G * RIGHT[2] / RIGHT[0])
    S = cr * math.sqrt((G + 1) / (2 * G) * ps / RIGHT[2] + (G - 1) / (2 * G))
    xs = X0 + S * T_END
    right = x > X0 + us * T_END + 5 * h
    j = np.argmin(np.diff(rho[right]))
    x_num = 0.5 * (x[right][j] + x[right][j + 1])
    assert abs(x_num - xs) <= 2 * h
    # conservation with the boundary fluxes of the undisturbed end states
    FL, _ = _flux(*LEFT)
    FR, _ = _flux(*RIGHT)
    expect = U0.sum(axis=1) * h + T_END * (FL - FR)
    assert np.allclose(U.sum(axis=1) * h, expect, rtol=1e-12, atol=1e-12)


def test_lax_tube_converges_at_first_order():
    errs = []
    for N in (100, 200, 400):
        _, U, h = _run(N, 9)
        ex, _ = _exact_rho(N, h)
        errs.append(np.abs(U[0] - ex).mean())
    assert errs[1] < 0.65 * errs[0] and errs[2] < 0.65 * errs[1]
