"""Pins for the oracle's Burgers right-hand side (Sec. 4.2).

- Values printed in Table 8 (accuracy test, t = 0.1/lam).
- Scale invariance: the lam = 1e3 errors are the lam = 1 errors times 1e3
  (Table 8 prints exactly that; the selection is invariant under u -> a u).
- Where u > 0 on the whole line the flux needs no splitting, so the scheme
  is the ENO-MR reconstruction of the values f = u^2/2 -- the advection
  scheme (a = 1) applied to those values, pinned by Tables 5-7.
- Mixed signs: the global Lax-Friedrichs split; the scheme commutes with
  the reflection u(x) -> -u(-x) that maps solutions to solutions.
- Discrete conservation on a periodic line.
"""
import numpy as np
import pytest

import oracle
from burgers_exact import dt_schedule, errors, exact, exact_entropy
from conftest import read_golden
from paper_2311_15504_gb300 import workloads as wl


def run(R, hinv, lam=1.0):
    n = 2 * hinv
    u, h = wl.burgers_sine3(n, lam)
    P = oracle.Problem(oracle.EQ_BURGERS, R, n, dx=h, bc=oracle.BC_PERIODIC)
    t = 0.1 / lam
    for dt in dt_schedule(R, h, t, lam):
        u = P.step_ssprk3(u, dt)
    return u, h, t


ROWS = read_golden("burgers_errors_table_8.txt")


@pytest.mark.parametrize("row", ROWS)
def test_paper_burgers_errors(row):
    """Table 8 in FP64.  The paper does not state how its last step lands
    on t or how the exact solution was evaluated; the printed values are
    matched to 15 % on the coarsest grid (h = 1/32, where those details
    matter most) and to 2 % on the finer ones."""
    p = row.split()
    R, hinv, l1p, lip = int(p[0]), int(p[1]), float(p[2]), float(p[3])
    u, h, t = run(R, hinv)
    l1, li = errors(u, h, t)
    tol = 0.15 if hinv <= 32 else 0.02
    print(f"R={R} h=1/{hinv}: L1 {l1:.3e} (paper {l1p:.2e}), Linf {li:.3e} (paper {lip:.2e})")
    assert abs(l1 / l1p - 1.0) <= tol
    assert abs(li / lip - 1.0) <= tol


def test_burgers_orders_follow_table_8():
    """Observed orders between consecutive printed grids (h <= 1/64)."""
    by_r = {}
    for row in ROWS:
        p = row.split()
        by_r.setdefault(int(p[0]), []).append((int(p[1]), float(p[2])))
    for R, rows in by_r.items():
        rows = [r for r in rows if r[0] >= 64]
        for (h0, e0), (h1, e1) in zip(rows, rows[1:]):
            printed = np.log(e0 / e1) / np.log(h1 / h0)
            l0 = errors(*run(R, h0))[0]
            l1 = errors(*run(R, h1))[0]
            got = np.log(l0 / l1) / np.log(h1 / h0)
            assert abs(got - printed) <= 0.1, (R, h0, h1, got, printed)


@pytest.mark.parametrize("R", [5, 9])
def test_burgers_scale_invariance(R):
    u1, h, t1 = run(R, 64, 1.0)
    u3, _, t3 = run(R, 64, 1e3)
    e1 = errors(u1, h, t1, 1.0)
    e3 = errors(u3, h, t3, 1e3)
    assert e3[0] / e1[0] == pytest.approx(1e3, rel=1e-6)
    assert e3[1] / e1[1] == pytest.approx(1e3, rel=1e-6)


@pytest.mark.parametrize("R", [5, 9, 13, 17])
def test_positive_burgers_is_advection_of_flux_values(R):
    rng = np.random.Generator(np.random.PCG64(R))
    n = 96
    u = 1.0 + 0.5 * np.sin(2 * np.pi * np.arange(n) / n) + 0.2 * rng.random(n)
    u[40:52] += 1.0  # a jump
    h = 0.01
    b = oracle.rhs_burgers(u, h, R, want_sel=True)
    f = 0.5 * (u * u)
    a = oracle.rhs_advection(f, h, R, a=1.0, want_sel=True)
    assert np.array_equal(b["sel"], a["sel"])
    assert np.array_equal(b["rhs"], a["rhs"])
    # all negative: the mirror image, f^+ = 0
    bn = oracle.rhs_burgers(-u, h, R, want_sel=True)
    an = oracle.rhs_advection(f, h, R, a=-1.0, want_sel=True)
    assert np.array_equal(bn["rhs"], -an["rhs"])


@pytest.mark.parametrize("R", [5, 9, 17])
def test_mixed_sign_reflection_and_conservation(R):
    rng = np.random.Generator(np.random.PCG64(100 + R))
    n = 128
    x = np.arange(n) / n
    u = np.sin(2 * np.pi * x) + 0.3 * np.sin(6 * np.pi * x + 1.0) + 0.05 * rng.standard_normal(n)
    h = 1.0 / n
    r = oracle.rhs_burgers(u, h, R)["rhs"]
    # conservation: sum_i L_i = 0 up to rounding
    assert abs(r.sum()) <= 1e-12 * n * np.abs(r).max()
    # reflection x -> -x (cell j -> -j mod n on the periodic grid), u -> -u
    ref = np.roll(u[::-1], 1)
    rr = oracle.rhs_burgers(-ref, h, R)["rhs"]
    assert np.allclose(-np.roll(rr[::-1], 1), r, rtol=0, atol=1e-11 * np.abs(r).max())


def test_entropy_solution_reference():
    """The Hopf-Lax reference: equal to the characteristic solution before
    the shock forms, mass-conserving after, and its shock moves at the
    Rankine-Hugoniot speed (u_L + u_R) / 2, which is 1 for this data (the
    data are odd about u = 1 around the shock)."""
    x = np.linspace(0.0, 2.0, 64, endpoint=False)
    assert np.abs(exact_entropy(x, 0.3) - exact(x, 0.3)).max() < 1e-13
    n = 4000
    xx = (np.arange(n) + 0.5) * 2.0 / n
    pos = []
    for t in (1.5, 2.0):
        u = exact_entropy(xx, t)
        assert abs(u.mean() * 2.0 - 2.0) < 1e-3  # midpoint rule across one jump
        j = np.argmax(np.abs(np.diff(u)))
        pos.append(0.5 * (xx[j] + xx[j + 1]))
        uL, uR = u[j], u[j + 1]
        assert abs(0.5 * (uL + uR) - 1.0) < 5e-3
    assert abs((pos[1] - pos[0]) % 2.0 - 0.5) <= 2.0 * 2.0 / n


def _shock_run(N, R, cfl=0.3, T=2.0):
    u, h = wl.burgers_sine3(N)
    P = oracle.Problem(oracle.EQ_BURGERS, R, N, dx=h, bc=oracle.BC_PERIODIC)
    u0, t, n = u.copy(), 0.0, 0
    while t < T and n < 100000:
        dt = min(P.cfl_dt(u, cfl), T - t)
        assert dt > 0.0
        u = P.step_ssprk3(u, dt)
        t += dt
        n += 1
    return u0, u, h


@pytest.mark.parametrize("R", [5, 9, 13, 17])
def test_shock_run_against_entropy_solution(R):
    """Sec. 4.2's second run (h = 1/64, CFL 0.3, t = 2, a shock at x = 1)
    against the exact entropy solution: L1 error, no new extrema, the shock
    within two cells, the smooth part within 1e-3, mass conserved."""
    N = 128
    u0, u, h = _shock_run(N, R)
    x = h * np.arange(N)
    ex = exact_entropy(x, 2.0)
    assert np.abs(u - ex).mean() < 5e-3
    assert u.max() <= ex.max() + 1e-3 and u.min() >= ex.min() - 1e-3
    j = np.argmax(np.abs(np.diff(u)))
    assert abs(0.5 * (x[j] + x[j + 1]) - 1.0) <= 2 * h
    far = np.abs(x - 1.0) > 6 * h
    assert np.abs(u - ex)[far].max() < 1e-3
    assert abs(u.sum() - u0.sum()) * h < 1e-11


def test_shock_run_converges_at_first_order():
    errs = []
    for N in (128, 256, 512):
        _, u, h = _shock_run(N, 9)
        errs.append(np.abs(u - exact_entropy(h * np.arange(N), 2.0)).mean())
    assert errs[1] < 0.6 * errs[0] and errs[2] < 0.6 * errs[1]
