"""Pins for the oracle's single-window ENO-MR reconstruction (Sec. 3.2-3.3).

Brute force: for every candidate the polynomial of Eq. (Polynomial_Construction)
is rebuilt in exact rational arithmetic, its indicator taken from the
derivative definition of Eq. (CurrentIS), and the candidates are walked in
printed order with a strict comparison against IS_0 of Eq. (Baseline_IS).
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2311_15504_gb300.workloads import random_window
from test_oracle_tables import exact_weights, golden_candidates

ORDERS = [5, 7, 9, 11, 13, 15, 17]


def brute_force(R, w):
    """Exact selection and value for window w (floats, exactly representable)."""
    g = (R + 1) // 2
    f = [Fraction(float(x)) for x in w]
    v = lambda l: f[l + g - 1]  # noqa: E731
    isl = max(abs(v(0) - v(-1)), abs(v(0) - 2 * v(-1) + v(-2)))
    isr = max(abs(v(0) - v(1)), abs(v(0) - 2 * v(1) + v(2)))
    is0 = min(isl, isr)
    tested = [(m, n) for (m, n) in golden_candidates() if 1 <= m <= g - 1 and 1 <= n <= g - 1]
    for t, (m, n) in enumerate(tested):
        a, b = exact_weights(m, n)
        vals = [v(l) for l in range(-m, n + 1)]
        IS = abs(sum(bb * x for bb, x in zip(b, vals)))
        if IS < is0:
            return t, sum(aa * x for aa, x in zip(a, vals)), is0, IS
    T = len(tested)
    da, db = v(1) - v(0), v(0) - v(-1)
    if da * db > 0:
        if abs(da) <= abs(db):
            return T, v(0) + da / 2, is0, None
        return T + 1, v(0) + db / 2, is0, None
    return T + 2, v(0), is0, None


@pytest.mark.parametrize("R", ORDERS)
def test_brute_force_integer_and_step_windows(R):
    """Integer data: every indicator is an exact integer in FP64, so the
    oracle's selection must equal the exact one bit for bit (ties included)."""
    rng = np.random.Generator(np.random.PCG64(100 + R))
    g = (R + 1) // 2
    ties = 0
    for k in range(300):
        w = random_window(rng, 2 * g - 1, "int" if k % 3 else "step")
        if k % 3 == 0:
            w = np.round(w)  # integer-valued step
        t, val, is0, IS = brute_force(R, w)
        got, sel = oracle.mr(R, w)
        assert sel == t, (w, sel, t)
        assert got == pytest.approx(float(val), abs=1e-13 * (1 + np.abs(w).max()))
        # count exact ties IS == IS_0 that the strict rule skipped
        tested = [(m, n) for (m, n) in golden_candidates()
                  if 1 <= m <= g - 1 and 1 <= n <= g - 1]
        for (m, n) in tested[:min(t, len(tested))]:
            _, b = exact_weights(m, n)
            vals = [Fraction(float(w[l + g - 1])) for l in range(-m, n + 1)]
            if abs(sum(bb * x for bb, x in zip(b, vals))) == is0:
                ties += 1
    if R <= 9:
        assert ties > 0  # the strict comparison was exercised


@pytest.mark.parametrize("R", ORDERS)
def test_brute_force_float_windows(R):
    rng = np.random.Generator(np.random.PCG64(200 + R))
    g = (R + 1) // 2
    for _ in range(200):
        w = random_window(rng, 2 * g - 1, "float") * rng.choice([1e-3, 1.0, 1e3])
        t, val, is0, IS = brute_force(R, w)
        got, sel = oracle.mr(R, w)
        if sel != t:
            # only a near-tie in FP64 may flip the outcome
            ois0, mag0, ois, mag = oracle.mr_indicators(R, w)
            k = min(sel, t)
            assert abs(ois[k] - ois0) <= 1e-12 * max(mag[k], mag0)
            continue
        assert got == pytest.approx(float(val), rel=1e-13, abs=1e-13 * np.abs(w).max())


@pytest.mark.parametrize("R", [5, 7, 9, 11])
def test_exhaustive_binary_windows(R):
    g = (R + 1) // 2
    for bits in itertools.product([0.0, 1.0], repeat=2 * g - 1):
        w = np.array(bits)
        t, val, _, _ = brute_force(R, w)
        got, sel = oracle.mr(R, w)
        assert sel == t, (bits, sel, t)
        assert got == pytest.approx(float(val), rel=4e-16 * (2 * g), abs=1e-15)


@pytest.mark.parametrize("R", ORDERS)
def test_flat_side_forces_minmod(R):
    """IS_0 = 0 (flat on one side): no strict inequality can hold."""
    g = (R + 1) // 2
    T = oracle.num_tested(R)
    rng = np.random.Generator(np.random.PCG64(300 + R))
    for _ in range(20):
        w = rng.standard_normal(2 * g - 1)
        w[g - 1:g + 2] = w[g - 1]  # v(0) = v(1) = v(2)
        val, sel = oracle.mr(R, w)
        assert sel >= T
        # minmod(a, b) with a = 0 gives S(0,0) -> f_j
        assert sel == T + 2 and val == w[g - 1]
    # constant window -> exactly the constant
    assert oracle.mr(R, np.full(2 * g - 1, 3.25)) == (3.25, T + 2)


@pytest.mark.parametrize("R", ORDERS)
def test_scale_invariance(R):
    """Sec. 3.3: IS(lam f) = |lam| IS(f), so the selection does not change;
    with lam a power of two the value scales bit for bit."""
    g = (R + 1) // 2
    rng = np.random.Generator(np.random.PCG64(400 + R))
    for _ in range(100):
        w = rng.standard_normal(2 * g - 1)
        val, sel = oracle.mr(R, w)
        for lam in (2.0 ** 20, 2.0 ** -30, -4.0):
            v2, s2 = oracle.mr(R, lam * w)
            assert s2 == sel and v2 == lam * val
        ois0, mag0, ois, mag = oracle.mr_indicators(R, w)
        near = np.any(np.abs(ois - ois0) <= 1e-9 * np.maximum(mag, mag0))
        if not near:
            for lam in (1e6, -3.7e-4):
                v2, s2 = oracle.mr(R, lam * w)
                assert s2 == sel
                assert v2 == pytest.approx(lam * val, rel=1e-12, abs=1e-12 * abs(lam))


@pytest.mark.parametrize("R", ORDERS)
def test_polynomial_reproduction(R):
    """Cell averages of a polynomial of degree <= R-2 reconstruct
    H(x_{j+1/2}) exactly up to rounding through the top stencil."""
    g = (R + 1) // 2
    rng = np.random.Generator(np.random.PCG64(500 + R))
    for _ in range(20):
        deg = int(rng.integers(0, R - 1))
        c = rng.standard_normal(deg + 1)

        def avg(s):  # exact cell average over [s-1/2, s+1/2] in xi units
            return sum(Fraction(float(cd)) * ((Fraction(2 * s + 1, 2) ** (d + 1)
                       - Fraction(2 * s - 1, 2) ** (d + 1)) / (d + 1)) for d, cd in enumerate(c))

        w = np.array([float(avg(s)) for s in range(-(g - 1), g)])
        exact = float(sum(Fraction(float(cd)) * Fraction(1, 2) ** d for d, cd in enumerate(c)))
        val, sel = oracle.mr(R, w)
        if deg >= 1:
            assert sel == 0
        a_top = oracle.candidate(R, 0)[2]
        mag = float(np.abs(a_top * w).sum())  # rounding scale of the sum
        assert abs(val - exact) <= 8 * R * 2.0 ** -52 * mag


@pytest.mark.parametrize("R", ORDERS)
def test_eno_property_single_jump(R):
    """Sec. 3.3: with one jump |df| >> the smooth variation, no selected
    stencil contains both cells next to the jump."""
    g = (R + 1) // 2
    T = oracle.num_tested(R)
    rng = np.random.Generator(np.random.PCG64(600 + R))
    for _ in range(200):
        p = int(rng.integers(-(g - 2), g))          # jump between cells p-1 and p
        eps = 1e-4
        l = np.arange(-(g - 1), g)
        w = eps * (0.3 * l + 0.1 * l * l) + rng.choice([-1, 1]) * (l >= p)
        _, sel = oracle.mr(R, w)
        if sel < T:
            m, n, _, _ = oracle.candidate(R, sel)
        else:
            m, n = [(0, 1), (1, 0), (0, 0)][sel - T]
        assert not (-m <= p - 1 and p <= n), (p, m, n)
