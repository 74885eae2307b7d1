"""Pins for the oracle's coefficient tables (Sec. 3.1-3.2, Tables 1-4).

The a_l and b_l used by the oracle are checked against an exact-rational
derivation written here from the definitions -- Eq. (Polynomial_Construction)
(cell averages of P on S_{j-m}^{j+n} equal f_k), Eq. (ReconstructedFlux)
(a_l are the weights of P(x_{j+1/2})) and Eq. (CurrentIS) (b_l are the
weights of h^{m+n} d^{m+n}P/dx^{m+n}) -- and against the paper's printed
Tables 3-4 and the printed order of Eq. (Candidates).
"""
import math
from fractions import Fraction

import pytest

import oracle
from conftest import read_golden

ORDERS = [5, 7, 9, 11, 13, 15, 17]


def _cell_average_matrix(m, n):
    """M[s][d] = (1/h) * integral over cell j+s of xi^d, xi = (x - x_j)/h."""
    K = m + n
    return [[(Fraction(2 * s + 1, 2) ** (d + 1) - Fraction(2 * s - 1, 2) ** (d + 1)) / (d + 1)
             for d in range(K + 1)] for s in range(-m, n + 1)]


def _inverse(A):
    n = len(A)
    M = [row[:] + [Fraction(int(i == j)) for j in range(n)] for i, row in enumerate(A)]
    for k in range(n):
        piv = next(i for i in range(k, n) if M[i][k] != 0)
        M[k], M[piv] = M[piv], M[k]
        f = M[k][k]
        M[k] = [x / f for x in M[k]]
        for i in range(n):
            if i != k and M[i][k] != 0:
                f = M[i][k]
                M[i] = [x - f * y for x, y in zip(M[i], M[k])]
    return [row[n:] for row in M]


_cache = {}


def exact_weights(m, n):
    """(a_l, b_l) for l = -m..n as Fractions, from the definitions."""
    if (m, n) not in _cache:
        K = m + n
        Minv = _inverse(_cell_average_matrix(m, n))  # coefficients c = Minv f
        a = [sum(Fraction(1, 2) ** d * Minv[d][l] for d in range(K + 1)) for l in range(K + 1)]
        b = [math.factorial(K) * Minv[K][l] for l in range(K + 1)]
        _cache[(m, n)] = (a, b)
    return _cache[(m, n)]


def golden_candidates():
    return [tuple(int(x) for x in r.split()) for r in read_golden("eq_candidates_order.txt")]


def test_printed_candidate_order_matches_oracle():
    gold = golden_candidates()
    assert len(gold) == 29
    for s, (m, n) in enumerate(gold):
        om, on, _, _ = oracle.paper_stencil(s)
        assert (om, on) == (m, n)


def test_printed_a_tables_equal_exact_derivation():
    """Tables 1-2 as typed in the oracle equal the exact weights."""
    for s in range(29):
        m, n, den, num = oracle.paper_stencil(s)
        a, _ = exact_weights(m, n)
        assert [Fraction(x, den) for x in num] == a, (m, n)
        assert sum(a) == 1


def test_oracle_weights_are_correctly_rounded_exact_values():
    for R in ORDERS:
        for t in range(oracle.num_tested(R)):
            m, n, a, b = oracle.candidate(R, t)
            ea, eb = exact_weights(m, n)
            assert list(a) == [float(x) for x in ea], (R, m, n)
            assert list(b) == [float(x) for x in eb], (R, m, n)
            # b_l are the (m+n)-th undivided-difference weights: integers
            assert all(x.denominator == 1 for x in eb)
            assert sum(eb) == 0


def test_b_matches_printed_tables_except_two_typos():
    """Tables 3-4 agree with the derivation everywhere except the entry
    printed -3423 in columns S_{j-8}^{j+6} (l=-1) and S_{j-7}^{j+7} (l=0),
    where the derivation gives -3432 = -C(14,7)."""
    mismatches = []
    for row in read_golden("bl_tables_3_4.txt"):
        head, vals = row.split(":")
        m, n = (int(x) for x in head.split())
        printed = [int(x) for x in vals.split()]
        _, b = exact_weights(m, n)
        assert len(printed) == m + n + 1
        for idx, (p, e) in enumerate(zip(printed, b)):
            if p != e:
                mismatches.append((m, n, idx - m, p, int(e)))
    assert sorted(mismatches) == [(7, 7, 0, -3423, -3432), (8, 6, -1, -3423, -3432)]


@pytest.mark.parametrize("R", ORDERS)
def test_candidate_list_reading(R):
    """Tested list for order R: Eq. (Candidates) entries with 1 <= m,n <= g-1,
    in printed order (the reading for orders the paper does not list)."""
    g = (R + 1) // 2
    want = [(m, n) for (m, n) in golden_candidates() if 1 <= m <= g - 1 and 1 <= n <= g - 1]
    got = [oracle.candidate(R, t)[:2] for t in range(oracle.num_tested(R))]
    assert got == want
    assert got[0] == (g - 1, g - 1)
    assert got[-1] == (1, 1)
    assert len(got) == {5: 4, 7: 7, 9: 10, 11: 14, 13: 18, 15: 22, 17: 26}[R]


def test_printed_pool_sizes():
    """Sec. 3.1: one candidate of 1, 3, 5, 7 and 17 points, two of every
    other size."""
    sizes = [m + n + 1 for m, n in golden_candidates()]
    for k in range(1, 18):
        assert sizes.count(k) == (1 if k in (1, 3, 5, 7, 17) else 2), k
