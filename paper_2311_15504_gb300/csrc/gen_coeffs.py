"""Generate enomr_coeffs.h: per-order candidate tables for the CUDA kernels.

Derivation (independent of any table typed from the paper): with the
primitive V(x) = integral of H, the cell averages f_k fix V at the cell
edges xi = -m-1/2, ..., n+1/2 (cumulative sums).  The reconstruction
P = V' of Eq. (Polynomial_Construction) evaluated at xi = 1/2 is the
derivative of the Lagrange interpolant of V, so

    a_s = sum_{i > s} L_i'(1/2)                      (Eq. ReconstructedFlux)

and the indicator of Eq. (CurrentIS), h^K P^(K) with K = m+n, is the
(K+1)-th divided difference of V times (K+1)!:

    b_s = sum_{i > s} (K+1)! / prod_{k != i} (xi_i - xi_k).

The candidate order is Eq. (Candidates); order R = 2r-1 keeps the entries
with m, n <= r-1 and tests those with m, n >= 1 (Sec. 3.2, Step 3.1).

Run:  python gen_coeffs.py  (writes enomr_coeffs.h next to this file).
"""
from __future__ import annotations

import math
import os
import sys
from fractions import Fraction

# Eq. (Candidates), printed order, as (m, n) for S_{j-m}^{j+n}
EQ_CANDIDATES = [
    (8, 8), (7, 8), (8, 7), (7, 7), (8, 6), (6, 7), (7, 6), (6, 6), (7, 5),
    (5, 6), (6, 5), (5, 5), (6, 4), (4, 5), (5, 4), (4, 4), (5, 3), (3, 4), (4, 3),
    (3, 3), (2, 3), (3, 2), (2, 2), (1, 2), (2, 1), (1, 1), (0, 1), (1, 0), (0, 0),
]
ORDERS = [5, 7, 9, 11, 13, 15, 17]


def weights(m: int, n: int):
    K = m + n
    xi = [Fraction(-2 * m - 1, 2) + i for i in range(K + 2)]
    half = Fraction(1, 2)
    # Lagrange derivative weights at xi = 1/2
    dL = []
    for i in range(K + 2):
        den = Fraction(1)
        for k in range(K + 2):
            if k != i:
                den *= xi[i] - xi[k]
        s = Fraction(0)
        for j in range(K + 2):
            if j == i:
                continue
            prod = Fraction(1)
            for k in range(K + 2):
                if k != i and k != j:
                    prod *= half - xi[k]
            s += prod
        dL.append(s / den)
    dd = []
    for i in range(K + 2):
        den = Fraction(1)
        for k in range(K + 2):
            if k != i:
                den *= xi[i] - xi[k]
        dd.append(Fraction(math.factorial(K + 1)) / den)
    a = [sum(dL[i] for i in range(s + 1, K + 2)) for s in range(K + 1)]
    b = [sum(dd[i] for i in range(s + 1, K + 2)) for s in range(K + 1)]
    return a, b


def tested(R: int):
    g = (R + 1) // 2
    return [(m, n) for (m, n) in EQ_CANDIDATES if 1 <= m <= g - 1 and 1 <= n <= g - 1]


def hexlit(x: Fraction) -> str:
    v = float(x)
    if v == 0.0:
        return "0.0"
    return repr(v) if v.is_integer() else v.hex()


def generate() -> str:
    out = []
    out.append("// Generated by gen_coeffs.py -- do not edit by hand.")
    out.append("// ENO-MR candidate tables (arXiv 2311.15504, Eq. Candidates, Tables 1-4),")
    out.append("// derived in exact rational arithmetic and rounded once to double.")
    out.append("#pragma once")
    out.append("")
    out.append("namespace enomr {")
    out.append("")
    out.append("template <int R> struct Tab;           // T = number of tested candidates")
    out.append("template <int R, int t> struct Cand;   // m, n of the t-th tested candidate")
    out.append("")
    for R in ORDERS:
        g = (R + 1) // 2
        W = 2 * g - 1
        lst = tested(R)
        T = len(lst)
        out.append(f"// ---- order {R}: g = {g}, window {W}, {T} tested candidates")
        out.append(f"template <> struct Tab<{R}> {{ static constexpr int T = {T}; }};")
        bs, as_ = [], []
        for t, (m, n) in enumerate(lst):
            out.append(f"template <> struct Cand<{R}, {t}> {{ static constexpr int m = {m}, n = {n}; }};")
            a, b = weights(m, n)
            rowb = [Fraction(0)] * W
            rowa = [Fraction(0)] * W
            for s in range(m + n + 1):
                l = s - m
                rowb[l + g - 1] = b[s]
                rowa[l + g - 1] = a[s]
            bs.append(rowb)
            as_.append(rowa)
        out.append(f"// b_l (rows t, columns l = -(g-1)..g-1; zero outside the stencil)")
        out.append(f"static __constant__ double kB{R}[{T * W}] = {{")
        for row in bs:
            out.append("    " + ", ".join(hexlit(x) for x in row) + ",")
        out.append("};")
        out.append(f"// a_l (same layout)")
        out.append(f"static __constant__ double kA{R}[{T * W}] = {{")
        for row in as_:
            out.append("    " + ", ".join(hexlit(x) for x in row) + ",")
        out.append("};")
        out.append("")
    out.append("template <int R> struct Coef;")
    for R in ORDERS:
        out.append(f"template <> struct Coef<{R}> {{")
        out.append(f"    __device__ static __forceinline__ double b(int i) {{ return kB{R}[i]; }}")
        out.append(f"    __device__ static __forceinline__ double a(int i) {{ return kA{R}[i]; }}")
        out.append(f"    __device__ static __forceinline__ const double *a_table() {{ return kA{R}; }}")
        out.append("};")
    out.append("")
    out.append("}  // namespace enomr")
    out.append("")
    return "\n".join(out)


def main(argv):
    here = os.path.dirname(os.path.abspath(__file__))
    path = os.path.join(here, "enomr_coeffs.h")
    text = generate()
    if len(argv) > 1 and argv[1] == "--check":
        with open(path) as f:
            if f.read() != text:
                print("enomr_coeffs.h is stale", file=sys.stderr)
                return 1
        return 0
    with open(path, "w") as f:
        f.write(text)
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
