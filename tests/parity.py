"""Helpers for comparing the CUDA path with the oracle.

Selection: ids must be equal except at near-ties.  Where the two choices
differ, the decision that first diverged is located and checked against
the oracle's own quantities: either an indicator test IS_t < IS_0 that is
within 1e-12 of the scale of the terms forming it (sum_l |b_l| max|v|), or
a minmod decision whose compared slopes are within the same relative
distance.  Values: the oracle is re-run with the CUDA path's selection
forced, so every cell is compared, with the bound
|d| <= 1e-12 * max(||L||_inf, ||F||_inf / h).
"""
from __future__ import annotations

import numpy as np

import oracle

TIE_REL = 1e-12
VAL_REL = 1e-12


def _bsum(R):
    return [float(np.abs(oracle.candidate(R, t)[3]).sum()) for t in range(oracle.num_tested(R))]


def classify_mismatches(R, sel_gpu, sel_orc, windows):
    """Return (n_mismatch, n_near_tie, worst) for flattened selection arrays
    and the oracle's windows [..., 2g-1] (same leading shape)."""
    sel_gpu = np.asarray(sel_gpu).reshape(-1)
    sel_orc = np.asarray(sel_orc).reshape(-1)
    win = np.asarray(windows).reshape(sel_orc.shape[0], -1)
    T = oracle.num_tested(R)
    g = (R + 1) // 2
    bsum = _bsum(R)
    bad = np.nonzero(sel_gpu != sel_orc)[0]
    ties = 0
    worst = 0.0
    for i in bad:
        w = win[i]
        vmax = float(np.abs(w).max())
        is0, _, is_, _ = oracle.mr_indicators(R, w)
        k = int(min(sel_gpu[i], sel_orc[i]))
        if k < T:
            scale = max(bsum[k], 4.0) * vmax
            rel = abs(is_[k] - is0) / scale if scale > 0 else np.inf
        else:
            a = w[g] - w[g - 1]
            b = w[g - 1] - w[g - 2]
            scale = 2.0 * vmax
            rel = min(abs(abs(a) - abs(b)), abs(a), abs(b)) / scale if scale > 0 else np.inf
        worst = max(worst, rel)
        if rel <= TIE_REL:
            ties += 1
    return len(bad), ties, worst


def assert_selection(R, sel_gpu, sel_orc, windows, what=""):
    n, ties, worst = classify_mismatches(R, sel_gpu, sel_orc, windows)
    assert n == ties, f"{what}: {n - ties} selection mismatches that are not near-ties (worst {worst:.2e})"
    return n


def assert_values(gpu, ref, flux_scale_over_h, what=""):
    gpu = np.asarray(gpu)
    ref = np.asarray(ref)
    scale = max(float(np.abs(ref).max()), float(flux_scale_over_h))
    err = float(np.abs(gpu - ref).max())
    assert err <= VAL_REL * scale, f"{what}: max|d| = {err:.3e} > {VAL_REL:.0e} * {scale:.3e}"
    return err / scale if scale > 0 else 0.0


def euler_flux_scale(U, gamma=1.4):
    """max |F(U)| over cells and components (normal fluxes of both axes)."""
    U = np.asarray(U)
    rho = U[0]
    if U.shape[0] == 3:
        u = U[1] / rho
        p = (gamma - 1) * (U[2] - 0.5 * rho * u * u)
        return float(max(np.abs(U[1]).max(), np.abs(U[1] * u + p).max(),
                         np.abs((U[2] + p) * u).max()))
    u, v = U[1] / rho, U[2] / rho
    p = (gamma - 1) * (U[3] - 0.5 * rho * (u * u + v * v))
    return float(max(np.abs(U[1]).max(), np.abs(U[2]).max(), np.abs(U[1] * u + p).max(),
                     np.abs(U[2] * v + p).max(), np.abs((U[3] + p) * u).max(),
                     np.abs((U[3] + p) * v).max()))
