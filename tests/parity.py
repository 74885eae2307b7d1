"""Helpers for comparing the CUDA path with the oracle.

Selection: ids must be equal except at near-ties.  Where the two choices
differ, the decision that first diverged is located and checked against
the oracle's own quantities: either an indicator test IS_t < IS_0 that is
within 1e-12 of the scale of the terms forming it (sum_l |b_l| max|v|), or
a minmod decision whose compared slopes are within the same relative
distance.  Values: the oracle is re-run with the CUDA path's selection
forced, so every cell is compared, with the bound
|d| <= 1e-12 * max(||L||_inf, ||F||_inf / h), and |d| <= 1e-12 ||L||_inf
where the flux term is small enough for that bound to be attainable.
"""
from __future__ import annotations

import numpy as np

import oracle

TIE_REL = 1e-12
VAL_REL = 1e-12
# strict 1e-12 ||L||_inf bound where ||F||_inf / h <= STRICT_RATIO ||L||_inf
STRICT_RATIO = 64.0


def _bsum(R):
    return [float(np.abs(oracle.candidate(R, t)[3]).sum()) for t in range(oracle.num_tested(R))]


def classify_mismatches(R, sel_gpu, sel_orc, windows, scale_fn=None):
    """Return (n_mismatch, n_near_tie, worst) for flattened selection arrays
    and the oracle's windows [..., 2g-1] (same leading shape).  scale_fn(i)
    gives the magnitude of the terms that formed window i (default max|v|)."""
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
        if scale_fn is not None:
            vmax = max(vmax, float(scale_fn(int(i))))
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


def assert_selection(R, sel_gpu, sel_orc, windows, what="", scale_fn=None):
    n, ties, worst = classify_mismatches(R, sel_gpu, sel_orc, windows, scale_fn)
    assert n == ties, f"{what}: {n - ties} selection mismatches that are not near-ties (worst {worst:.2e})"
    return n


def assert_values(gpu, ref, flux_scale_over_h, what="", strict=None):
    """Bound |GPU - oracle| elementwise and return err / ||L||_inf.

    The general bound is 1e-12 * max(||L||_inf, ||F||_inf / h): L is a
    difference of two interface fluxes divided by h, so a rounding error of
    a few ulps in F (the two sides' different operation orders) reaches
    ~eps ||F||_inf / h in L however small L is.  On a fine grid of smooth
    data ||F||_inf / h exceeds ||L||_inf by up to the number of cells per
    wavelength, and there no bound in ||L||_inf alone can hold.  Where that
    floor is far below the strict bound (||F||_inf / h <= STRICT_RATIO
    ||L||_inf, the default of strict=None), |GPU - oracle| <= 1e-12
    ||L||_inf is asserted as well.
    """
    gpu = np.asarray(gpu)
    ref = np.asarray(ref)
    lnorm = float(np.abs(ref).max())
    scale = max(lnorm, float(flux_scale_over_h))
    err = float(np.abs(gpu - ref).max())
    rel_l = err / lnorm if lnorm > 0 else (0.0 if err == 0 else np.inf)
    if strict is None:
        strict = float(flux_scale_over_h) <= STRICT_RATIO * lnorm
    print(f"{what}: max|d| = {err:.3e}, /||L|| = {rel_l:.2e}, "
          f"/max(||L||,||F||/h) = {err / scale if scale > 0 else 0.0:.2e}"
          f"{' (strict)' if strict else ''}")
    assert err <= VAL_REL * scale, f"{what}: max|d| = {err:.3e} > {VAL_REL:.0e} * {scale:.3e}"
    if strict:
        assert err <= VAL_REL * lnorm, (
            f"{what}: max|d| = {err:.3e} > {VAL_REL:.0e} * ||L||_inf = {lnorm:.3e}")
    return rel_l


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


def _phys_flux(Uc, gamma):
    c = Uc.shape[0]
    rho, un = Uc[0], Uc[1] / Uc[0]
    ut = Uc[2] / Uc[0] if c == 4 else 0.0
    p = (gamma - 1) * (Uc[-1] - 0.5 * rho * (un * un + ut * ut))
    F = [Uc[1], Uc[1] * un + p] + ([Uc[2] * un] if c == 4 else []) + [(Uc[-1] + p) * un]
    return np.array(F)


def euler_scale_fn(line_state, n_lines, nlen, R, bc, alpha, gamma=1.4):
    """scale_fn for Euler selections laid out [side][field][line][nlen+1]:
    the largest 1/2 (|L_f| |F| + alpha_f |L_f| |U|) over the window cells,
    with L from the oracle's Roe eigen-system.  line_state(line) returns the
    line's cells as [nlen, c] in line components (rho, m_n, [m_t], E);
    alpha(line) the oracle's per-field alpha."""
    g = (R + 1) // 2
    cache = {}

    def cells(line):
        if line not in cache:
            cache[line] = line_state(line)
        return cache[line]

    def gidx(j):
        if bc == 0:
            return j % nlen
        return min(max(j, 0), nlen - 1)

    def fn(i):
        NI = nlen + 1
        k = i % NI
        line = (i // NI) % n_lines
        c = cells(line).shape[1]
        field = (i // (NI * n_lines)) % c
        side = i // (NI * n_lines * c)
        X = cells(line)
        _, Lm, _ = oracle.euler_eigen(X[gidx(k - 1)], X[gidx(k)], gamma)
        a = alpha(line)[field]
        best = 0.0
        for l in range(-(g - 1), g):
            j = k - 1 + l if side == 0 else k - l
            Uc = X[gidx(j)]
            m = 0.5 * (np.abs(Lm[field]) @ np.abs(_phys_flux(Uc, gamma))
                       + a * (np.abs(Lm[field]) @ np.abs(Uc)))
            best = max(best, float(m))
        return best
    return fn


def shock_gate(step_fn, U0, steps, seeds=(1, 2)):
    """Rounding-sensitivity envelope of the oracle itself: the L1 distance
    between its trajectory and the same trajectory with a one-ulp random
    perturbation after the first step (largest over seeds).  The shock-case
    gate is max(1e-6, 4 * envelope)."""
    base = U0.copy()
    for dt in steps:
        base = step_fn(base, dt)
    env = 0.0
    for sd in seeds:
        rng = np.random.Generator(np.random.PCG64(sd))
        b = step_fn(U0.copy(), steps[0])
        b = b + np.spacing(np.abs(b)) * rng.choice([-1, 0, 1], size=b.shape)
        for dt in steps[1:]:
            b = step_fn(b, dt)
        env = max(env, float(np.abs(b - base).mean()))
    return base, max(1e-6, 4.0 * env), env


def forced_replay(stage_gpu, sel_gpu, to_host, rhs_forced, U0_dev, U0, steps, flips_fn=None):
    """Advance the CUDA path and the oracle side by side with the CUDA path's
    per-stage selections forced on the oracle.

    Per SSP-RK3 step of size dt (Eq. TVD3rdRK, in the paper's written form):
    the CUDA path takes its three stages explicitly (stage_gpu(s, Un, Us,
    out, dt)), its selection at every stage state (sel_gpu) is handed to
    the oracle's right-hand side (rhs_forced(V, sel)), and the oracle
    combines its own stages.  With every discrete choice shared, the two
    trajectories differ by rounding propagated through a Lipschitz map, not
    by the selection flips that make free-running shock trajectories
    diverge, so the final states can be compared at a fixed tolerance.

    flips_fn(U_stage_host, sel), if given, counts the stage's flips against
    the oracle's own selection on the CUDA path's stage state and asserts
    that each is a near-tie; its counts are summed.  Returns (final CUDA
    state, final oracle state, total flips, stage evaluations).
    """
    import torch
    Un = U0_dev.clone()
    U1, U2, U3 = torch.empty_like(Un), torch.empty_like(Un), torch.empty_like(Un)
    V = np.array(U0, dtype=np.float64, copy=True)
    flips = 0
    nstage = 0
    for dt in steps:
        sels = []
        for s, (Us, out) in enumerate(((Un, U1), (U1, U2), (U2, U3)), start=1):
            sel = sel_gpu(Us)
            if flips_fn is not None:
                flips += flips_fn(to_host(Us), sel)
            sels.append(sel)
            stage_gpu(s, Un, Us, out, dt)
            nstage += 1
        V1 = V + dt * rhs_forced(V, sels[0])
        V2 = 0.75 * V + 0.25 * (V1 + dt * rhs_forced(V1, sels[1]))
        V = (1.0 / 3.0) * V + (2.0 / 3.0) * (V2 + dt * rhs_forced(V2, sels[2]))
        Un, U3 = U3, Un
    return to_host(Un), V, flips, nstage


def classify_euler2d_flips(U, dx, dy, R, bc, sel, ref_sel, chunk=64, gamma=1.4):
    """Classify every selection flip of a 2D Euler RHS (CUDA selections sel
    against the oracle's ref_sel, both in the [x sweep | y sweep] layout of
    enomr_debug_selection).  A sweep of a line depends on that line only,
    so the oracle's windows are formed on stacks of at most `chunk` flipped
    lines at a time (memory stays bounded on a 4096^2 grid).  Returns
    (flips, near-ties, worst relative distance) summed over both sweeps."""
    U = np.asarray(U)
    _, ny, nx = U.shape
    nsx = 8 * ny * (nx + 1)
    sel = np.asarray(sel).reshape(-1)
    ref_sel = np.asarray(ref_sel).reshape(-1)
    flips = np.nonzero(sel != ref_sel)[0]
    total = ties = 0
    worst = 0.0
    for sweep in ("x", "y"):
        sub = flips[flips < nsx] if sweep == "x" else flips[flips >= nsx] - nsx
        if sub.size == 0:
            continue
        nlen, nlines = (nx, ny) if sweep == "x" else (ny, nx)
        lines = np.unique((sub // (nlen + 1)) % nlines)
        gs = (sel[:nsx] if sweep == "x" else sel[nsx:]).reshape(2, 4, nlines, nlen + 1)
        rs = (ref_sel[:nsx] if sweep == "x" else ref_sel[nsx:]).reshape(2, 4, nlines, nlen + 1)
        for c0 in range(0, lines.size, chunk):
            ln = lines[c0:c0 + chunk]
            Ul = U[:, ln, :] if sweep == "x" else U[:, :, ln]
            o = oracle.rhs_euler2d(np.ascontiguousarray(Ul), dx, dy, R, bc=bc, gamma=gamma,
                                   want_sel=True, want_win=True)
            L = ln.size
            if sweep == "x":
                osel, win = o["sel_x"], o["win_x"]
                X = (lambda Ul_: lambda y: Ul_[:, y, :].T.copy())(Ul)
                fn = euler_scale_fn(X, L, nlen, R, bc, (lambda o_: lambda y: o_["alpha_x"][y])(o),
                                    gamma)
            else:
                osel, win = o["sel_y"], o["win_y"]
                X = (lambda Ul_: lambda x: Ul_[[0, 2, 1, 3], :, x].T.copy())(Ul)
                fn = euler_scale_fn(X, L, nlen, R, bc, (lambda o_: lambda x: o_["alpha_y"][x])(o),
                                    gamma)
            # the stacked lines' sweep equals the full problem's on those lines
            assert np.array_equal(osel, rs[:, :, ln, :])
            n, t, w = classify_mismatches(R, gs[:, :, ln, :], osel, win, fn)
            total += n
            ties += t
            worst = max(worst, w)
    return total, ties, worst
