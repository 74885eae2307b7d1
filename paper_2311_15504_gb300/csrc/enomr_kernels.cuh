// enomr_kernels.cuh -- device core of the ENO-MR right-hand side shared by
// every equation: ghost indexing, the ENO-MR selection and reconstruction
// of one window, and the stage epilogue.
//
// arXiv 2311.15504: Sec. 2.1 (Eq. 1DWENOFD), Sec. 3.1 (Eq. Candidates),
// Sec. 3.2 (Steps 1-3), Eq. TVD3rdRK.
//
// Design (GB300): the path is bound by the FP64 pipe, not by HBM, so the
// kernels minimise FP64 instructions:
//  * |x|, max, min and every IS < IS_0 test run on the integer ALU: for
//    non-negative doubles the IEEE bit pattern orders like an int64.
//  * the baseline indicator uses fma(-2, v_{-1}, v_0) + v_{-2}, which rounds
//    exactly like the written (v_0 - 2 v_{-1}) + v_{-2};
//  * the walk over candidates is unrolled at compile time (coefficients are
//    constant-bank operands) and warp-uniform: a lane that found its
//    stencil is predicated off, and the warp leaves the walk as soon as no
//    lane is still searching;
//  * the reconstruction on the chosen stencil is one dot product over the
//    window with a row of a shared-memory coefficient table (constant
//    operands when the whole warp took the top stencil), the minmod
//    fallback is a single fma.
#pragma once

#include <stdint.h>

#include "enomr_coeffs.h"
#include "enomr_common.cuh"
#include "enomr_internal.h"

namespace enomr {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ long long abits(double x)
{
    return __double_as_longlong(x) & 0x7fffffffffffffffLL;
}

__device__ __forceinline__ long long imax64(long long a, long long b) { return a > b ? a : b; }
__device__ __forceinline__ long long imin64(long long a, long long b) { return a < b ? a : b; }

// Cell of (possibly ghost) index i on a line of n cells: periodic wrap
// (bc 0) or clamp (bc 1).  A tile's cells lie within one line length of the
// line in all but the shortest lines, so the wrap is one add or subtract
// there; the 64-bit remainder (a long software sequence) only beyond.
__device__ __forceinline__ long long ghost(long long i, long long n, int bc)
{
    if (bc == 0) {
        if (i >= 0 && i < n) return i;
        if (i < 0 && i >= -n) return i + n;
        if (i >= n && i < 2 * n) return i - n;
        long long r = i % n;
        return r < 0 ? r + n : r;
    }
    return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

// ---------------------------------------------------------------------------
// Sec. 3.2 Steps 2-3.1: walk the tested candidates in printed order; the
// first with IS = |sum b_l v_l| < IS_0 wins.
// ---------------------------------------------------------------------------
template <int R, int t>
__device__ __forceinline__ void walk(const double *v, long long is0, int &sel, bool &active)
{
    if constexpr (t < Tab<R>::T) {
        constexpr int g = (R + 1) / 2, W = 2 * g - 1;
        constexpr int m = Cand<R, t>::m, n = Cand<R, t>::n;
        if (active) {
            double s = Coef<R>::b(t * W + g - 1 - m) * v[g - 1 - m];
#pragma unroll
            for (int l = -m + 1; l <= n; ++l) s = fma(Coef<R>::b(t * W + g - 1 + l), v[g - 1 + l], s);
            if (abits(s) < is0) {
                sel = t;
                active = false;
            }
        }
        if (__any_sync(FULL, active)) walk<R, t + 1>(v, is0, sel, active);
    }
}

// ENO-MR value of one window v[0..W-1] (v[g-1] = f_j).  All 32 lanes must
// call it together; lanes with valid == false take part in the warp votes
// only.  sA: shared copy of the a_l table of order R.
template <int R>
__device__ __forceinline__ double mr_value(const double *v, const double *sA, bool valid, int &sel)
{
    constexpr int g = (R + 1) / 2, W = 2 * g - 1, T = Tab<R>::T, c = g - 1;
    // Step 1, Eq. (Baseline_IS)
    const double d1L = v[c] - v[c - 1];
    const double d2L = fma(-2.0, v[c - 1], v[c]) + v[c - 2];
    const double d1R = v[c] - v[c + 1];
    const double d2R = fma(-2.0, v[c + 1], v[c]) + v[c + 2];
    const long long is0 = imin64(imax64(abits(d1L), abits(d2L)), imax64(abits(d1R), abits(d2R)));
    // IS >= 0 always, so with IS_0 = 0 no candidate can pass: skip the walk
    // (same outcome as testing every candidate).
    bool active = valid && is0 != 0;
    sel = T;
    walk<R, 0>(v, is0, sel, active);
    active = active || (valid && is0 == 0);
    // Step 3.2: minmod(a, b), a = f_{j+1} - f_j = -d1R, b = f_j - f_{j-1} = d1L
    double mm = 0.0;
    if (active || !valid) {
        const long long ba = __double_as_longlong(d1R), bb = __double_as_longlong(d1L);
        const bool nz = abits(d1R) != 0 && abits(d1L) != 0;
        const bool same = nz && ((ba ^ bb) < 0);  // a = -d1R: signs of a, b agree
        if (!same) {
            sel = T + 2;
        } else if (abits(d1R) <= abits(d1L)) {
            sel = T;
            mm = -d1R;
        } else {
            sel = T + 1;
            mm = d1L;
        }
    }
    double val;
    if (__all_sync(FULL, sel == 0)) {
        val = Coef<R>::a(0) * v[0];
#pragma unroll
        for (int l = 1; l < W; ++l) val = fma(Coef<R>::a(l), v[l], val);
    } else if (sel < T) {
        const double *row = sA + sel * W;
        val = 0.0;
#pragma unroll
        for (int l = 0; l < W; ++l) val = fma(row[l], v[l], val);
    } else {
        val = fma(0.5, mm, v[c]);
    }
    return val;
}

// Value of the ENO-MR reconstruction of window v with the choice given
// (frozen): a tested stencil (table row), or a minmod outcome T, T+1, T+2;
// the same operations as mr_value's evaluation of that choice.
template <int R>
__device__ __forceinline__ double mr_value_forced(const double *v, const double *sA, int sel)
{
    constexpr int g = (R + 1) / 2, W = 2 * g - 1, T = Tab<R>::T, c = g - 1;
    if (sel < T) {
        const double *row = sA + sel * W;
        double val = 0.0;
#pragma unroll
        for (int l = 0; l < W; ++l) val = fma(row[l], v[l], val);
        return val;
    }
    double mm = 0.0;
    if (sel == T) mm = -(v[c] - v[c + 1]);
    if (sel == T + 1) mm = v[c] - v[c - 1];
    return fma(0.5, mm, v[c]);
}

template <int R>
__device__ __forceinline__ void load_a_table(double *sA, int tid, int nthreads)
{
    constexpr int g = (R + 1) / 2, W = 2 * g - 1, T = Tab<R>::T;
    for (int i = tid; i < T * W; i += nthreads) sA[i] = Coef<R>::a_table()[i];
}

// ---------------------------------------------------------------------------
// Epilogue: the flux difference dF = F_{i+1/2} - F_{i-1/2} of a cell ->
// D = -dF / h (+ the other sweep's partial right-hand side) -> output.
// The stage combination is contracted, c0 U^n + c1 (U + dt D) =
// fma(c0, U^n, c1 fma(dt, D, U)): 6 FP64 operations per component instead
// of 7.  The two directional differences are added with both rounded,
// D = Dprev + (-dF / h): a sum that commutes, so a state symmetric under
// exchanging x and y keeps that symmetry bit for bit (an fma there would
// round the two directions differently).
//
// Forms.  The mode (store, or SSP-RK stage), whether an earlier sweep's
// partial right-hand side is added, and (per CTA) whether the tile's flux
// differences are all exactly zero are uniform, so each combination is
// compiled as its own code and chosen by a branch outside the per-cell
// code (with_epilogue_form).  Folded into one body with run-time tests,
// the forms not taken are issued predicated off in every cell, and the FP64
// pipe is charged per warp instruction whether or not a lane is on: in the
// row sweep, whose form is always a plain store, the stage form's and the
// sum's unused instructions took about three quarters of the FP64 issue.
// ---------------------------------------------------------------------------
template <int V> struct IC {
    static constexpr int value = V;
};

template <int MODE, bool PREV, bool ZERO>
__device__ __forceinline__ double epilogue_form(const Epilogue &e, long long idx, double dF,
                                               double inv_h, double Us, bool src, double S)
{
    double D;
    if constexpr (ZERO) {
        // the flux difference is exactly +0 (a tile on one state per line):
        // -dF / h is -0 and Dprev + (-0) is Dprev, bit for bit, without FP64
        D = PREV ? e.Dprev[idx] : -0.0;
    } else {
        // explicitly rounded: with the product feeding the sum directly the
        // compiler would contract them into an fma, and D_x + D_y would no
        // longer commute
        D = __dmul_rn(-dF, inv_h);
        if constexpr (PREV) D = __dadd_rn(e.Dprev[idx], D);
    }
    if (src) D = __dadd_rn(D, S);  // body force, after the two directional differences
    double o;
    if constexpr (MODE == EPI_STORE)
        o = D;
    else if constexpr (MODE == EPI_EULER)
        o = fma(*e.dt_dev, D, Us);
    else
        o = fma(e.c0, e.Un[idx], e.c1 * fma(*e.dt_dev, D, Us));
    e.out[idx] = o;
    return o;
}

// Calls f(IC<form>, IC<prev>) with the launch's epilogue form.  A stage
// with c0 = 0 and c1 = 1 (the first SSP-RK3 stage, the inner stages of the
// linear SSP-RK(m, m-1) family) is a forward-Euler step, U + dt D, with one
// FP64 operation per component instead of three: 1 * x is x, and
// fma(0, U^n, x) is x for every finite U^n except that x = -0 comes out +0,
// the one difference (a zero's sign) between the two forms.
template <class F> __device__ __forceinline__ void with_epilogue_form(const Epilogue &e, F &&f)
{
    if (e.mode == EPI_STORE) {
        if (e.Dprev)
            f(IC<EPI_STORE>{}, IC<1>{});
        else
            f(IC<EPI_STORE>{}, IC<0>{});
    } else if (e.c0 == 0.0 && e.c1 == 1.0) {
        if (e.Dprev)
            f(IC<EPI_EULER>{}, IC<1>{});
        else
            f(IC<EPI_EULER>{}, IC<0>{});
    } else {
        if (e.Dprev)
            f(IC<EPI_STAGE>{}, IC<1>{});
        else
            f(IC<EPI_STAGE>{}, IC<0>{});
    }
}

}  // namespace enomr
