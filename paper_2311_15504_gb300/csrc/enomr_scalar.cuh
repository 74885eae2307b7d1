// enomr_scalar.cuh -- scalar conservation laws: linear advection and the
// inviscid Burgers equation (arXiv 2311.15504, Sec. 4.1, Sec. 4.2).
// One thread per interface; a CTA stages TP + 2g - 1 split flux values.
#pragma once

#include "enomr_kernels.cuh"

namespace enomr {

// ---------------------------------------------------------------------------
// Scalar advection f(u) = a u, alpha = |a|: f^+ = a u, f^- = 0 for a >= 0
// (mirror for a < 0).  One thread per interface.
// ---------------------------------------------------------------------------
template <int R, int TP>
__global__ void __launch_bounds__(TP) k_advection(AdvArgs A)
{
    constexpr int g = (R + 1) / 2, W = 2 * g - 1, S = TP + 2 * g - 1, T = Tab<R>::T;
    __shared__ double sf[S];
    __shared__ double sFh[TP];
    __shared__ double sA[T * W];
    const int p = threadIdx.x;
    const long long x0 = (long long)blockIdx.x * (TP - 1);
    load_a_table<R>(sA, p, TP);
    for (int s = p; s < S; s += TP) sf[s] = A.a * A.U[ghost(x0 - g + s, A.n, A.bc)];
    __syncthreads();
    const long long k = x0 + p;  // interface x_{k-1/2}
    const bool valid = k <= A.n;
    double v[W];
    if (A.a >= 0.0) {
#pragma unroll
        for (int j = 0; j < W; ++j) v[j] = sf[p + j];           // f^+ at cell k-1+l
    } else {
#pragma unroll
        for (int j = 0; j < W; ++j) v[j] = sf[p + 2 * g - 1 - j];  // f^- at cell k-l
    }
    int sel;
    const double fh = mr_value<R>(v, sA, valid, sel);
    sFh[p] = fh;
    if (A.sel && valid) {
        const long long NI = A.n + 1;
        A.sel[(A.a >= 0.0 ? 0 : NI) + k] = (uint8_t)sel;
        A.sel[(A.a >= 0.0 ? NI : 0) + k] = (uint8_t)(T + 2);
    }
    __syncthreads();
    if (p < TP - 1) {
        const long long i = x0 + p;
        if (i < A.n) {
            with_epilogue_form(A.epi, [&](auto M, auto P) {
                epilogue_form<decltype(M)::value, decltype(P)::value != 0, false>(
                    A.epi, i, sFh[p + 1] - sFh[p], A.inv_h, A.U[i], false, 0.0);
            });
        }
    }
}

// ---------------------------------------------------------------------------
// Inviscid Burgers f(u) = u^2/2 (Sec. 4.2).  f'(u) = u: where u keeps one
// sign over the line the flux is not split (f^+ = f, f^- = 0, or the
// mirror); otherwise the global Lax-Friedrichs split with alpha = max |u|.
// The case is uniform over the launch (read from the speed reduction of
// the same state), so a warp never diverges on it.  One thread per
// interface; split values are formed as written, 1/2 (f +- alpha u).
// ---------------------------------------------------------------------------
template <int R, int TP>
__global__ void __launch_bounds__(TP) k_burgers(AdvArgs A)
{
    constexpr int g = (R + 1) / 2, W = 2 * g - 1, S = TP + 2 * g - 1, T = Tab<R>::T;
    __shared__ double sp[S];
    __shared__ double sm[S];
    __shared__ double sFh[TP];
    __shared__ double sA[T * W];
    const int p = threadIdx.x;
    const long long x0 = (long long)blockIdx.x * (TP - 1);
    load_a_table<R>(sA, p, TP);
    const double alpha = A.speed[0];
    const unsigned long long flags = (unsigned long long)__double_as_longlong(A.speed[1]);
    const int mode = !(flags & SGN_NEG) ? 0 : (!(flags & SGN_POS) ? 1 : 2);
    for (int s = p; s < S; s += TP) {
        const double u = A.U[ghost(x0 - g + s, A.n, A.bc)];
        const double f = 0.5 * __dmul_rn(u, u);
        double fp, fm;
        if (mode == 0) {
            fp = f;
            fm = 0.0;
        } else if (mode == 1) {
            fp = 0.0;
            fm = f;
        } else {
            const double au = __dmul_rn(alpha, u);
            fp = 0.5 * __dadd_rn(f, au);
            fm = 0.5 * __dsub_rn(f, au);
        }
        sp[s] = fp;
        sm[s] = fm;
    }
    __syncthreads();
    const long long k = x0 + p;  // interface x_{k-1/2}
    const bool valid = k <= A.n;
    double v[W];
    int selp = T + 2, selm = T + 2;
    double hp = 0.0, hm = 0.0;
    if (mode != 1) {
#pragma unroll
        for (int j = 0; j < W; ++j) v[j] = sp[p + j];           // f^+ at cell k-1+l
        hp = mr_value<R>(v, sA, valid, selp);
    }
    if (mode != 0) {
#pragma unroll
        for (int j = 0; j < W; ++j) v[j] = sm[p + 2 * g - 1 - j];  // f^- at cell k-l
        hm = mr_value<R>(v, sA, valid, selm);
    }
    sFh[p] = __dadd_rn(hp, hm);
    if (A.sel && valid) {
        A.sel[k] = (uint8_t)selp;
        A.sel[A.n + 1 + k] = (uint8_t)selm;
    }
    __syncthreads();
    if (p < TP - 1) {
        const long long i = x0 + p;
        if (i < A.n) {
            with_epilogue_form(A.epi, [&](auto M, auto P) {
                epilogue_form<decltype(M)::value, decltype(P)::value != 0, false>(
                    A.epi, i, sFh[p + 1] - sFh[p], A.inv_h, A.U[i], false, 0.0);
            });
        }
    }
}

}  // namespace enomr
