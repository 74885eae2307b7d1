// enomr_orders.cuh -- launchers of the per-order kernels.  Each
// enomr_o<R>.cu defines ENOMR_R and includes this file, so the seven orders
// compile as separate translation units in parallel.
#pragma once

#include "enomr_scalar.cuh"
#include "enomr_sweep.cuh"
#include "enomr_tma.cuh"
#include "enomr_vjp.cuh"

namespace enomr {

// Interfaces per CTA of the scalar kernels (sweep tile shapes: enomr_sweep.cuh).
constexpr int ADV_TP = 256;

template <int R> cudaError_t launch_advection(const AdvArgs &a, cudaStream_t s)
{
    const long long tiles = (a.n + ADV_TP - 2) / (ADV_TP - 1);
    k_advection<R, ADV_TP><<<(unsigned)tiles, ADV_TP, 0, s>>>(a);
    return cudaGetLastError();
}

template <int R> cudaError_t launch_burgers(const AdvArgs &a, cudaStream_t s)
{
    const long long tiles = (a.n + ADV_TP - 2) / (ADV_TP - 1);
    k_burgers<R, ADV_TP><<<(unsigned)tiles, ADV_TP, 0, s>>>(a);
    return cudaGetLastError();
}

template <int R> cudaError_t launch_euler1d(const SweepArgs &a, cudaStream_t s)
{
    const long long tiles = (a.nx + E1_TP - 2) / (E1_TP - 1);
    k_sweep<R, 3, 0, E1_TP, 1><<<dim3((unsigned)tiles, 1), E1_TP, 0, s>>>(a);
    return cudaGetLastError();
}

// Tiles of the 2D sweeps (the grid of one launch of the loading instances).
inline dim3 grid_x(const SweepArgs &a)
{
    return dim3((unsigned)((a.nx + X_TP - 2) / (X_TP - 1)), (unsigned)((a.ny + X_NL - 1) / X_NL));
}
inline dim3 grid_y(const SweepArgs &a)
{
    return dim3((unsigned)((a.nx + Y_NL - 1) / Y_NL), (unsigned)((a.ny + Y_TP - 2) / (Y_TP - 1)));
}

template <int R> cudaError_t launch_euler2d_x(const SweepArgs &a, bool low, cudaStream_t s)
{
    if (!row_epilogue_ok(a)) return cudaErrorInvalidValue;
    if (low)
        k_sweep<R, 4, 0, X_TP, X_NL, false, SWEEP_LOW_CTAS><<<grid_x(a), X_TP * X_NL, 0, s>>>(a);
    else
        k_sweep<R, 4, 0, X_TP, X_NL><<<grid_x(a), X_TP * X_NL, 0, s>>>(a);
    return cudaGetLastError();
}

template <int R> cudaError_t launch_euler2d_y(const SweepArgs &a, bool low, cudaStream_t s)
{
    if (low)
        k_sweep<R, 4, 1, Y_TP, Y_NL, false, SWEEP_LOW_CTAS><<<grid_y(a), Y_TP * Y_NL, 0, s>>>(a);
    else
        k_sweep<R, 4, 1, Y_TP, Y_NL><<<grid_y(a), Y_TP * Y_NL, 0, s>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_advection<ENOMR_R>(const AdvArgs &, cudaStream_t);
template cudaError_t launch_burgers<ENOMR_R>(const AdvArgs &, cudaStream_t);
template cudaError_t launch_euler1d<ENOMR_R>(const SweepArgs &, cudaStream_t);
// with boundary sides / body force (the 2D problems of Sec. 4.4)
template <int R> cudaError_t launch_euler2d_x_ext(const SweepArgs &a, bool low, cudaStream_t s)
{
    if (!row_epilogue_ok(a)) return cudaErrorInvalidValue;
    if (low)
        k_sweep<R, 4, 0, X_TP, X_NL, true, SWEEP_LOW_CTAS><<<grid_x(a), X_TP * X_NL, 0, s>>>(a);
    else
        k_sweep<R, 4, 0, X_TP, X_NL, true><<<grid_x(a), X_TP * X_NL, 0, s>>>(a);
    return cudaGetLastError();
}

template <int R> cudaError_t launch_euler2d_y_ext(const SweepArgs &a, bool low, cudaStream_t s)
{
    if (low)
        k_sweep<R, 4, 1, Y_TP, Y_NL, true, SWEEP_LOW_CTAS><<<grid_y(a), Y_TP * Y_NL, 0, s>>>(a);
    else
        k_sweep<R, 4, 1, Y_TP, Y_NL, true><<<grid_y(a), Y_TP * Y_NL, 0, s>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_euler2d_x<ENOMR_R>(const SweepArgs &, bool, cudaStream_t);
template cudaError_t launch_euler2d_y<ENOMR_R>(const SweepArgs &, bool, cudaStream_t);
template cudaError_t launch_euler2d_x_ext<ENOMR_R>(const SweepArgs &, bool, cudaStream_t);
template cudaError_t launch_euler2d_y_ext<ENOMR_R>(const SweepArgs &, bool, cudaStream_t);

}  // namespace enomr

namespace enomr {

template <int R> cudaError_t launch_batch_stage(const BatchArgs &a, int tp, int grid,
                                                cudaStream_t s)
{
    switch (tp) {
    case 32: k_batch_stage<R, 32><<<grid, 32, 0, s>>>(a); break;
    case 64: k_batch_stage<R, 64><<<grid, 64, 0, s>>>(a); break;
    case 128: k_batch_stage<R, 128><<<grid, 128, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template cudaError_t launch_batch_stage<ENOMR_R>(const BatchArgs &, int, int, cudaStream_t);

}  // namespace enomr

namespace enomr {

template <int R> cudaError_t launch_sweep_vjp(const VjpArgs &a, int C, int dir, cudaStream_t s)
{
    if (C == 3) {
        const long long tiles = (a.nx + 62) / 63;
        k_sweep_vjp<R, 3, 0, 64, 1><<<dim3((unsigned)tiles, 1), 64, 0, s>>>(a);
    } else if (dir == 0) {
        const long long tx = (a.nx + 62) / 63;
        k_sweep_vjp<R, 4, 0, 64, 1><<<dim3((unsigned)tx, (unsigned)a.ny), 64, 0, s>>>(a);
    } else {
        const long long tx = (a.nx + 1) / 2;
        const long long ty = (a.ny + 30) / 31;
        k_sweep_vjp<R, 4, 1, 32, 2><<<dim3((unsigned)tx, (unsigned)ty), 64, 0, s>>>(a);
    }
    return cudaGetLastError();
}

template <int R> cudaError_t launch_advection_vjp(const AdvArgs &a, const double *Lbar, double *Ubar,
                                                  double scale, const double *scale_dev,
                                                  cudaStream_t s)
{
    const long long tiles = (a.n + ADV_TP - 2) / (ADV_TP - 1);
    k_advection_vjp<R, ADV_TP><<<(unsigned)tiles, ADV_TP, 0, s>>>(a, Lbar, Ubar, scale, scale_dev);
    return cudaGetLastError();
}

template cudaError_t launch_sweep_vjp<ENOMR_R>(const VjpArgs &, int, int, cudaStream_t);
template cudaError_t launch_advection_vjp<ENOMR_R>(const AdvArgs &, const double *, double *, double,
                                                   const double *, cudaStream_t);

}  // namespace enomr

namespace enomr {

template <int R> cudaError_t launch_euler2d_x_tma(const CUtensorMap &map, const SweepArgs &a,
                                                  bool low, cudaStream_t s)
{
    return low ? launch_sweep_tma<R, 0, X_TP, X_NL, SWEEP_LOW_CTAS, true>(map, a, s)
               : launch_sweep_tma<R, 0, X_TP, X_NL, TmaCtas<R, 0, X_TP, X_NL>::value, false>(map, a,
                                                                                          s);
}

template <int R> cudaError_t launch_euler2d_y_tma(const CUtensorMap &map, const SweepArgs &a,
                                                  bool low, cudaStream_t s)
{
    return low ? launch_sweep_tma<R, 1, Y_TP, Y_NL, SWEEP_LOW_CTAS, true>(map, a, s)
               : launch_sweep_tma<R, 1, Y_TP, Y_NL, TmaCtas<R, 1, Y_TP, Y_NL>::value, false>(map, a,
                                                                                          s);
}

template cudaError_t launch_euler2d_x_tma<ENOMR_R>(const CUtensorMap &, const SweepArgs &, bool,
                                                   cudaStream_t);
template cudaError_t launch_euler2d_y_tma<ENOMR_R>(const CUtensorMap &, const SweepArgs &, bool,
                                                   cudaStream_t);

}  // namespace enomr
