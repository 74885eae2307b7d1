// enomr_internal.h -- launch arguments shared by the API translation unit and
// the per-order kernel translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace enomr {

// Status bits of the device status word (ST_TMA_TIMEOUT: a bounded wait for
// a tile copy of the TMA sweeps ran out and the launch stopped early).
enum : int { ST_NONPHYS_CELL = 1, ST_NONPHYS_ROE = 2, ST_TMA_TIMEOUT = 8 };

// Resident threads per SM of the high-occupancy sweep instances.
constexpr int SWEEP_HIGH_THREADS_PER_SM = 1280;

// Tile shapes of the sweeps (interfaces per line x lines per CTA).
constexpr int E1_TP = 64;
constexpr int X_TP = 128, X_NL = 2;
constexpr int Y_TP = 64, Y_NL = 4;

// Burgers sign flags (second word of AdvArgs::speed): some u < 0, some u > 0
enum : unsigned long long { SGN_NEG = 1ULL, SGN_POS = 2ULL };

// What a sweep does with its flux difference D_i = -(F_{i+1/2}-F_{i-1/2})/h.
enum EpiMode : int {
    EPI_STORE = 0,   // out = D (+ Dprev)
    EPI_STAGE = 1,   // out = c0*Un + c1*(Us + dt*(D (+ Dprev)))
    EPI_EULER = 2    // device form of EPI_STAGE with c0 = 0, c1 = 1: Us + dt*(D (+ Dprev))
};

struct Epilogue {
    int mode;
    double c0, c1;
    const double *dt_dev;  // device scalar dt (EPI_STAGE)
    const double *Un;      // U^n, same layout as the state (EPI_STAGE)
    const double *Dprev;   // partial RHS of an earlier sweep, or nullptr
    double *out;
};

// A boundary side (device copy of enomr_side): kind below / above the
// along-side position split0 + rate t, with an inflow state each
// (conserved, global component order rho, m_x, m_y, E).
enum : int { SIDE_TRANSMISSIVE = 1, SIDE_REFLECTIVE = 2, SIDE_INFLOW = 3 };
struct SideDev {
    int kind_lo, kind_hi;
    double split0, rate;
    double st_lo[4], st_hi[4];
};

// One 1D line sweep of the Euler equations (1D: C = 3; 2D x or y sweep: C = 4).
struct SweepArgs {
    const double *U;       // stage state, [C][ny][nx]
    long long nx, ny;
    int bc;                // 0 periodic, 1 transmissive
    double gm1, inv_gm1, gamma;
    double inv_h;
    const double *alpha;   // [lines][3]: max|un-c|, max|un|, max|un+c|
    double *alpha_next;    // 1D only: accumulate the output state's alpha here, or nullptr
    uint8_t *sel;          // optional selection dump for this sweep
    const uint8_t *sel_in; // optional forced selections (same layout): every
                           // interface is evaluated in full with these choices
    double *ft_out;        // optional: f^+ + f^- per field and interface, [C][lines][nlen+1]
    int *status;
    Epilogue epi;
    // 2D sweeps with boundary sides or a body force (the EXT instances):
    // sides at the low / high end of the lines
    const SideDev *side_lo, *side_hi;
    double pos_h;          // along-side coordinate of line L: (L + 1/2) pos_h
    const double *t_dev;   // time of U^n; the stage is at *t_dev + t_coef * *dt_time
    const double *dt_time;
    double t_coef;
    // body force in line components (normal, tangential); applied when src
    int src;
    double g_n, g_t;
};

struct AdvArgs {
    const double *U;       // [nx]
    long long n;
    int bc;
    double a, inv_h;
    const double *speed;   // Burgers: [max |u|, sign flags as bits] of U
    uint8_t *sel;          // optional [2][n+1]
    Epilogue epi;
};

struct AlphaArgs {
    const double *U;
    long long nx, ny;
    double gm1, gamma, inv_dx, inv_dy;
    double *ax;            // [ny][3], zeroed before the launch
    double *ay;            // [nx][3] (2D only), zeroed before the launch
    double *smax;          // CFL wave-speed max (may be nullptr)
    int *status;
};

// Batched 1D Euler (problem-major packing: problem p's [3][n_p] block starts
// at base[p]).
struct BatchTile {
    int prob;  // problem index
    int x0;    // first interface of the tile
};

struct BatchArgs {
    const double *Us, *Un;
    double *out;
    const long long *base, *n;
    const double *inv_dx;
    const double *alpha;   // [nprob][3] of Us
    double *alpha_next;    // [nprob][3] of out, or nullptr
    const double *dt;      // [nprob]
    const BatchTile *tiles;
    long long ntiles;
    int tiles_per_item;    // consecutive tiles a CTA takes per work item
    int bc;
    double gm1, inv_gm1, gamma, c0, c1;
    int *status;
};

struct BatchAlphaArgs {
    const double *U;
    const long long *base, *n;
    const double *inv_dx;
    const BatchTile *tiles;  // tiles of TP - 1 cells
    long long ntiles;
    int cells_per_tile;
    double gm1, gamma, cfl;
    double *alpha;           // [nprob][3], zeroed before the launch
    int *status;
};

template <int R> cudaError_t launch_batch_stage(const BatchArgs &a, int tp, int grid,
                                                cudaStream_t s);
cudaError_t launch_batch_alpha(const BatchAlphaArgs &a, cudaStream_t s);
cudaError_t launch_batch_dt(const double *alpha, const double *inv_dx, double cfl, long long nprob,
                            double *dt, cudaStream_t s);

template <int R> cudaError_t launch_advection(const AdvArgs &a, cudaStream_t s);
template <int R> cudaError_t launch_burgers(const AdvArgs &a, cudaStream_t s);
template <int R> cudaError_t launch_euler1d(const SweepArgs &a, cudaStream_t s);
// the 2D sweeps; low: the low-occupancy instance (more registers per thread)
template <int R> cudaError_t launch_euler2d_x(const SweepArgs &a, bool low, cudaStream_t s);
template <int R> cudaError_t launch_euler2d_x_ext(const SweepArgs &a, bool low, cudaStream_t s);
template <int R> cudaError_t launch_euler2d_y_ext(const SweepArgs &a, bool low, cudaStream_t s);
template <int R> cudaError_t launch_euler2d_y(const SweepArgs &a, bool low, cudaStream_t s);
}  // namespace enomr

// the sweeps staged by the Tensor Memory Accelerator (enomr_tma.cuh)
struct CUtensorMap_st;
namespace enomr {
template <int R> cudaError_t launch_euler2d_x_tma(const CUtensorMap_st &map, const SweepArgs &a,
                                                  bool low, cudaStream_t s);
template <int R> cudaError_t launch_euler2d_y_tma(const CUtensorMap_st &map, const SweepArgs &a,
                                                  bool low, cudaStream_t s);
// Box extents {x, y, components} of the tile copies of the TMA sweeps: the
// x sweep copies TP + 2g cells (an even count) of X_NL rows, the y sweep
// Y_NL columns of TP + 2g - 1 cells; g = (order + 1) / 2.
inline void tma_box(int order, int dir, unsigned box[3])
{
    box[0] = dir == 0 ? (unsigned)(X_TP + order + 1) : (unsigned)Y_NL;
    box[1] = dir == 0 ? (unsigned)X_NL : (unsigned)(Y_TP + order);
    box[2] = 4;
}

// Transpose-Jacobian product of one sweep (enomr_vjp.cuh).
struct VjpArgs {
    const double *U;      // stage state [C][ny][nx]
    const double *Lbar;   // cotangent of L(U), same layout
    double *Ubar;         // output, accumulated with atomicAdd
    long long nx, ny;
    int bc;
    double gm1, inv_gm1, gamma, inv_h, scale;
    const double *scale_dev;  // if set, the cotangent scale is scale * *scale_dev
    const double *alpha;  // [lines][3]
    double *alpha_bar;    // [lines][3], accumulated
    int *status;
    // optional frozen forward data of this state (written by a forward
    // sweep with sel / ft_out): when given, the kernel reads the selections
    // and the per-field reconstructed values instead of recomputing them
    const uint8_t *sel_in;
    const double *ft_in;
};

template <int R> cudaError_t launch_sweep_vjp(const VjpArgs &a, int C, int dir, cudaStream_t s);
template <int R> cudaError_t launch_advection_vjp(const AdvArgs &a, const double *Lbar,
                                                  double *Ubar, double scale,
                                                  const double *scale_dev, cudaStream_t s);

cudaError_t launch_alpha(int C, const AlphaArgs &a, cudaStream_t s);
cudaError_t launch_scalar_speed(const double *U, long long n, double inv_dx, double *speed,
                                double *smax, int *status, cudaStream_t s);
cudaError_t launch_set_dt(const double *smax, double cfl, double dt_fixed, double *dt_dev,
                          cudaStream_t s);

}  // namespace enomr
