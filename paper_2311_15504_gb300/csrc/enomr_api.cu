// enomr_api.cu -- host side of libenomr.so: context, argument checks,
// per-line alpha / CFL reduction kernel and the RK3 stage sequencing.
// The C ABI is declared in include/enomr.h.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <new>

#include "../../include/enomr.h"
#include "enomr_common.cuh"
#include "enomr_internal.h"

using namespace enomr;

struct enomr_ctx {
    int eq, ndim, order, bc;
    long long nx, ny;
    double dx, dy, gamma, adv;
    cudaStream_t stream;
    double *ax, *ay;   // per-line alpha [ny][3], [nx][3]
    double *smax;      // CFL wave-speed maximum
    double *dt;        // device dt
    int *status;
    double *U1, *U2;   // SSP-RK3 stage buffers
    double *D;         // 2D: x-sweep partial RHS
    long long nstate;  // doubles in one state
    // adjoint scratch: argmax cell of each alpha, alpha cotangents, stage cotangents
    unsigned long long *ix, *iy;
    double *axb, *ayb;
    double *Ub1, *Ub2;
    // forward data of the recomputed stages U^n and U^(1) for the adjoint
    uint8_t *fsel[2];
    double *fft[2];
    long long nsel, nft;
    // optional per-kernel event timing (enomr_profile_begin/end)
    int prof_kernel, prof_max, prof_n;
    cudaEvent_t *prof_ev;
    // boundary sides (x low, x high, y low, y high), body force, time
    SideDev *sides_d;
    bool custom_sides;
    double gx, gy;
    double *t_dev;
    // staging of the 2D sweeps: ENOMR_STAGING_AUTO / _LOADS / _TMA
    int staging;
    // occupancy of the 2D sweeps: ENOMR_OCCUPANCY_AUTO / _HIGH / _LOW
    int occupancy;
    int sms;  // SMs of the device the context was created on
};

static void prof_start(enomr_ctx *c, int k)
{
    if (c->prof_kernel == k && c->prof_n < c->prof_max)
        cudaEventRecord(c->prof_ev[2 * c->prof_n], c->stream);
}

static void prof_stop(enomr_ctx *c, int k)
{
    if (c->prof_kernel == k && c->prof_n < c->prof_max) {
        cudaEventRecord(c->prof_ev[2 * c->prof_n + 1], c->stream);
        c->prof_n++;
    }
}

namespace enomr {

// ---------------------------------------------------------------------------
// alpha_k per line (reading of Eq. LF_Flux_Split for systems: per
// characteristic field, max over the cells of the line) and the CFL
// wave-speed maximum.  Tile: 32 columns x 32 rows, 256 threads; thread
// (tx, ty) reads rows 4 ty .. 4 ty + 3 of column tx.
// Maxima of non-negative doubles are taken on their bit patterns.
//
// Only representative cells are evaluated.  A cell whose state is bitwise
// equal to its left neighbour's has that neighbour's speeds: it changes
// neither its row's maxima nor the CFL maximum.  One equal to the cell above
// changes none of its column's maxima.  So each row's maxima are attained
// at a row representative (the first cell of its tile row, or one that
// differs from its left neighbour) and each column's at a column
// representative (likewise along the column).  The neighbours are compared
// across tile edges too (the column left of the tile and the row above it
// are read for that), so the first cell of a run of equal cells along a
// line, the one that carries the run's speeds, is the only representative
// it needs, and a tile inside a constant region evaluates nothing.  Every
// other cell is skipped, and so is its status check, which its equal
// neighbour's covers.  The
// representatives are compacted into a list that whole warps evaluate, so
// skipped cells take no FP64 issue slots.  Every evaluated cell updates its
// row, its column and the CFL maximum with its own speeds: the results are
// the maxima over all cells, bit for bit.
// ---------------------------------------------------------------------------
template <int C>
__global__ void __launch_bounds__(256, 5) k_alpha(AlphaArgs A)
{
    __shared__ unsigned long long srow[32][3], scol[32][3], scfl;
    __shared__ unsigned short list[1024];  // tile cell index: row * 32 + column
    __shared__ int nlist;
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const long long x = (long long)blockIdx.x * 32 + tx;
    const long long ty0 = (long long)blockIdx.y * 32, y0 = ty0 + 4 * ty;
    const long long ncell = A.nx * A.ny;
    if (tid < 96) {
        srow[tid / 3][tid % 3] = 0;
        scol[tid / 3][tid % 3] = 0;
    }
    if (tid == 0) {
        scfl = 0;
        nlist = 0;
    }
    // the cell above this thread's first row (in the tile above for ty = 0)
    double up[C] = {};
    bool have_up = false;
    if (C == 4 && y0 > 0 && x < A.nx && y0 < A.ny) {
        const long long i = (y0 - 1) * A.nx + x;
#pragma unroll
        for (int q = 0; q < C; ++q) up[q] = A.U[q * ncell + i];
        have_up = true;
    }
    // the column left of the tile for this warp's rows: lane l < 4 C holds
    // component l % C of row 4 ty + l / C
    const long long xl = (long long)blockIdx.x * 32 - 1;
    double lv = 0.0;
    if (xl >= 0 && tx < 4 * C && y0 + tx / C < A.ny)
        lv = A.U[(tx % C) * ncell + (y0 + tx / C) * A.nx + xl];
    // all of this thread's loads first (4 rows x C components in flight),
    // then the comparisons and the list appends
    double ur[4][C];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const long long y = y0 + j;
        const bool valid = x < A.nx && y < A.ny;
#pragma unroll
        for (int q = 0; q < C; ++q) ur[j][q] = valid ? A.U[q * ncell + y * A.nx + x] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const long long y = y0 + j;
        const bool valid = x < A.nx && y < A.ny;
        double u[C];
#pragma unroll
        for (int q = 0; q < C; ++q) u[q] = ur[j][q];
        bool same_left = tx > 0 || xl >= 0;
#pragma unroll
        for (int q = 0; q < C; ++q) {
            const double li = __shfl_up_sync(0xffffffffu, u[q], 1);
            const double lo = __shfl_sync(0xffffffffu, lv, j * C + q);
            const double l = tx > 0 ? li : lo;
            same_left = same_left && (__double_as_longlong(l) == __double_as_longlong(u[q]));
        }
        bool rep = valid && !same_left;
        if (C == 4) {
            bool same_up = j > 0 || have_up;
#pragma unroll
            for (int q = 0; q < C; ++q)
                same_up = same_up && (__double_as_longlong(up[q]) == __double_as_longlong(u[q]));
            rep = rep || (valid && !same_up);
#pragma unroll
            for (int q = 0; q < C; ++q) up[q] = u[q];
        }
        const unsigned need = __ballot_sync(0xffffffffu, rep);
        if (need) {
            int base = 0;
            if (tx == 0) base = atomicAdd(&nlist, __popc(need));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (rep)
                list[base + __popc(need & ((1u << tx) - 1u))] =
                    (unsigned short)((4 * ty + j) * 32 + tx);
        }
    }
    __syncthreads();
    const int n = nlist;
    if (n == 0) return;  // every cell repeats one outside the tile
    for (int b = ty * 32; b < n; b += 256) {
        const int t = b + tx;
        if (t < n) {
            const int e = list[t], r = e >> 5, cx = e & 31;
            const long long i = (ty0 + r) * A.nx + (long long)blockIdx.x * 32 + cx;
            const CellWaves cw = cell_waves<C>(A.U[i], A.U[ncell + i],
                                               (C == 4) ? A.U[2 * ncell + i] : 0.0,
                                               A.U[(C - 1) * ncell + i], A.gm1, A.gamma, A.status);
            const double u = cw.u, v = cw.v, c = cw.c;
            atomicMax(&srow[r][0], (unsigned long long)__double_as_longlong(fabs(__dsub_rn(u, c))));
            atomicMax(&srow[r][1], (unsigned long long)__double_as_longlong(fabs(u)));
            atomicMax(&srow[r][2], (unsigned long long)__double_as_longlong(fabs(__dadd_rn(u, c))));
            if (C == 4) {
                atomicMax(&scol[cx][0], (unsigned long long)__double_as_longlong(fabs(__dsub_rn(v, c))));
                atomicMax(&scol[cx][1], (unsigned long long)__double_as_longlong(fabs(v)));
                atomicMax(&scol[cx][2], (unsigned long long)__double_as_longlong(fabs(__dadd_rn(v, c))));
            }
            double s = __dmul_rn(__dadd_rn(fabs(u), c), A.inv_dx);
            if (C == 4) s = __fma_rn(__dadd_rn(fabs(v), c), A.inv_dy, s);
            atomicMax(&scfl, (unsigned long long)__double_as_longlong(s));
        }
    }
    __syncthreads();
    if (tid < 32) {
        const long long y = ty0 + tid;
        if (y < A.ny)
            for (int k = 0; k < 3; ++k) atomicMax((unsigned long long *)(A.ax + 3 * y + k), srow[tid][k]);
        if (C == 4 && x < A.nx)
            for (int k = 0; k < 3; ++k) atomicMax((unsigned long long *)(A.ay + 3 * x + k), scol[tid][k]);
    }
    if (tid == 0 && A.smax) atomicMax((unsigned long long *)A.smax, scfl);
}

// First cell (smallest index along its line) whose wave speed equals the
// line's alpha bit for bit: the frozen argmax of the adjoint.
template <int C>
__global__ void __launch_bounds__(256) k_alpha_argmax(AlphaArgs A, unsigned long long *ix,
                                                     unsigned long long *iy)
{
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const long long x = (long long)blockIdx.x * 32 + tx;
    const long long ncell = A.nx * A.ny;
    for (int r = 0; r < 4; ++r) {
        const long long y = (long long)blockIdx.y * 32 + ty + 8 * r;
        if (x >= A.nx || y >= A.ny) continue;
        const long long i = y * A.nx + x;
        const CellWaves cw = cell_waves<C>(A.U[i], A.U[ncell + i], (C == 4) ? A.U[2 * ncell + i] : 0.0,
                                           A.U[(C - 1) * ncell + i], A.gm1, A.gamma, A.status);
        const double sx[3] = {fabs(__dsub_rn(cw.u, cw.c)), fabs(cw.u), fabs(__dadd_rn(cw.u, cw.c))};
        for (int k = 0; k < 3; ++k)
            if (__double_as_longlong(sx[k]) == __double_as_longlong(A.ax[3 * y + k]))
                atomicMin(ix + 3 * y + k, (unsigned long long)x);
        if (C == 4) {
            const double sy[3] = {fabs(__dsub_rn(cw.v, cw.c)), fabs(cw.v), fabs(__dadd_rn(cw.v, cw.c))};
            for (int k = 0; k < 3; ++k)
                if (__double_as_longlong(sy[k]) == __double_as_longlong(A.ay[3 * x + k]))
                    atomicMin(iy + 3 * x + k, (unsigned long long)y);
        }
    }
}

// alpha_k = |lambda_k(U_a)| at the frozen argmax cell a: add
// alpha_bar * sign(lambda_k) * d lambda_k / dU to Ubar(a).  One thread per
// (line, k); lines 0..ny-1 are rows (x sweep), then nx columns (y sweep).
template <int C>
__global__ void k_alpha_vjp(const double *U, long long nx, long long ny, double gm1, double gamma,
                            const unsigned long long *ix, const unsigned long long *iy,
                            const double *axb, const double *ayb, double *Ubar)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nl = (C == 4) ? ny + nx : ny;
    if (t >= 3 * nl) return;
    const long long line = t / 3;
    const int k = (int)(t - 3 * line);
    const bool ysw = line >= ny;
    const double ab = ysw ? ayb[3 * (line - ny) + k] : axb[3 * line + k];
    const unsigned long long a = ysw ? iy[3 * (line - ny) + k] : ix[3 * line + k];
    if (ab == 0.0 || a == ~0ULL) return;
    const long long ncell = nx * ny;
    const long long i = ysw ? (long long)a * nx + (line - ny) : line * nx + (long long)a;
    const int qn = ysw ? 2 : 1, qt = ysw ? 1 : 2;
    const double rho = U[i], mn = U[qn * ncell + i], E = U[(C - 1) * ncell + i];
    const double mt = (C == 4) ? U[qt * ncell + i] : 0.0;
    const double ir = 1.0 / rho;
    const double un = mn * ir, ut = mt * ir;
    const double p = gm1 * (E - 0.5 * rho * (un * un + ut * ut));
    const double c = sqrt(gamma * p * ir);
    const double lam = (k == 0) ? un - c : ((k == 1) ? un : un + c);
    const double lb = (lam > 0.0) ? ab : ((lam < 0.0) ? -ab : 0.0);
    const double un_b = lb;
    const double c_b = (k == 0) ? -lb : ((k == 2) ? lb : 0.0);
    const double p_b = c_b * gamma * ir / (2.0 * c);
    double r_b = -c_b * c * ir * 0.5 - un_b * un * ir + p_b * 0.5 * gm1 * (un * un + ut * ut);
    const double mn_b = un_b * ir - p_b * gm1 * un;
    const double mt_b = -p_b * gm1 * ut;
    const double E_b = p_b * gm1;
    atomicAdd(Ubar + i, r_b);
    atomicAdd(Ubar + qn * ncell + i, mn_b);
    if (C == 4) atomicAdd(Ubar + qt * ncell + i, mt_b);
    atomicAdd(Ubar + (C - 1) * ncell + i, E_b);
}

// alpha_k of every line evaluated at a given cell of the line (the frozen
// argmax cells of a reference state): |lambda_k(U_a)|, by the same helper
// as k_alpha, so with the reference state itself the maxima come back bit
// for bit.  One thread per (line, k); rows (x sweep) first, then columns.
template <int C>
__global__ void k_alpha_at(const double *U, long long nx, long long ny, double gm1, double gamma,
                           const unsigned long long *ix, const unsigned long long *iy,
                           double *ax, double *ay, int *status)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nl = (C == 4) ? ny + nx : ny;
    if (t >= 3 * nl) return;
    const long long line = t / 3;
    const int k = (int)(t - 3 * line);
    const bool ysw = line >= ny;
    const unsigned long long a = ysw ? iy[3 * (line - ny) + k] : ix[3 * line + k];
    double *out = ysw ? ay + 3 * (line - ny) + k : ax + 3 * line + k;
    const long long nlen = ysw ? ny : nx;
    if (a >= (unsigned long long)nlen) {  // no cell attained the maximum (non-finite state)
        *out = __longlong_as_double(0x7ff8000000000000LL);
        atomicOr(status, ST_NONPHYS_CELL);
        return;
    }
    const long long ncell = nx * ny;
    const long long i = ysw ? (long long)a * nx + (line - ny) : line * nx + (long long)a;
    const CellWaves cw = cell_waves<C>(U[i], U[ncell + i], (C == 4) ? U[2 * ncell + i] : 0.0,
                                       U[(C - 1) * ncell + i], gm1, gamma, status);
    const double un = ysw ? cw.v : cw.u;
    *out = (k == 0) ? fabs(__dsub_rn(un, cw.c)) : ((k == 1) ? fabs(un) : fabs(__dadd_rn(un, cw.c)));
}

// y = a x (+ y if acc)
__global__ void k_axpy(long long n, double a, const double *x, double *y, int acc)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = acc ? fma(a, x[i], y[i]) : a * x[i];
}

__global__ void k_set_dt(const double *smax, double cfl, double dt_fixed, double *dt)
{
    // a state without any wave speed (Burgers with u = 0) is steady: dt = 0;
    // a non-finite maximum (a non-physical state, flagged in the status
    // word) gives NaN, never a step that does not advance
    const double sm = *smax;
    *dt = dt_fixed > 0.0 ? dt_fixed
                         : ((sm > 0.0 && sm < __longlong_as_double(0x7ff0000000000000LL))
                                ? cfl / sm
                                : (sm == 0.0 ? 0.0 : __longlong_as_double(0x7ff8000000000000LL)));
}

__global__ void k_advance_time(double *t, const double *dt, double mult)
{
    *t = *t + mult * *dt;
}

// Burgers: max |u| over the line (the Lax-Friedrichs alpha and the CFL
// speed, f'(u) = u) and which signs occur.  speed[0] and speed[1] are
// zeroed before the launch; maxima are taken on the bit patterns.
__global__ void __launch_bounds__(256) k_scalar_speed(const double *U, long long n, double inv_dx,
                                                      double *speed, double *smax, int *status)
{
    unsigned long long m = 0, fl = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long b = __double_as_longlong(U[i]);
        const unsigned long long a = (unsigned long long)(b & 0x7fffffffffffffffLL);
        if (!below_1e300(U[i])) atomicOr(status, ST_NONPHYS_CELL);
        m = m > a ? m : a;
        if (a != 0) fl |= (b < 0) ? SGN_NEG : SGN_POS;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, m, o);
        m = m > w ? m : w;
        fl |= __shfl_xor_sync(0xffffffffu, fl, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax((unsigned long long *)speed, m);
        if (fl) atomicOr((unsigned long long *)(speed + 1), fl);
        if (smax) {
            const double s = __dmul_rn(__longlong_as_double((long long)m), inv_dx);
            atomicMax((unsigned long long *)smax, (unsigned long long)__double_as_longlong(s));
        }
    }
}

cudaError_t launch_scalar_speed(const double *U, long long n, double inv_dx, double *speed,
                                double *smax, int *status, cudaStream_t s)
{
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_scalar_speed<<<(unsigned)blocks, 256, 0, s>>>(U, n, inv_dx, speed, smax, status);
    return cudaGetLastError();
}

cudaError_t launch_alpha(int C, const AlphaArgs &a, cudaStream_t s)
{
    dim3 grid((unsigned)((a.nx + 31) / 32), (unsigned)((a.ny + 31) / 32));
    if (C == 4)
        k_alpha<4><<<grid, 256, 0, s>>>(a);
    else
        k_alpha<3><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_set_dt(const double *smax, double cfl, double dt_fixed, double *dt_dev,
                          cudaStream_t s)
{
    k_set_dt<<<1, 1, 0, s>>>(smax, cfl, dt_fixed, dt_dev);
    return cudaGetLastError();
}

}  // namespace enomr

// ---------------------------------------------------------------------------
// dispatch helpers
// ---------------------------------------------------------------------------
template <template <int> class F, typename... Args>
static cudaError_t by_order(int R, Args &&...args)
{
    switch (R) {
    case 5: return F<5>::run(args...);
    case 7: return F<7>::run(args...);
    case 9: return F<9>::run(args...);
    case 11: return F<11>::run(args...);
    case 13: return F<13>::run(args...);
    case 15: return F<15>::run(args...);
    case 17: return F<17>::run(args...);
    default: return cudaErrorInvalidValue;
    }
}

template <int R> struct AdvF {
    static cudaError_t run(const AdvArgs &a, cudaStream_t s) { return launch_advection<R>(a, s); }
};
template <int R> struct BurgF {
    static cudaError_t run(const AdvArgs &a, cudaStream_t s) { return launch_burgers<R>(a, s); }
};
template <int R> struct E1F {
    static cudaError_t run(const SweepArgs &a, cudaStream_t s) { return launch_euler1d<R>(a, s); }
};
template <int R> struct E2XF {
    static cudaError_t run(const SweepArgs &a, bool low, cudaStream_t s)
    {
        return launch_euler2d_x<R>(a, low, s);
    }
};
template <int R> struct E2XEF {
    static cudaError_t run(const SweepArgs &a, bool low, cudaStream_t s)
    {
        return launch_euler2d_x_ext<R>(a, low, s);
    }
};
template <int R> struct E2YEF {
    static cudaError_t run(const SweepArgs &a, bool low, cudaStream_t s)
    {
        return launch_euler2d_y_ext<R>(a, low, s);
    }
};
template <int R> struct E2YF {
    static cudaError_t run(const SweepArgs &a, bool low, cudaStream_t s)
    {
        return launch_euler2d_y<R>(a, low, s);
    }
};
template <int R> struct E2XTF {
    static cudaError_t run(const CUtensorMap &m, const SweepArgs &a, bool low, cudaStream_t s)
    {
        return launch_euler2d_x_tma<R>(m, a, low, s);
    }
};
template <int R> struct E2YTF {
    static cudaError_t run(const CUtensorMap &m, const SweepArgs &a, bool low, cudaStream_t s)
    {
        return launch_euler2d_y_tma<R>(m, a, low, s);
    }
};

// cuTensorMapEncodeTiled from the driver, looked up once (nullptr if the
// driver does not provide it: the sweeps then stage with plain loads).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// Tensor map of a 2D Euler state U [4][ny][nx] with the box of sweep dir.
// A tile copy needs 16-byte aligned rows (nx even), a 16-byte aligned base
// and 32-bit coordinates; otherwise false (the sweeps then use plain loads).
static bool state_map(const enomr_ctx *c, const double *U, int dir, CUtensorMap *m)
{
    if ((c->nx & 1) || (reinterpret_cast<uintptr_t>(U) & 15) || c->nx > (1LL << 30) ||
        c->ny > (1LL << 30))
        return false;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)c->nx, (cuuint64_t)c->ny, 4};
    const cuuint64_t strides[2] = {(cuuint64_t)c->nx * 8, (cuuint64_t)(c->nx * c->ny) * 8};
    unsigned b[3];
    tma_box(c->order, dir, b);
    const cuuint32_t box[3] = {b[0], b[1], b[2]};
    const cuuint32_t es[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<double *>(U), dims, strides, box,
               es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int R> struct VjpF {
    static cudaError_t run(const VjpArgs &a, int C, int dir, cudaStream_t s)
    {
        return launch_sweep_vjp<R>(a, C, dir, s);
    }
};
template <int R> struct AdvVjpF {
    static cudaError_t run(const AdvArgs &a, const double *Lb, double *Ub, double sc,
                           const double *sc_dev, cudaStream_t s)
    {
        return launch_advection_vjp<R>(a, Lb, Ub, sc, sc_dev, s);
    }
};

static enomr_status cu(cudaError_t e) { return e == cudaSuccess ? ENOMR_OK : ENOMR_ECUDA; }

#define CU_TRY(expr)                              \
    do {                                          \
        enomr_status st_ = cu(expr);              \
        if (st_ != ENOMR_OK) return st_;          \
    } while (0)

static int valid_order(int R) { return R >= 5 && R <= 17 && (R % 2) == 1; }

// Per-line alpha of state U (zeroes the maxima first); smax on request.
static enomr_status compute_alpha(enomr_ctx *c, const double *U, bool want_smax)
{
    if (c->eq == ENOMR_ADVECTION) return ENOMR_OK;
    if (c->eq == ENOMR_BURGERS) {
        CU_TRY(cudaMemsetAsync(c->ax, 0, sizeof(double) * 2, c->stream));
        if (want_smax) CU_TRY(cudaMemsetAsync(c->smax, 0, sizeof(double), c->stream));
        prof_start(c, 3);
        cudaError_t e = launch_scalar_speed(U, c->nx, 1.0 / c->dx, c->ax,
                                            want_smax ? c->smax : nullptr, c->status, c->stream);
        prof_stop(c, 3);
        return cu(e);
    }
    const int C = c->ndim == 2 ? 4 : 3;
    CU_TRY(cudaMemsetAsync(c->ax, 0, sizeof(double) * 3 * c->ny, c->stream));
    if (C == 4) CU_TRY(cudaMemsetAsync(c->ay, 0, sizeof(double) * 3 * c->nx, c->stream));
    if (want_smax) CU_TRY(cudaMemsetAsync(c->smax, 0, sizeof(double), c->stream));
    AlphaArgs a;
    a.U = U;
    a.nx = c->nx;
    a.ny = c->ny;
    a.gm1 = c->gamma - 1.0;
    a.gamma = c->gamma;
    a.inv_dx = 1.0 / c->dx;
    a.inv_dy = 1.0 / c->dy;
    a.ax = c->ax;
    a.ay = c->ay;
    a.smax = want_smax ? c->smax : nullptr;
    a.status = c->status;
    prof_start(c, 3);
    cudaError_t e = launch_alpha(C, a, c->stream);
    prof_stop(c, 3);
    return cu(e);
}

static SweepArgs sweep_args(enomr_ctx *c, const double *U, bool ysweep)
{
    SweepArgs a;
    a.U = U;
    a.nx = c->nx;
    a.ny = c->ny;
    a.bc = c->bc;
    a.gamma = c->gamma;
    a.gm1 = c->gamma - 1.0;
    a.inv_gm1 = 1.0 / (c->gamma - 1.0);
    a.inv_h = 1.0 / (ysweep ? c->dy : c->dx);
    a.alpha = ysweep ? c->ay : c->ax;
    a.alpha_next = nullptr;
    a.sel = nullptr;
    a.sel_in = nullptr;
    a.ft_out = nullptr;
    a.status = c->status;
    memset(&a.epi, 0, sizeof(a.epi));
    a.side_lo = c->sides_d + (ysweep ? 2 : 0);
    a.side_hi = c->sides_d + (ysweep ? 3 : 1);
    a.pos_h = ysweep ? c->dx : c->dy;
    a.t_dev = c->t_dev;
    a.dt_time = c->dt;
    a.t_coef = 0.0;
    // the body force is added by the sweep that finishes the right-hand side
    a.src = (c->gx != 0.0 || c->gy != 0.0) && ysweep;
    a.g_n = ysweep ? c->gy : c->gx;
    a.g_t = ysweep ? c->gx : c->gy;
    return a;
}

// boundary sides or a body force: the 2D sweeps' EXT instances
static bool extended(const enomr_ctx *c)
{
    return c->custom_sides || c->gx != 0.0 || c->gy != 0.0;
}

// The 2D sweeps' low-occupancy instances: forced, or (automatic) for grids
// whose x sweep has fewer tiles than four waves of the high-occupancy
// instance.  Measured on GB300 (order 9): the paper's RP1 801^2 (3.7 waves),
// double Mach reflection 1200x300 and Rayleigh-Taylor 200x800 whole runs
// are 3-7 % faster with the low instance, the four-quadrant Riemann state at
// 1024^2 (11 waves) and above is 30-40 % slower with it.
static bool low_occupancy(const enomr_ctx *c)
{
    if (c->occupancy == ENOMR_OCCUPANCY_LOW) return true;
    if (c->occupancy == ENOMR_OCCUPANCY_HIGH) return false;
    const long long tiles = ((c->nx + X_TP - 2) / (X_TP - 1)) * ((c->ny + X_NL - 1) / X_NL);
    return tiles < 4LL * c->sms * (SWEEP_HIGH_THREADS_PER_SM / (X_TP * X_NL));
}

// Evaluate L(U) into the epilogue.  The alpha of U must be current.
static enomr_status rhs_with_epilogue(enomr_ctx *c, const double *U, const Epilogue &epi,
                                      uint8_t *sel, double *ft = nullptr, double t_coef = 0.0,
                                      const uint8_t *sel_in = nullptr)
{
    if (c->eq == ENOMR_ADVECTION || c->eq == ENOMR_BURGERS) {
        AdvArgs a;
        a.U = U;
        a.n = c->nx;
        a.bc = c->bc;
        a.a = c->adv;
        a.inv_h = 1.0 / c->dx;
        a.speed = c->ax;
        a.sel = sel;
        a.epi = epi;
        prof_start(c, 1);
        cudaError_t e = c->eq == ENOMR_ADVECTION ? by_order<AdvF>(c->order, a, c->stream)
                                                 : by_order<BurgF>(c->order, a, c->stream);
        prof_stop(c, 1);
        return cu(e);
    }
    if (c->ndim == 1) {
        SweepArgs a = sweep_args(c, U, false);
        a.sel = sel;
        a.ft_out = ft;
        a.epi = epi;
        prof_start(c, 1);
        cudaError_t e = by_order<E1F>(c->order, a, c->stream);
        prof_stop(c, 1);
        return cu(e);
    }
    // 2D: x sweep -> D, y sweep adds D and applies the epilogue.  The plain
    // sweeps stage their tiles by TMA where the state allows it (same
    // results bit for bit); the EXT instances always load.
    const bool ext = extended(c);
    CUtensorMap mx, my;
    const bool tma = !ext && c->staging != ENOMR_STAGING_LOADS && state_map(c, U, 0, &mx) &&
                     state_map(c, U, 1, &my);
    if (c->staging == ENOMR_STAGING_TMA && !tma) return ENOMR_EINVAL;
    const bool low = low_occupancy(c);
    // Automatic staging: TMA for both sweeps wherever the state allows it
    // (measured on GB300, 4096^2 Riemann state, orders 5-17: faster at every
    // order in both directions, e.g. row sweep 0.35 against 0.39 ms and
    // column sweep 0.75 against 0.81 ms at order 9, 0.58 against 0.74 and
    // 1.17 against 1.35 ms at order 17).
    const bool tma_x = tma;
    const bool tma_y = tma;
    SweepArgs ax = sweep_args(c, U, false);
    ax.sel = sel;
    ax.sel_in = sel_in;
    ax.ft_out = ft;
    ax.epi.mode = EPI_STORE;
    ax.epi.out = c->D;
    ax.t_coef = t_coef;
    prof_start(c, 1);
    cudaError_t e = ext     ? by_order<E2XEF>(c->order, ax, low, c->stream)
                    : tma_x ? by_order<E2XTF>(c->order, mx, ax, low, c->stream)
                            : by_order<E2XF>(c->order, ax, low, c->stream);
    prof_stop(c, 1);
    CU_TRY(e);
    SweepArgs ay = sweep_args(c, U, true);
    ay.sel = sel ? sel + 8LL * c->ny * (c->nx + 1) : nullptr;
    ay.sel_in = sel_in ? sel_in + 8LL * c->ny * (c->nx + 1) : nullptr;
    ay.ft_out = ft ? ft + 4LL * c->ny * (c->nx + 1) : nullptr;
    ay.epi = epi;
    ay.epi.Dprev = c->D;
    ay.t_coef = t_coef;
    prof_start(c, 2);
    e = ext     ? by_order<E2YEF>(c->order, ay, low, c->stream)
        : tma_y ? by_order<E2YTF>(c->order, my, ay, low, c->stream)
                : by_order<E2YF>(c->order, ay, low, c->stream);
    prof_stop(c, 2);
    return cu(e);
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

ENOMR_API const char *enomr_strerror(int s)
{
    switch (s) {
    case ENOMR_OK: return "ok";
    case ENOMR_EINVAL: return "invalid argument";
    case ENOMR_ENOMEM: return "device allocation failed";
    case ENOMR_ECUDA: return "CUDA error";
    case ENOMR_ENONPHYS: return "non-physical state (rho<=0, p<=0, Roe c^2<=0 or NaN)";
    case ENOMR_ETIMEOUT: return "device wait timed out";
    default: return "unknown status";
    }
}

ENOMR_API int enomr_num_tested(int R)
{
    static const int T[7] = {4, 7, 10, 14, 18, 22, 26};
    return valid_order(R) ? T[(R - 5) / 2] : -1;
}

ENOMR_API void enomr_free(enomr_ctx *c)
{
    if (!c) return;
    cudaFree(c->ax);
    cudaFree(c->ay);
    cudaFree(c->smax);
    cudaFree(c->dt);
    cudaFree(c->status);
    cudaFree(c->U1);
    cudaFree(c->U2);
    cudaFree(c->D);
    cudaFree(c->ix);
    cudaFree(c->iy);
    cudaFree(c->axb);
    cudaFree(c->ayb);
    cudaFree(c->Ub1);
    cudaFree(c->Ub2);
    cudaFree(c->sides_d);
    cudaFree(c->t_dev);
    for (int i = 0; i < 2; ++i) {
        cudaFree(c->fsel[i]);
        cudaFree(c->fft[i]);
    }
    if (c->prof_ev) {
        for (int i = 0; i < 2 * c->prof_max; ++i) cudaEventDestroy(c->prof_ev[i]);
        free(c->prof_ev);
    }
    delete c;
}

ENOMR_API enomr_status enomr_init(enomr_ctx **out, int eq, int ndim, int64_t nx, int64_t ny,
                                  double dx, double dy, int order, double gamma, int bc,
                                  double adv_speed, void *stream)
{
    if (!out) return ENOMR_EINVAL;
    *out = nullptr;
    if (!valid_order(order)) return ENOMR_EINVAL;
    if (eq != ENOMR_ADVECTION && eq != ENOMR_EULER && eq != ENOMR_BURGERS) return ENOMR_EINVAL;
    if (eq == ENOMR_BURGERS && ndim != 1) return ENOMR_EINVAL;
    if (bc != ENOMR_PERIODIC && bc != ENOMR_TRANSMISSIVE) return ENOMR_EINVAL;
    if (ndim != 1 && ndim != 2) return ENOMR_EINVAL;
    if (eq == ENOMR_ADVECTION && ndim != 1) return ENOMR_EINVAL;
    if (ndim == 1) ny = 1;
    if (nx < 1 || ny < 1 || nx > (1LL << 40) || ny > (1LL << 40)) return ENOMR_EINVAL;
    if (!(dx > 0.0) || (ndim == 2 && !(dy > 0.0))) return ENOMR_EINVAL;
    if (eq == ENOMR_EULER && !(gamma > 1.0)) return ENOMR_EINVAL;
    if (eq == ENOMR_ADVECTION && !(adv_speed == adv_speed)) return ENOMR_EINVAL;
    const int g = (order + 1) / 2;
    if (bc == ENOMR_PERIODIC && (nx < 2 * g || (ndim == 2 && ny < 2 * g))) return ENOMR_EINVAL;
    // grid dimensions of the sweep kernels
    if (ndim == 2 && ny > 2LL * 65535) return ENOMR_EINVAL;

    enomr_ctx *c = new (std::nothrow) enomr_ctx();
    if (!c) return ENOMR_ENOMEM;
    c->eq = eq;
    c->ndim = ndim;
    c->order = order;
    c->bc = bc;
    c->nx = nx;
    c->ny = ny;
    c->dx = dx;
    c->dy = ndim == 2 ? dy : 1.0;
    c->gamma = gamma;
    c->adv = adv_speed;
    c->stream = (cudaStream_t)stream;
    const int C = eq != ENOMR_EULER ? 1 : (ndim == 2 ? 4 : 3);
    c->nstate = (long long)C * nx * ny;
    bool ok = cudaMalloc(&c->ax, sizeof(double) * 3 * ny) == cudaSuccess &&
              cudaMalloc(&c->ay, sizeof(double) * 3 * nx) == cudaSuccess &&
              cudaMalloc(&c->smax, sizeof(double)) == cudaSuccess &&
              cudaMalloc(&c->dt, sizeof(double)) == cudaSuccess &&
              cudaMalloc(&c->status, sizeof(int)) == cudaSuccess &&
              cudaMalloc(&c->U1, sizeof(double) * c->nstate) == cudaSuccess &&
              cudaMalloc(&c->U2, sizeof(double) * c->nstate) == cudaSuccess &&
              (ndim == 1 || cudaMalloc(&c->D, sizeof(double) * c->nstate) == cudaSuccess) &&
              cudaMalloc(&c->ix, sizeof(unsigned long long) * 3 * ny) == cudaSuccess &&
              cudaMalloc(&c->iy, sizeof(unsigned long long) * 3 * nx) == cudaSuccess &&
              cudaMalloc(&c->axb, sizeof(double) * 3 * ny) == cudaSuccess &&
              cudaMalloc(&c->ayb, sizeof(double) * 3 * nx) == cudaSuccess &&
              cudaMalloc(&c->Ub1, sizeof(double) * c->nstate) == cudaSuccess &&
              cudaMalloc(&c->Ub2, sizeof(double) * c->nstate) == cudaSuccess &&
              cudaMalloc(&c->sides_d, sizeof(SideDev) * 4) == cudaSuccess &&
              cudaMalloc(&c->t_dev, sizeof(double)) == cudaSuccess;
    if (ok && eq == ENOMR_EULER) {
        c->nsel = ndim == 2 ? 8 * ny * (nx + 1) + 8 * nx * (ny + 1) : 6 * (nx + 1);
        c->nft = ndim == 2 ? 4 * ny * (nx + 1) + 4 * nx * (ny + 1) : 3 * (nx + 1);
        for (int i = 0; i < 2 && ok; ++i)
            ok = cudaMalloc(&c->fsel[i], c->nsel) == cudaSuccess &&
                 cudaMalloc(&c->fft[i], sizeof(double) * c->nft) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        enomr_free(c);
        return ENOMR_ENOMEM;
    }
    {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            enomr_free(c);
            return ENOMR_ECUDA;
        }
        c->sms = sms;
    }
    if (cudaMemset(c->status, 0, sizeof(int)) != cudaSuccess ||
        cudaMemset(c->t_dev, 0, sizeof(double)) != cudaSuccess ||
        cudaMemset(c->dt, 0, sizeof(double)) != cudaSuccess) {
        enomr_free(c);
        return ENOMR_ECUDA;
    }
    *out = c;
    return ENOMR_OK;
}

ENOMR_API enomr_status enomr_set_stream(enomr_ctx *c, void *stream)
{
    if (!c) return ENOMR_EINVAL;
    c->stream = (cudaStream_t)stream;
    return ENOMR_OK;
}

ENOMR_API enomr_status enomr_rhs(enomr_ctx *c, const double *U, double *dUdt)
{
    if (!c || !U || !dUdt || (const double *)dUdt == U) return ENOMR_EINVAL;
    enomr_status st = compute_alpha(c, U, false);
    if (st) return st;
    Epilogue e;
    memset(&e, 0, sizeof(e));
    e.mode = EPI_STORE;
    e.out = dUdt;
    return rhs_with_epilogue(c, U, e, nullptr);
}

static const double RK_C0[3] = {0.0, 0.75, 1.0 / 3.0};
static const double RK_C1[3] = {1.0, 0.25, 2.0 / 3.0};

static enomr_status stage_impl(enomr_ctx *c, int s, const double *Un, const double *Us,
                               double *Uout, bool alpha_current = false, uint8_t *sel = nullptr,
                               double *ft = nullptr)
{
    enomr_status st = alpha_current ? ENOMR_OK : compute_alpha(c, Us, false);
    if (st) return st;
    Epilogue e;
    memset(&e, 0, sizeof(e));
    e.mode = EPI_STAGE;
    e.c0 = RK_C0[s - 1];
    e.c1 = RK_C1[s - 1];
    e.dt_dev = c->dt;
    e.Un = Un;
    e.out = Uout;
    static const double RK_T[3] = {0.0, 1.0, 0.5};  // stage times t + RK_T dt
    return rhs_with_epilogue(c, Us, e, sel, ft, RK_T[s - 1]);
}

ENOMR_API enomr_status enomr_stage(enomr_ctx *c, int s, const double *Un, const double *Us,
                                   double *Uout, double dt)
{
    if (!c || s < 1 || s > 3 || !Un || !Us || !Uout || !(dt > 0.0)) return ENOMR_EINVAL;
    if (s == 1 && Us != Un) return ENOMR_EINVAL;
    if ((const double *)Uout == Us && s != 1) return ENOMR_EINVAL;
    if (s == 1 && (const double *)Uout == Un) return ENOMR_EINVAL;
    CU_TRY(launch_set_dt(c->smax, 0.0, dt, c->dt, c->stream));
    return stage_impl(c, s, Un, Us, Uout);
}

static enomr_status set_step_dt(enomr_ctx *c, const double *U, double dt, double cfl)
{
    if (dt > 0.0) return cu(launch_set_dt(c->smax, 0.0, dt, c->dt, c->stream));
    if (!(cfl > 0.0)) return ENOMR_EINVAL;
    if (c->eq == ENOMR_ADVECTION) {
        if (!(c->adv != 0.0)) return ENOMR_EINVAL;
        return cu(launch_set_dt(c->smax, 0.0, cfl * c->dx / fabs(c->adv), c->dt, c->stream));
    }
    enomr_status st = compute_alpha(c, U, true);
    if (st) return st;
    return cu(launch_set_dt(c->smax, cfl, 0.0, c->dt, c->stream));
}

ENOMR_API enomr_status enomr_step(enomr_ctx *c, double *U, double dt, double cfl, double *dt_used)
{
    if (!c || !U) return ENOMR_EINVAL;
    enomr_status st = set_step_dt(c, U, dt, cfl);
    if (st) return st;
    // with a CFL step the alpha of U^n was just computed with the wave-speed max
    const bool alpha_done = !(dt > 0.0) && c->eq != ENOMR_ADVECTION;
    if ((st = stage_impl(c, 1, U, U, c->U1, alpha_done))) return st;
    if ((st = stage_impl(c, 2, U, c->U1, c->U2))) return st;
    if ((st = stage_impl(c, 3, U, c->U2, U))) return st;
    if (extended(c)) {  // the time only matters to boundary sides
        k_advance_time<<<1, 1, 0, c->stream>>>(c->t_dev, c->dt, 1.0);
        CU_TRY(cudaGetLastError());
    }
    if (dt_used) {
        CU_TRY(cudaMemcpyAsync(dt_used, c->dt, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CU_TRY(cudaStreamSynchronize(c->stream));
    }
    return ENOMR_OK;
}

static enomr_status axpy(enomr_ctx *c, double a, const double *x, double *y, int acc);

// Coefficients alpha_{m,0..m-1} of the linear SSP-RK(m, m-1) family:
// alpha_{2,*} = (0, 1); alpha_{m,k} = (2/k) alpha_{m-1,k-1} for 1 <= k <= m-2,
// alpha_{m,m-1} = (2/m) alpha_{m-1,m-2}, alpha_{m,0} = 1 - sum_{k>=1} alpha_{m,k}.
static void lssp_alphas(int m, double *out)
{
    double a[40] = {0.0, 1.0};
    for (int mm = 3; mm <= m; ++mm) {
        double b[40];
        double sum = 0.0;
        for (int k = 1; k <= mm - 2; ++k) b[k] = (2.0 / k) * a[k - 1];
        b[mm - 1] = (2.0 / mm) * a[mm - 2];
        for (int k = 1; k <= mm - 1; ++k) sum += b[k];
        b[0] = 1.0 - sum;
        for (int k = 0; k < mm; ++k) a[k] = b[k];
    }
    for (int k = 0; k < m; ++k) out[k] = a[k];
}

ENOMR_API enomr_status enomr_step_lssp(enomr_ctx *c, double *U, double dt, int m)
{
    if (!c || !U || !(dt > 0.0) || m < 2 || m > 32) return ENOMR_EINVAL;
    double al[40];
    lssp_alphas(m, al);
    enomr_status st;
    // every stage advances by dt/2: u^(s) = u^(s-1) + dt/2 L(u^(s-1))
    CU_TRY(launch_set_dt(c->smax, 0.0, 0.5 * dt, c->dt, c->stream));
    double *acc = c->Ub1;                      // sum_{k<=m-2} alpha_k u^(k)
    if ((st = axpy(c, al[0], U, acc, 0))) return st;
    const double *cur = U;
    double *bufs[2] = {c->U1, c->U2};
    for (int s = 1; s <= m - 1; ++s) {
        double *next = bufs[s & 1];
        st = compute_alpha(c, cur, false);
        if (st) return st;
        Epilogue e;
        memset(&e, 0, sizeof(e));
        e.mode = EPI_STAGE;
        e.c0 = 0.0;
        e.c1 = 1.0;
        e.dt_dev = c->dt;
        e.Un = cur;
        e.out = next;
        // c->dt holds dt/2 here: stage s starts at t + (s - 1) dt/2
        if ((st = rhs_with_epilogue(c, cur, e, nullptr, nullptr, (double)(s - 1)))) return st;
        if (s <= m - 2 && al[s] != 0.0)
            if ((st = axpy(c, al[s], next, acc, 1))) return st;
        cur = next;
    }
    // u^{n+1} = acc + alpha_{m-1} (u^(m-1) + dt/2 L(u^(m-1)))
    st = compute_alpha(c, cur, false);
    if (st) return st;
    Epilogue e;
    memset(&e, 0, sizeof(e));
    e.mode = EPI_STAGE;
    e.c0 = 1.0;
    e.c1 = al[m - 1];
    e.dt_dev = c->dt;
    e.Un = acc;
    e.out = U;
    if ((st = rhs_with_epilogue(c, cur, e, nullptr, nullptr, (double)(m - 1)))) return st;
    if (extended(c)) {  // t += dt (2 x the stored dt/2, exact)
        k_advance_time<<<1, 1, 0, c->stream>>>(c->t_dev, c->dt, 2.0);
        CU_TRY(cudaGetLastError());
    }
    return ENOMR_OK;
}

ENOMR_API enomr_status enomr_cfl_dt(enomr_ctx *c, const double *U, double cfl, double *dt_host)
{
    if (!c || !U || !dt_host || !(cfl > 0.0)) return ENOMR_EINVAL;
    enomr_status st = set_step_dt(c, U, 0.0, cfl);
    if (st) return st;
    CU_TRY(cudaMemcpyAsync(dt_host, c->dt, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CU_TRY(cudaStreamSynchronize(c->stream));
    return ENOMR_OK;
}

ENOMR_API enomr_status enomr_stage_frozen(enomr_ctx *c, int s, const double *Un,
                                          const double *Us, double *Uout, double dt,
                                          const double *Uref)
{
    if (!c || s < 1 || s > 3 || !Un || !Us || !Uout || !Uref || !(dt > 0.0)) return ENOMR_EINVAL;
    if (c->eq != ENOMR_EULER || c->ndim != 2 || extended(c)) return ENOMR_EINVAL;
    if (s == 1 && Us != Un) return ENOMR_EINVAL;
    if ((const double *)Uout == Us || (const double *)Uout == Uref) return ENOMR_EINVAL;
    if (s == 1 && (const double *)Uout == Un) return ENOMR_EINVAL;
    CU_TRY(launch_set_dt(c->smax, 0.0, dt, c->dt, c->stream));
    // the choices of Uref: its per-line alpha, the selections of its sweeps
    // (into fsel[0]; the right-hand side goes to the stage scratch and is
    // discarded) and the cells attaining each alpha
    enomr_status st = compute_alpha(c, Uref, false);
    if (st) return st;
    Epilogue er;
    memset(&er, 0, sizeof(er));
    er.mode = EPI_STORE;
    er.out = c->U2;
    if ((st = rhs_with_epilogue(c, Uref, er, c->fsel[0]))) return st;
    CU_TRY(cudaMemsetAsync(c->ix, 0xff, sizeof(unsigned long long) * 3 * c->ny, c->stream));
    CU_TRY(cudaMemsetAsync(c->iy, 0xff, sizeof(unsigned long long) * 3 * c->nx, c->stream));
    AlphaArgs aa;
    memset(&aa, 0, sizeof(aa));
    aa.U = Uref;
    aa.nx = c->nx;
    aa.ny = c->ny;
    aa.gm1 = c->gamma - 1.0;
    aa.gamma = c->gamma;
    aa.ax = c->ax;
    aa.ay = c->ay;
    aa.status = c->status;
    dim3 grid((unsigned)((c->nx + 31) / 32), (unsigned)((c->ny + 31) / 32));
    k_alpha_argmax<4><<<grid, 256, 0, c->stream>>>(aa, c->ix, c->iy);
    CU_TRY(cudaGetLastError());
    // alpha of Us at those cells, then the stage with the frozen selections
    const long long nl = c->ny + c->nx;
    k_alpha_at<4><<<(unsigned)((3 * nl + 255) / 256), 256, 0, c->stream>>>(
        Us, c->nx, c->ny, c->gamma - 1.0, c->gamma, c->ix, c->iy, c->ax, c->ay, c->status);
    CU_TRY(cudaGetLastError());
    Epilogue e;
    memset(&e, 0, sizeof(e));
    e.mode = EPI_STAGE;
    e.c0 = RK_C0[s - 1];
    e.c1 = RK_C1[s - 1];
    e.dt_dev = c->dt;
    e.Un = Un;
    e.out = Uout;
    return rhs_with_epilogue(c, Us, e, nullptr, nullptr, 0.0, c->fsel[0]);
}

ENOMR_API enomr_status enomr_debug_selection(enomr_ctx *c, const double *U, uint8_t *sel)
{
    if (!c || !U || !sel) return ENOMR_EINVAL;
    enomr_status st = compute_alpha(c, U, false);
    if (st) return st;
    // the RHS is written to the stage buffer and discarded
    Epilogue e;
    memset(&e, 0, sizeof(e));
    e.mode = EPI_STORE;
    e.out = c->U2;
    return rhs_with_epilogue(c, U, e, sel);
}

ENOMR_API enomr_status enomr_get_status(enomr_ctx *c)
{
    if (!c) return ENOMR_EINVAL;
    int h = 0;
    CU_TRY(cudaMemcpyAsync(&h, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CU_TRY(cudaStreamSynchronize(c->stream));
    CU_TRY(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
    CU_TRY(cudaStreamSynchronize(c->stream));
    if (h & ST_TMA_TIMEOUT) return ENOMR_ETIMEOUT;
    return h ? ENOMR_ENONPHYS : ENOMR_OK;
}

ENOMR_API enomr_status enomr_set_staging(enomr_ctx *c, int mode)
{
    if (!c || mode < ENOMR_STAGING_AUTO || mode > ENOMR_STAGING_TMA) return ENOMR_EINVAL;
    c->staging = mode;
    return ENOMR_OK;
}

ENOMR_API enomr_status enomr_set_occupancy(enomr_ctx *c, int mode)
{
    if (!c || mode < ENOMR_OCCUPANCY_AUTO || mode > ENOMR_OCCUPANCY_LOW) return ENOMR_EINVAL;
    c->occupancy = mode;
    return ENOMR_OK;
}

// Ubar += scale * J(U)^T Lbar, scale = factor * (*factor_dev if given).
static enomr_status rhs_vjp_impl(enomr_ctx *c, const double *U, const double *Lbar, double *Ubar,
                                 double scale, const uint8_t *sel_in = nullptr,
                                 const double *ft_in = nullptr,
                                 const double *scale_dev = nullptr)
{
    if (c->eq == ENOMR_ADVECTION) {
        AdvArgs a;
        memset(&a, 0, sizeof(a));
        a.U = U;
        a.n = c->nx;
        a.bc = c->bc;
        a.a = c->adv;
        a.inv_h = 1.0 / c->dx;
        return cu(by_order<AdvVjpF>(c->order, a, Lbar, Ubar, scale, scale_dev, c->stream));
    }
    const int C = c->ndim == 2 ? 4 : 3;
    enomr_status st = compute_alpha(c, U, false);
    if (st) return st;
    CU_TRY(cudaMemsetAsync(c->ix, 0xff, sizeof(unsigned long long) * 3 * c->ny, c->stream));
    CU_TRY(cudaMemsetAsync(c->iy, 0xff, sizeof(unsigned long long) * 3 * c->nx, c->stream));
    CU_TRY(cudaMemsetAsync(c->axb, 0, sizeof(double) * 3 * c->ny, c->stream));
    CU_TRY(cudaMemsetAsync(c->ayb, 0, sizeof(double) * 3 * c->nx, c->stream));
    AlphaArgs aa;
    memset(&aa, 0, sizeof(aa));
    aa.U = U;
    aa.nx = c->nx;
    aa.ny = c->ny;
    aa.gm1 = c->gamma - 1.0;
    aa.gamma = c->gamma;
    aa.ax = c->ax;
    aa.ay = c->ay;
    aa.status = c->status;
    dim3 grid((unsigned)((c->nx + 31) / 32), (unsigned)((c->ny + 31) / 32));
    if (C == 4)
        k_alpha_argmax<4><<<grid, 256, 0, c->stream>>>(aa, c->ix, c->iy);
    else
        k_alpha_argmax<3><<<grid, 256, 0, c->stream>>>(aa, c->ix, c->iy);
    CU_TRY(cudaGetLastError());
    VjpArgs v;
    v.U = U;
    v.Lbar = Lbar;
    v.Ubar = Ubar;
    v.nx = c->nx;
    v.ny = c->ny;
    v.bc = c->bc;
    v.gm1 = c->gamma - 1.0;
    v.inv_gm1 = 1.0 / (c->gamma - 1.0);
    v.gamma = c->gamma;
    v.scale = scale;
    v.scale_dev = scale_dev;
    v.status = c->status;
    v.inv_h = 1.0 / c->dx;
    v.alpha = c->ax;
    v.alpha_bar = c->axb;
    v.sel_in = sel_in;
    v.ft_in = ft_in;
    CU_TRY(by_order<VjpF>(c->order, v, C, 0, c->stream));
    if (C == 4) {
        v.inv_h = 1.0 / c->dy;
        v.alpha = c->ay;
        v.alpha_bar = c->ayb;
        v.sel_in = sel_in ? sel_in + 8LL * c->ny * (c->nx + 1) : nullptr;
        v.ft_in = ft_in ? ft_in + 4LL * c->ny * (c->nx + 1) : nullptr;
        CU_TRY(by_order<VjpF>(c->order, v, C, 1, c->stream));
    }
    const long long nl = (C == 4) ? c->ny + c->nx : c->ny;
    const unsigned blocks = (unsigned)((3 * nl + 255) / 256);
    if (C == 4)
        k_alpha_vjp<4><<<blocks, 256, 0, c->stream>>>(U, c->nx, c->ny, c->gamma - 1.0, c->gamma,
                                                      c->ix, c->iy, c->axb, c->ayb, Ubar);
    else
        k_alpha_vjp<3><<<blocks, 256, 0, c->stream>>>(U, c->nx, c->ny, c->gamma - 1.0, c->gamma,
                                                      c->ix, c->iy, c->axb, c->ayb, Ubar);
    return cu(cudaGetLastError());
}

static enomr_status axpy(enomr_ctx *c, double a, const double *x, double *y, int acc)
{
    k_axpy<<<1216, 256, 0, c->stream>>>(c->nstate, a, x, y, acc);
    return cu(cudaGetLastError());
}

ENOMR_API enomr_status enomr_rhs_vjp(enomr_ctx *c, const double *U, const double *Lbar,
                                     double *Ubar, double scale, int accumulate)
{
    if (!c || !U || !Lbar || !Ubar || (const double *)Ubar == U || (const double *)Ubar == Lbar)
        return ENOMR_EINVAL;
    if (c->eq == ENOMR_BURGERS || extended(c)) return ENOMR_EINVAL;
    if (!accumulate) CU_TRY(cudaMemsetAsync(Ubar, 0, sizeof(double) * c->nstate, c->stream));
    return rhs_vjp_impl(c, U, Lbar, Ubar, scale);
}

// Transpose of one SSP-RK3 step from U^n whose dt is already in c->dt.
static enomr_status step_vjp_impl(enomr_ctx *c, const double *Un, const double *Ubar_np1,
                                  double *Ubar_n);

ENOMR_API enomr_status enomr_step_vjp(enomr_ctx *c, const double *Un, double dt,
                                      const double *Ubar_np1, double *Ubar_n)
{
    if (!c || !Un || !Ubar_np1 || !Ubar_n || !(dt > 0.0)) return ENOMR_EINVAL;
    if (c->eq == ENOMR_BURGERS || extended(c)) return ENOMR_EINVAL;
    if ((const double *)Ubar_n == Ubar_np1 || (const double *)Ubar_n == Un) return ENOMR_EINVAL;
    CU_TRY(launch_set_dt(c->smax, 0.0, dt, c->dt, c->stream));
    return step_vjp_impl(c, Un, Ubar_np1, Ubar_n);
}

ENOMR_API enomr_status enomr_step_vjp_cfl(enomr_ctx *c, const double *Un, double cfl,
                                          const double *Ubar_np1, double *Ubar_n)
{
    if (!c || !Un || !Ubar_np1 || !Ubar_n || !(cfl > 0.0)) return ENOMR_EINVAL;
    if (c->eq == ENOMR_BURGERS || extended(c)) return ENOMR_EINVAL;
    if ((const double *)Ubar_n == Ubar_np1 || (const double *)Ubar_n == Un) return ENOMR_EINVAL;
    // the forward step's dt, recomputed from U^n by the same kernels: the
    // same bits, without a host round trip
    enomr_status st = set_step_dt(c, Un, 0.0, cfl);
    if (st) return st;
    return step_vjp_impl(c, Un, Ubar_np1, Ubar_n);
}

static enomr_status step_vjp_impl(enomr_ctx *c, const double *Un, const double *Ubar_np1,
                                  double *Ubar_n)
{
    enomr_status st;
    // recompute the stages from the step's checkpoint U^n
    // the recomputed stages also keep their selections and per-field values,
    // which the transposes at U^n and U^(1) then reuse
    const bool keep = c->eq == ENOMR_EULER;
    if ((st = stage_impl(c, 1, Un, Un, c->U1, false, keep ? c->fsel[0] : nullptr,
                         keep ? c->fft[0] : nullptr)))
        return st;
    if ((st = stage_impl(c, 2, Un, c->U1, c->U2, false, keep ? c->fsel[1] : nullptr,
                         keep ? c->fft[1] : nullptr)))
        return st;
    // U^{n+1} = 1/3 U^n + 2/3 (U2 + dt L(U2))
    if ((st = axpy(c, 1.0 / 3.0, Ubar_np1, Ubar_n, 0))) return st;
    if ((st = axpy(c, 2.0 / 3.0, Ubar_np1, c->Ub2, 0))) return st;
    // the step's dt is on the device (c->dt): the cotangent scales are
    // formed there, (2/3) dt, (1/4) dt and dt
    if ((st = rhs_vjp_impl(c, c->U2, Ubar_np1, c->Ub2, 2.0 / 3.0, nullptr, nullptr, c->dt)))
        return st;
    // U2 = 3/4 U^n + 1/4 (U1 + dt L(U1))
    if ((st = axpy(c, 0.75, c->Ub2, Ubar_n, 1))) return st;
    if ((st = axpy(c, 0.25, c->Ub2, c->Ub1, 0))) return st;
    if ((st = rhs_vjp_impl(c, c->U1, c->Ub2, c->Ub1, 0.25, keep ? c->fsel[1] : nullptr,
                           keep ? c->fft[1] : nullptr, c->dt)))
        return st;
    // U1 = U^n + dt L(U^n)
    if ((st = axpy(c, 1.0, c->Ub1, Ubar_n, 1))) return st;
    return rhs_vjp_impl(c, Un, c->Ub1, Ubar_n, 1.0, keep ? c->fsel[0] : nullptr,
                        keep ? c->fft[0] : nullptr, c->dt);
}

ENOMR_API enomr_status enomr_debug_alpha(enomr_ctx *c, double *alpha_x, double *alpha_y,
                                         double *alpha_bar_x, double *alpha_bar_y,
                                         uint64_t *argmax_x, uint64_t *argmax_y)
{
    if (!c) return ENOMR_EINVAL;
    const size_t bx = sizeof(double) * 3 * c->ny, by = sizeof(double) * 3 * c->nx;
    if (argmax_x) CU_TRY(cudaMemcpyAsync(argmax_x, c->ix, bx, cudaMemcpyDeviceToDevice, c->stream));
    if (argmax_y && c->ndim == 2)
        CU_TRY(cudaMemcpyAsync(argmax_y, c->iy, by, cudaMemcpyDeviceToDevice, c->stream));
    if (alpha_x) CU_TRY(cudaMemcpyAsync(alpha_x, c->ax, bx, cudaMemcpyDeviceToDevice, c->stream));
    if (alpha_y && c->ndim == 2)
        CU_TRY(cudaMemcpyAsync(alpha_y, c->ay, by, cudaMemcpyDeviceToDevice, c->stream));
    if (alpha_bar_x)
        CU_TRY(cudaMemcpyAsync(alpha_bar_x, c->axb, bx, cudaMemcpyDeviceToDevice, c->stream));
    if (alpha_bar_y && c->ndim == 2)
        CU_TRY(cudaMemcpyAsync(alpha_bar_y, c->ayb, by, cudaMemcpyDeviceToDevice, c->stream));
    return ENOMR_OK;
}

ENOMR_API enomr_status enomr_set_side(enomr_ctx *c, int side, const enomr_side *d)
{
    if (!c || !d || c->eq != ENOMR_EULER || c->ndim != 2 || c->bc != ENOMR_TRANSMISSIVE)
        return ENOMR_EINVAL;
    if (side < 0 || side > 3) return ENOMR_EINVAL;
    const int g = (c->order + 1) / 2;
    const long long across = side < 2 ? c->nx : c->ny;
    const int kinds[2] = {d->kind_lo, d->kind_hi};
    for (int i = 0; i < 2; ++i) {
        if (kinds[i] < ENOMR_SIDE_TRANSMISSIVE || kinds[i] > ENOMR_SIDE_INFLOW) return ENOMR_EINVAL;
        if (kinds[i] == ENOMR_SIDE_REFLECTIVE && across < g) return ENOMR_EINVAL;
        const double *st = i ? d->state_hi : d->state_lo;
        if (kinds[i] == ENOMR_SIDE_INFLOW) {
            const double q2 = st[1] * st[1] + st[2] * st[2];
            if (!(st[0] > 0.0) || !((st[3] - 0.5 * q2 / st[0]) > 0.0)) return ENOMR_EINVAL;
        }
    }
    if (d->split0 != d->split0 || d->split_rate != d->split_rate) return ENOMR_EINVAL;
    SideDev h[4];
    // the sides are read by sweeps already queued on the context's stream,
    // which may be a non-blocking one: let them finish before the copy
    CU_TRY(cudaStreamSynchronize(c->stream));
    if (c->custom_sides) {
        CU_TRY(cudaMemcpy(h, c->sides_d, sizeof(h), cudaMemcpyDeviceToHost));
    } else {
        for (int i = 0; i < 4; ++i) {
            memset(&h[i], 0, sizeof(SideDev));
            h[i].kind_lo = h[i].kind_hi = SIDE_TRANSMISSIVE;
            h[i].split0 = __builtin_inf();
        }
    }
    h[side].kind_lo = d->kind_lo;
    h[side].kind_hi = d->kind_hi;
    h[side].split0 = d->split0;
    h[side].rate = d->split_rate;
    for (int q = 0; q < 4; ++q) {
        h[side].st_lo[q] = d->state_lo[q];
        h[side].st_hi[q] = d->state_hi[q];
    }
    CU_TRY(cudaMemcpy(c->sides_d, h, sizeof(h), cudaMemcpyHostToDevice));
    c->custom_sides = true;
    return ENOMR_OK;
}

ENOMR_API enomr_status enomr_set_body_force(enomr_ctx *c, double gx, double gy)
{
    if (!c || c->eq != ENOMR_EULER || c->ndim != 2) return ENOMR_EINVAL;
    if (gx != gx || gy != gy) return ENOMR_EINVAL;
    if ((gx != 0.0 || gy != 0.0) && !c->custom_sides) {
        // the EXT sweeps read the sides: make them the default ones (after
        // the work already queued on the context's stream)
        CU_TRY(cudaStreamSynchronize(c->stream));
        SideDev h[4];
        for (int i = 0; i < 4; ++i) {
            memset(&h[i], 0, sizeof(SideDev));
            h[i].kind_lo = h[i].kind_hi = SIDE_TRANSMISSIVE;
            h[i].split0 = __builtin_inf();
        }
        CU_TRY(cudaMemcpy(c->sides_d, h, sizeof(h), cudaMemcpyHostToDevice));
    }
    c->gx = gx;
    c->gy = gy;
    return ENOMR_OK;
}

ENOMR_API enomr_status enomr_set_time(enomr_ctx *c, double t)
{
    if (!c || t != t) return ENOMR_EINVAL;
    CU_TRY(cudaMemcpyAsync(c->t_dev, &t, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CU_TRY(cudaStreamSynchronize(c->stream));
    return ENOMR_OK;
}

ENOMR_API enomr_status enomr_get_time(enomr_ctx *c, double *t)
{
    if (!c || !t) return ENOMR_EINVAL;
    CU_TRY(cudaMemcpyAsync(t, c->t_dev, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CU_TRY(cudaStreamSynchronize(c->stream));
    return ENOMR_OK;
}

ENOMR_API enomr_status enomr_profile_begin(enomr_ctx *c, int kernel, int max_launches)
{
    if (!c || kernel < 0 || kernel > 3 || max_launches < 0 || max_launches > 100000)
        return ENOMR_EINVAL;
    if (c->prof_ev) {
        for (int i = 0; i < 2 * c->prof_max; ++i) cudaEventDestroy(c->prof_ev[i]);
        free(c->prof_ev);
        c->prof_ev = nullptr;
    }
    c->prof_kernel = 0;
    c->prof_max = 0;
    c->prof_n = 0;
    if (kernel == 0 || max_launches == 0) return ENOMR_OK;
    c->prof_ev = (cudaEvent_t *)calloc(2 * (size_t)max_launches, sizeof(cudaEvent_t));
    if (!c->prof_ev) return ENOMR_ENOMEM;
    for (int i = 0; i < 2 * max_launches; ++i)
        if (cudaEventCreate(&c->prof_ev[i]) != cudaSuccess) {
            for (int j = 0; j < i; ++j) cudaEventDestroy(c->prof_ev[j]);
            free(c->prof_ev);
            c->prof_ev = nullptr;
            return ENOMR_ECUDA;
        }
    c->prof_max = max_launches;
    c->prof_kernel = kernel;
    return ENOMR_OK;
}

ENOMR_API enomr_status enomr_profile_end(enomr_ctx *c, int *n_launches, double *total_ms)
{
    if (!c || !n_launches || !total_ms) return ENOMR_EINVAL;
    *n_launches = 0;
    *total_ms = 0.0;
    if (!c->prof_ev) return ENOMR_OK;
    CU_TRY(cudaStreamSynchronize(c->stream));
    double tot = 0.0;
    for (int i = 0; i < c->prof_n; ++i) {
        float ms = 0.0f;
        CU_TRY(cudaEventElapsedTime(&ms, c->prof_ev[2 * i], c->prof_ev[2 * i + 1]));
        tot += ms;
    }
    *n_launches = c->prof_n;
    *total_ms = tot;
    c->prof_kernel = 0;
    return ENOMR_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// FP64 FMA throughput probe: eight independent fma chains per thread.
// ---------------------------------------------------------------------------
namespace enomr {
__global__ void __launch_bounds__(256) k_fp64_fma(double *sink, long long iters, double seed)
{
    double a[8];
    const double m = 0.999999999999, q = 1e-12;
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = seed + 1e-3 * (threadIdx.x + 37 * i);
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = fma(a[i], m, q);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += a[i];
    if (s == -1.0) sink[blockIdx.x] = s;  // never true; keeps the chains live
}
}  // namespace enomr

extern "C" ENOMR_API enomr_status enomr_probe_fp64_fma(void *stream, int64_t iters,
                                                       double *sink, double *seconds,
                                                       double *flops)
{
    if (iters < 1 || !sink || !seconds || !flops) return ENOMR_EINVAL;
    int dev = 0, sms = 0;
    CU_TRY(cudaGetDevice(&dev));
    CU_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = sms * 8, threads = 256;
    cudaEvent_t e0, e1;
    CU_TRY(cudaEventCreate(&e0));
    CU_TRY(cudaEventCreate(&e1));
    enomr::k_fp64_fma<<<blocks, threads, 0, s>>>(sink, iters, 1.0);  // warm-up
    cudaEventRecord(e0, s);
    enomr::k_fp64_fma<<<blocks, threads, 0, s>>>(sink, iters, 1.0);
    cudaEventRecord(e1, s);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CU_TRY(err);
    *seconds = ms * 1e-3;
    *flops = 2.0 * 8.0 * (double)iters * blocks * threads;
    return ENOMR_OK;
}
