// enomr_batch.cu -- many independent 1D Euler problems of uneven size, one
// persistent launch per SSP-RK3 stage (C ABI in include/enomr.h).
//
// Packing: problem p's state is a dense [3][n_p] block starting at base[p]
// (in doubles) of one packed array; blocks follow each other.  Work unit: a
// tile of TP interfaces (TP-1 cells) of one problem; a table of all tiles of
// all problems is built once at set-up for each tile size, and the
// persistent stage kernel strides over it.  Per problem: alpha_k of U^n from
// a reduction over the problem's tiles, its CFL step, and the alpha of
// U^(1), U^(2) accumulated by the stage epilogues.  The arithmetic per
// interface, per cell and per problem is the one of enomr_step on a single
// problem, so each problem's result is bitwise the same.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/enomr.h"
#include "enomr_common.cuh"
#include "enomr_internal.h"

using namespace enomr;

namespace {
constexpr int kTileSizes[3] = {32, 64, 128};
}

struct enomr_batch {
    int order, bc;
    long long nprob, total;
    double gamma;
    cudaStream_t stream;
    long long *base, *n;
    double *inv_dx;
    BatchTile *tiles[3];
    long long ntiles[3];
    int tp_index, grid, per_item;
    double *alpha;  // [3][nprob][3]: alpha of U^n, U^(1), U^(2)
    double *dt;     // [nprob]
    int *status;
    double *U1, *U2;
};

namespace enomr {

// alpha of U^n per problem, reduced over its tiles of cells_per_tile cells
__global__ void __launch_bounds__(128) k_batch_alpha(BatchAlphaArgs A)
{
    __shared__ unsigned long long red[4][3];
    for (long long t = blockIdx.x; t < A.ntiles; t += gridDim.x) {
        const BatchTile tl = A.tiles[t];
        const long long n = A.n[tl.prob];
        const double *U = A.U + A.base[tl.prob];
        unsigned long long w[3] = {0, 0, 0};
        for (int j = threadIdx.x; j < A.cells_per_tile; j += blockDim.x) {
            const long long i = (long long)tl.x0 + j;
            if (i < n) {
                double s3[3];
                wave_speeds3(U[i], U[n + i], U[2 * n + i], A.gm1, A.gamma, s3, A.status);
                for (int k = 0; k < 3; ++k) {
                    const unsigned long long b = __double_as_longlong(s3[k]);
                    w[k] = w[k] > b ? w[k] : b;
                }
            }
        }
        for (int k = 0; k < 3; ++k) {
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long x = __shfl_xor_sync(0xffffffffu, w[k], o);
                w[k] = w[k] > x ? w[k] : x;
            }
        }
        __syncthreads();
        if ((threadIdx.x & 31) == 0)
            for (int k = 0; k < 3; ++k) red[threadIdx.x >> 5][k] = w[k];
        __syncthreads();
        if (threadIdx.x < 3) {
            unsigned long long m = 0;
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = m > red[i][threadIdx.x] ? m : red[i][threadIdx.x];
            atomicMax((unsigned long long *)(A.alpha + 3 * tl.prob + threadIdx.x), m);
        }
    }
}

// CFL step per problem: dt = cfl / (max(|u|+c) / dx), with
// max(|u|+c) = max(max|u-c|, max|u+c|) taken from alpha.
__global__ void k_batch_dt(const double *alpha, const double *inv_dx, double cfl, long long nprob,
                           double *dt)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < nprob) {
        const double a0 = alpha[3 * p], a2 = alpha[3 * p + 2];
        const double smax = __dmul_rn(a0 > a2 ? a0 : a2, inv_dx[p]);
        dt[p] = cfl / smax;
    }
}

cudaError_t launch_batch_alpha(const BatchAlphaArgs &a, cudaStream_t s)
{
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long grid = a.ntiles < (long long)sms * 16 ? a.ntiles : (long long)sms * 16;
    if (grid < 1) grid = 1;
    k_batch_alpha<<<(unsigned)grid, 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_batch_dt(const double *alpha, const double *inv_dx, double cfl, long long nprob,
                            double *dt, cudaStream_t s)
{
    k_batch_dt<<<(unsigned)((nprob + 255) / 256), 256, 0, s>>>(alpha, inv_dx, cfl, nprob, dt);
    return cudaGetLastError();
}

}  // namespace enomr

template <template <int> class F, typename... Args>
static cudaError_t by_order_b(int R, Args &&...args)
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

template <int R> struct BatchStageF {
    static cudaError_t run(const BatchArgs &a, int tp, int grid, cudaStream_t s)
    {
        return launch_batch_stage<R>(a, tp, grid, s);
    }
};

static enomr_status bcu(cudaError_t e) { return e == cudaSuccess ? ENOMR_OK : ENOMR_ECUDA; }
#define B_TRY(expr)                           \
    do {                                      \
        enomr_status st_ = bcu(expr);         \
        if (st_ != ENOMR_OK) return st_;      \
    } while (0)

static enomr_status batch_alpha_dt(enomr_batch *b, const double *U, double cfl, bool want_dt)
{
    B_TRY(cudaMemsetAsync(b->alpha, 0, sizeof(double) * 9 * b->nprob, b->stream));
    BatchAlphaArgs a;
    a.U = U;
    a.base = b->base;
    a.n = b->n;
    a.inv_dx = b->inv_dx;
    a.tiles = b->tiles[b->tp_index];
    a.ntiles = b->ntiles[b->tp_index];
    a.cells_per_tile = kTileSizes[b->tp_index] - 1;
    a.gm1 = b->gamma - 1.0;
    a.gamma = b->gamma;
    a.cfl = cfl;
    a.alpha = b->alpha;
    a.status = b->status;
    B_TRY(launch_batch_alpha(a, b->stream));
    if (want_dt) B_TRY(launch_batch_dt(b->alpha, b->inv_dx, cfl, b->nprob, b->dt, b->stream));
    return ENOMR_OK;
}

static const double B_C0[3] = {0.0, 0.75, 1.0 / 3.0};
static const double B_C1[3] = {1.0, 0.25, 2.0 / 3.0};

static enomr_status batch_stage(enomr_batch *b, int s, const double *Un, const double *Us,
                                double *out, int tp_index, int grid, int per_item)
{
    BatchArgs a;
    a.Us = Us;
    a.Un = Un;
    a.out = out;
    a.base = b->base;
    a.n = b->n;
    a.inv_dx = b->inv_dx;
    a.alpha = b->alpha + 3 * b->nprob * (s - 1);
    a.alpha_next = s < 3 ? b->alpha + 3 * b->nprob * s : nullptr;
    a.dt = b->dt;
    a.tiles = b->tiles[tp_index];
    a.ntiles = b->ntiles[tp_index];
    a.tiles_per_item = per_item;
    a.bc = b->bc;
    a.gm1 = b->gamma - 1.0;
    a.inv_gm1 = 1.0 / (b->gamma - 1.0);
    a.gamma = b->gamma;
    a.c0 = B_C0[s - 1];
    a.c1 = B_C1[s - 1];
    a.status = b->status;
    return bcu(by_order_b<BatchStageF>(b->order, a, kTileSizes[tp_index], grid, b->stream));
}

extern "C" {

ENOMR_API void enomr_batch_free(enomr_batch *b)
{
    if (!b) return;
    cudaFree(b->base);
    cudaFree(b->n);
    cudaFree(b->inv_dx);
    for (int i = 0; i < 3; ++i) cudaFree(b->tiles[i]);
    cudaFree(b->alpha);
    cudaFree(b->dt);
    cudaFree(b->status);
    cudaFree(b->U1);
    cudaFree(b->U2);
    delete b;
}

ENOMR_API enomr_status enomr_batch_init(enomr_batch **out, int64_t nprob, const int64_t *n,
                                        const double *dx, int order, double gamma, int bc,
                                        void *stream)
{
    if (!out) return ENOMR_EINVAL;
    *out = nullptr;
    if (nprob < 1 || nprob > (1LL << 30) || !n || !dx) return ENOMR_EINVAL;
    if (order < 5 || order > 17 || (order % 2) == 0 || !(gamma > 1.0)) return ENOMR_EINVAL;
    if (bc != ENOMR_PERIODIC && bc != ENOMR_TRANSMISSIVE) return ENOMR_EINVAL;
    const int g = (order + 1) / 2;
    std::vector<long long> hb(nprob), hn(nprob);
    std::vector<double> hi(nprob);
    long long total = 0;
    for (long long p = 0; p < nprob; ++p) {
        if (n[p] < 1 || n[p] > (1LL << 30) || !(dx[p] > 0.0)) return ENOMR_EINVAL;
        if (bc == ENOMR_PERIODIC && n[p] < 2 * g) return ENOMR_EINVAL;
        hb[p] = 3 * total;
        hn[p] = n[p];
        hi[p] = 1.0 / dx[p];
        total += n[p];
    }
    enomr_batch *b = new (std::nothrow) enomr_batch();
    if (!b) return ENOMR_ENOMEM;
    b->order = order;
    b->bc = bc;
    b->nprob = nprob;
    b->total = total;
    b->gamma = gamma;
    b->stream = (cudaStream_t)stream;
    b->tp_index = 1;
    b->per_item = 1;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    b->grid = sms * 8;
    bool ok = cudaMalloc(&b->base, sizeof(long long) * nprob) == cudaSuccess &&
              cudaMalloc(&b->n, sizeof(long long) * nprob) == cudaSuccess &&
              cudaMalloc(&b->inv_dx, sizeof(double) * nprob) == cudaSuccess &&
              cudaMalloc(&b->alpha, sizeof(double) * 9 * nprob) == cudaSuccess &&
              cudaMalloc(&b->dt, sizeof(double) * nprob) == cudaSuccess &&
              cudaMalloc(&b->status, sizeof(int)) == cudaSuccess &&
              cudaMalloc(&b->U1, sizeof(double) * 3 * total) == cudaSuccess &&
              cudaMalloc(&b->U2, sizeof(double) * 3 * total) == cudaSuccess;
    for (int ti = 0; ok && ti < 3; ++ti) {
        const int cells = kTileSizes[ti] - 1;
        std::vector<BatchTile> ht;
        for (long long p = 0; p < nprob; ++p)
            for (long long x0 = 0; x0 < hn[p]; x0 += cells) ht.push_back({(int)p, (int)x0});
        b->ntiles[ti] = (long long)ht.size();
        ok = cudaMalloc(&b->tiles[ti], sizeof(BatchTile) * ht.size()) == cudaSuccess &&
             cudaMemcpy(b->tiles[ti], ht.data(), sizeof(BatchTile) * ht.size(),
                        cudaMemcpyHostToDevice) == cudaSuccess;
    }
    ok = ok && cudaMemcpy(b->base, hb.data(), sizeof(long long) * nprob, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(b->n, hn.data(), sizeof(long long) * nprob, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(b->inv_dx, hi.data(), sizeof(double) * nprob, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(b->status, 0, sizeof(int)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        enomr_batch_free(b);
        return ENOMR_ENOMEM;
    }
    *out = b;
    return ENOMR_OK;
}

ENOMR_API enomr_status enomr_batch_set_stream(enomr_batch *b, void *stream)
{
    if (!b) return ENOMR_EINVAL;
    b->stream = (cudaStream_t)stream;
    return ENOMR_OK;
}

ENOMR_API int64_t enomr_batch_total_cells(const enomr_batch *b) { return b ? b->total : -1; }

ENOMR_API enomr_status enomr_batch_step(enomr_batch *b, double *U, double cfl)
{
    if (!b || !U || !(cfl > 0.0)) return ENOMR_EINVAL;
    enomr_status st = batch_alpha_dt(b, U, cfl, true);
    if (st) return st;
    if ((st = batch_stage(b, 1, U, U, b->U1, b->tp_index, b->grid, b->per_item))) return st;
    if ((st = batch_stage(b, 2, U, b->U1, b->U2, b->tp_index, b->grid, b->per_item))) return st;
    return batch_stage(b, 3, U, b->U2, U, b->tp_index, b->grid, b->per_item);
}

ENOMR_API enomr_status enomr_batch_autotune(enomr_batch *b, const double *U, int reps,
                                            int *tile, int *grid)
{
    if (!b || !U || reps < 1) return ENOMR_EINVAL;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    static const int mults[4] = {2, 4, 8, 16};
    static const int items[3] = {1, 2, 4};
    cudaEvent_t e0, e1;
    B_TRY(cudaEventCreate(&e0));
    B_TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    int bt = b->tp_index, bg = b->grid, bk = b->per_item;
    enomr_status st = ENOMR_OK;
    for (int ti = 0; ti < 3 && !st; ++ti) {
        b->tp_index = ti;
        st = batch_alpha_dt(b, U, 0.5, true);  // alpha and dt of U for stage 1
        for (int mi = 0; mi < 4 && !st; ++mi) {
            const int gsz = sms * mults[mi];
            for (int ki = 0; ki < 3 && !st; ++ki) {
                const int k = items[ki];
                st = batch_stage(b, 1, U, U, b->U1, ti, gsz, k);  // warm-up
                cudaEventRecord(e0, b->stream);
                for (int r = 0; r < reps && !st; ++r) st = batch_stage(b, 1, U, U, b->U1, ti, gsz, k);
                cudaEventRecord(e1, b->stream);
                if (!st && cudaEventSynchronize(e1) == cudaSuccess) {
                    float ms = 0.0f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (ms < best) {
                        best = ms;
                        bt = ti;
                        bg = gsz;
                        bk = k;
                    }
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tp_index = bt;
    b->grid = bg;
    b->per_item = bk;
    if (tile) *tile = kTileSizes[bt];
    if (grid) *grid = bg;
    return st;
}

ENOMR_API enomr_status enomr_batch_config(const enomr_batch *b, int *tile, int *grid,
                                          int *tiles_per_item)
{
    if (!b) return ENOMR_EINVAL;
    if (tile) *tile = kTileSizes[b->tp_index];
    if (grid) *grid = b->grid;
    if (tiles_per_item) *tiles_per_item = b->per_item;
    return ENOMR_OK;
}

ENOMR_API enomr_status enomr_batch_get_status(enomr_batch *b)
{
    if (!b) return ENOMR_EINVAL;
    int h = 0;
    B_TRY(cudaMemcpyAsync(&h, b->status, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    B_TRY(cudaStreamSynchronize(b->stream));
    B_TRY(cudaMemsetAsync(b->status, 0, sizeof(int), b->stream));
    B_TRY(cudaStreamSynchronize(b->stream));
    return h ? ENOMR_ENONPHYS : ENOMR_OK;
}

}  // extern "C"
