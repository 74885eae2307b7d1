// enomr_tma.cuh -- the 2D Euler sweeps with their tiles staged by the
// Tensor Memory Accelerator, in a persistent kernel with a two-deep ring.
//
// arXiv 2311.15504: the arithmetic is that of enomr_sweep.cuh (Sec. 2.1,
// Eq. 1DWENOFD; Sec. 3.2; Sec. 4; Eq. TVD3rdRK); only the staging of a
// tile's cells differs, so the results are those of the k_sweep instances
// bit for bit.
//
// Each CTA loops over tiles t = blockIdx.x, blockIdx.x + gridDim.x, ...
// One thread issues a cp.async.bulk.tensor copy of tile t + gridDim.x into
// the free slot of a two-slot ring before the CTA waits (mbarrier, bounded)
// for tile t, so the next tile's load overlaps this tile's arithmetic.  A
// copy moves one box of the state [4][ny][nx] (all four components at once):
//   x sweep: {BW = S + 1 cells, NL rows, 4} starting at an even x (16-byte
//            alignment of the innermost coordinate), the tile's first cell
//            at offset (x0 - g) - xs in {0, 1} of each row;
//   y sweep: {NL columns, S rows, 4}, i.e. [4][S][NL] in shared memory, the
//            lines interleaved, so that the threads of a warp (line =
//            tid % NL, p = tid / NL) read consecutive doubles: no bank
//            conflicts without padding.
// Positions outside the grid arrive as zeros; ghost cells (clamp or wrap)
// and the rows or columns past the last line are then filled from global
// memory with plain loads, by the tiles at the ends of the lines only.
#pragma once

#include <cuda.h>

#include "enomr_sweep.cuh"

namespace enomr {

template <int R, int C, int DIR, int TP, int NL, bool SP = false>
struct TmaSmem {
    static constexpr int g = (R + 1) / 2, W = 2 * g - 1, T = Tab<R>::T;
    static constexpr int S = TP + 2 * g - 1, NS = NL * S;
    static constexpr int BW = (DIR == 0) ? S + 1 : NL;        // box extent along x
    static constexpr int RAWN = (DIR == 0) ? NL * BW : S * NL;  // doubles per component
    static_assert(DIR != 0 || (S + 1) % 2 == 0, "x box width must be even (16-byte rows)");
    static_assert((C * RAWN * 8) % 128 == 0, "ring slots must stay 128-byte aligned");
    double raw[2][C * RAWN];  // ring of tile copies, global component order
    double sF[C * NS];
    double sP[SP ? 4 * NS : 1];  // sqrt(rho), u_n, u_t, H (SP: staged per cell)
    union {
        double sFh[C * NL * TP];
        unsigned short rep[NS];
    };
    unsigned long long red[TP * NL / 32][3];
    union {
        int list[TP * NL];
        unsigned short slist[NS];
    };
    double sA[T * W];
    unsigned long long full[2];  // mbarriers of the ring slots
    int nlist;
    int nrep;
};

// Tile view over the ring slot holding the current tile (u: the slot plus
// the row offset of the x sweep).  State components are mapped from line
// order (rho, m_n, m_t, E) to the global order of the copy.
template <int R, int C, int DIR, int TP, int NL, bool SP = false>
struct TmaTile {
    using SM = TmaSmem<R, C, DIR, TP, NL, SP>;
    static constexpr bool kLoads = false;
    // SP false: sqrt(rho), u_n, u_t, H are evaluated where an interface needs
    // them (the two centre cells of an interface that is not flat on one
    // state), not staged: 9 KB less shared memory per tile and no staging
    // stores, for a little more FP64 work on the long path.  SP true: staged
    // per cell, as the loading sweeps do.
    static constexpr bool kStagedP = SP;
    static constexpr int S = SM::S, BW = SM::BW, RAWN = SM::RAWN;
    SM &sm;
    double *u;
    __device__ __forceinline__ static int gq(int q)
    {
        return (DIR == 1 && C == 4 && (q == 1 || q == 2)) ? 3 - q : q;
    }
    __device__ __forceinline__ static int ri(int line, int s)
    {
        return (DIR == 0) ? line * BW + s : s * NL + line;
    }
    __device__ __forceinline__ static int ci(int line, int s)
    {
        return (DIR == 0) ? line * S + s : s * NL + line;
    }
    __device__ __forceinline__ double &U(int q, int line, int s) const
    {
        return u[gq(q) * RAWN + ri(line, s)];
    }
    __device__ __forceinline__ double &F(int q, int line, int s) const { return sm.sF[q * SM::NS + ci(line, s)]; }
    __device__ __forceinline__ double &P(int q, int line, int s) const
    {
        return sm.sP[SP ? q * SM::NS + ci(line, s) : 0];
    }
    __device__ __forceinline__ double &Fh(int q, int line, int p) const
    {
        return sm.sFh[q * NL * TP + ((DIR == 0) ? line * TP + p : p * NL + line)];
    }
    __device__ __forceinline__ unsigned short *rep() const { return sm.rep; }
    __device__ __forceinline__ unsigned short *slist() const { return sm.slist; }
    __device__ __forceinline__ int *list() const { return sm.list; }
    __device__ __forceinline__ int &nlist() const { return sm.nlist; }
    __device__ __forceinline__ int &nrep() const { return sm.nrep; }
    __device__ __forceinline__ unsigned long long (*red() const)[3] { return sm.red; }
};

// ---- PTX: mbarrier and bulk tensor copies (shared::cta addresses) ----------
__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// One try_wait on phase `parity`; true once that phase has completed.
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after about `limit` SM clock cycles.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity,
                                          long long limit)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map,
                                            unsigned long long *bar, int c0, int c1, int c2)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2),
        "r"(smem_u32(bar))
        : "memory");
}

// Wait limit of a tile copy: 2^31 cycles, about a second at 2 GHz.
constexpr long long TMA_WAIT_LIMIT = 1LL << 31;

// CTAs per SM of the high-occupancy TMA sweeps: five (48 registers per
// thread, as the loading instances) where five tiles' shared memory fits in
// an SM (228 KB, 1 KB reserved per CTA), else four (64 registers).
template <int R, int DIR, int TP, int NL>
struct TmaCtas {
    static constexpr int value =
        5 * (sizeof(TmaSmem<R, 4, DIR, TP, NL>) + 1024) <= 228 * 1024 ? 5 : 4;
};

template <int R, int DIR, int TP, int NL>
struct TmaGeom {
    static constexpr int g = (R + 1) / 2;
    // tiles per line group along the line, and line groups
    __host__ __device__ static long long nseg(long long nlen) { return (nlen + TP - 2) / (TP - 1); }
    __host__ __device__ static long long ngrp(long long nlines) { return (nlines + NL - 1) / NL; }
};

// Persistent TMA sweep over ntiles tiles (x sweep: segment-fastest order
// along the rows; y sweep: column-group-fastest, so that the concurrently
// processed tiles of a wave share DRAM pages).
template <int R, int DIR, int TP, int NL, int MINB, bool SP>
__global__ void __launch_bounds__(TP *NL, MINB)
    k_sweep_tma(const __grid_constant__ CUtensorMap map, SweepArgs A, long long ntiles)
{
    constexpr int C = 4;
    using SM = TmaSmem<R, C, DIR, TP, NL, SP>;
    using G = TmaGeom<R, DIR, TP, NL>;
    constexpr int g = SM::g, S = SM::S, NS = SM::NS, RAWN = SM::RAWN, NT = TP * NL;
    constexpr unsigned BYTES = (unsigned)(sizeof(double) * C * RAWN);
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    SM &sm = *reinterpret_cast<SM *>(smem_dyn);
    const int tid = threadIdx.x;
    const long long nx = A.nx, ny = A.ny, ncell = nx * ny;
    const long long nlen = (DIR == 0) ? nx : ny;
    const long long nlines = (DIR == 0) ? ny : nx;
    const long long nseg = G::nseg(nlen), ngrp = G::ngrp(nlines);

    // tile index -> (first interface, first line); the launcher keeps the
    // tile count below 2^31, so 32-bit division suffices (64-bit division is
    // a long software sequence)
    const unsigned nfast = (unsigned)((DIR == 0) ? nseg : ngrp);
    auto tile_of = [&](long long t, long long &x0, long long &l0) {
        const unsigned tt = (unsigned)t, q = tt / nfast, r = tt - q * nfast;
        const unsigned seg = (DIR == 0) ? r : q, grp = (DIR == 0) ? q : r;
        x0 = (long long)seg * (TP - 1);
        l0 = (long long)grp * NL;
    };
    auto issue = [&](long long t, int slot) {
        long long x0, l0;
        tile_of(t, x0, l0);
        mbar_expect_tx(&sm.full[slot], BYTES);
        if (DIR == 0) {
            const long long xs = (x0 - g) - ((x0 - g) & 1);
            tma_load_3d(sm.raw[slot], &map, &sm.full[slot], (int)xs, (int)l0, 0);
        } else {
            tma_load_3d(sm.raw[slot], &map, &sm.full[slot], (int)l0, (int)(x0 - g), 0);
        }
    };

    if (tid == 0) {
        mbar_init(&sm.full[0], 1);
        mbar_init(&sm.full[1], 1);
        fence_barrier_init();
        fence_proxy_async();
    }
    load_a_table<R>(sm.sA, tid, NT);
    __syncthreads();
    if (tid == 0 && (long long)blockIdx.x < ntiles) issue(blockIdx.x, 0);

    int it = 0;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        const int slot = it & 1;
        const long long tn = t + gridDim.x;
        if (tid == 0 && tn < ntiles) {
            // the other slot was released by the barrier that ended the
            // previous tile; order its generic-proxy accesses before the copy
            fence_proxy_async();
            issue(tn, slot ^ 1);
        }
        const bool ok = mbar_wait(&sm.full[slot], (unsigned)((it >> 1) & 1), TMA_WAIT_LIMIT);
        if (__syncthreads_or(!ok)) {
            // a copy never completed: report it, wait (bounded) for the copy
            // in flight into the other slot, and stop
            if (tid == 0) {
                atomicOr(A.status, ST_TMA_TIMEOUT);
                if (tn < ntiles) mbar_wait(&sm.full[slot ^ 1], (unsigned)(((it + 1) >> 1) & 1),
                                           TMA_WAIT_LIMIT);
            }
            return;
        }
        long long x0, l0;
        tile_of(t, x0, l0);
        double *base = sm.raw[slot];
        if (DIR == 0) base += (x0 - g) & 1;  // the copy started at the even x at or below x0 - g
        const TmaTile<R, C, DIR, TP, NL, SP> tile{sm, base};
        // ghost cells and lines past the last one: plain loads (the ends of
        // the lines only)
        if (x0 - g < 0 || x0 - g + S > nlen || l0 + NL > nlines) {
            for (int idx = tid; idx < NS; idx += NT) {
                int line, s;
                if (DIR == 0) {
                    line = idx / S;
                    s = idx - line * S;
                } else {
                    s = idx / NL;
                    line = idx - s * NL;
                }
                const long long craw = x0 - g + s, L = l0 + line;
                if (craw < 0 || craw >= nlen || L >= nlines) {
                    const long long Lc = L < nlines ? L : nlines - 1;
                    const long long cell = ghost(craw, nlen, A.bc);
                    const long long gi = (DIR == 0) ? Lc * nx + cell : cell * nx + Lc;
#pragma unroll
                    for (int q = 0; q < C; ++q)
                        base[q * RAWN + TmaTile<R, C, DIR, TP, NL, SP>::ri(line, s)] =
                            A.U[q * ncell + gi];
                }
            }
        }
        sweep_tile<R, C, DIR, TP, NL, false>(A, x0, l0, sm.sA, tile);
        __syncthreads();  // the slot and the tile arrays are free again
    }
}

// Host launcher: a persistent grid of (SMs x resident CTAs) CTAs, at most
// one per tile.  map: tensor map of the state U of a (tiled, 3D: {nx, ny, 4})
// with this sweep's box.
template <int R, int DIR, int TP, int NL, int MINB, bool SP>
cudaError_t launch_sweep_tma(const CUtensorMap &map, const SweepArgs &a, cudaStream_t s)
{
    using SM = TmaSmem<R, 4, DIR, TP, NL, SP>;
    using G = TmaGeom<R, DIR, TP, NL>;
    if (DIR == 0 && !row_epilogue_ok(a)) return cudaErrorInvalidValue;
    constexpr int kMaxDev = 64;
    static int ctas[kMaxDev] = {}, sms[kMaxDev] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
    auto k = k_sweep_tma<R, DIR, TP, NL, MINB, SP>;
    if (ctas[dev] == 0) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SM));
        if (e != cudaSuccess) return e;
        int n = 0, m = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, TP * NL, sizeof(SM));
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        if (n < 1) return cudaErrorInvalidConfiguration;
        sms[dev] = m;
        ctas[dev] = n < MINB ? n : MINB;  // the residency the registers were sized for
    }
    const long long nlen = DIR == 0 ? a.nx : a.ny, nlines = DIR == 0 ? a.ny : a.nx;
    const long long ntiles = G::nseg(nlen) * G::ngrp(nlines);
    if (ntiles >= (1LL << 31)) return cudaErrorInvalidValue;  // 32-bit tile indices
    long long grid = (long long)sms[dev] * ctas[dev];
    if (grid > ntiles) grid = ntiles;
    k<<<(unsigned)grid, TP * NL, sizeof(SM), s>>>(map, a, ntiles);
    return cudaGetLastError();
}

}  // namespace enomr
