// enomr_sweep.cuh -- Euler line sweeps (1D, and the x and y sweeps of 2D)
// and the batched persistent 1D stage.
//
// arXiv 2311.15504: Sec. 2.1 (Eq. 1DWENOFD, Eq. LF_Flux_Split), Sec. 3.2,
// Sec. 4 (Roe-averaged characteristic decomposition, Euler equations),
// Eq. TVD3rdRK.
//
// Rows of L are scaled to carry a unit entry (the scheme is invariant to
// such scalings, Sec. 3.3), so a projection costs 3 FMAs (1 for the shear
// field) instead of 4; the 1/2 of the splitting and the row scalings are
// folded into the back-projection.
// Tiles: a CTA stages TP + 2g - 1 cells of NL lines (with their ghost cells,
// wrapped or clamped) into shared memory together with primitive values
// and physical fluxes, computes TP interface fluxes per line (one per
// thread) and updates the TP - 1 cells between them; neighbouring tiles
// overlap by one interface.
#pragma once

#include "enomr_kernels.cuh"

namespace enomr {

// ---------------------------------------------------------------------------
// Euler line sweep.  DIR 0: lines are rows (x contiguous); DIR 1: lines are
// columns.  C = 3 (1D) or 4 (2D, components rho, m_x, m_y, E).
// ---------------------------------------------------------------------------
template <int R, int C, int TP, int NL>
struct SweepSmem {
    static constexpr int g = (R + 1) / 2, S = TP + 2 * g - 1;
    double sU[C][NL][S];
    double sF[C][NL][S];
    double sP[4][NL][S];  // sqrt(rho), u_n, u_t, H
    // the staging phase's arrays share storage with arrays of the later
    // phases (separated from them by barriers)
    union {
        double sFh[C][NL][TP];
        unsigned short rep[NL * S];  // staging: cell -> the representative it copies
    };
    unsigned long long red[TP * NL / 32][3];
    union {
        int list[TP * NL];             // interfaces (line * TP + p) that take the long path
        unsigned short slist[NL * S];  // staging: representatives to evaluate
    };
    int nlist;
    int nrep;
    static_assert(sizeof(unsigned short) * NL * S <= sizeof(double) * C * NL * TP &&
                      sizeof(unsigned short) * NL * S <= sizeof(int) * TP * NL,
                  "staging arrays must fit in the storage they share");
};

// Largest partly filled last warp of a tile's long-path list that is
// evaluated field-parallel (interface_flux, fsel).
constexpr int LONG_TAIL = 16;

// View of a tile's shared memory used by sweep_tile and interface_flux.
// U(q, line, s): state component q (line order: rho, m_n, [m_t], E) of
// staged cell s of tile line `line`; F: its normal flux; P: sqrt(rho), u_n,
// u_t, H (views with kStagedP; the others evaluate them where needed);
// Fh(q, line, p): flux of interface p.  kLoads: the staging phase
// loads the cells from global memory itself (true here); a view whose
// cells are already in shared memory (the TMA ring of enomr_tma.cuh) reads
// them in place.
template <int R, int C, int DIR, int TP, int NL>
struct ClassicTile {
    static constexpr bool kLoads = true;
    static constexpr bool kStagedP = true;  // P staged per cell (else evaluated on demand)
    SweepSmem<R, C, TP, NL> &sm;
    __device__ __forceinline__ double &U(int q, int line, int s) const { return sm.sU[q][line][s]; }
    __device__ __forceinline__ double &F(int q, int line, int s) const { return sm.sF[q][line][s]; }
    __device__ __forceinline__ double &P(int q, int line, int s) const { return sm.sP[q][line][s]; }
    __device__ __forceinline__ double &Fh(int q, int line, int p) const { return sm.sFh[q][line][p]; }
    __device__ __forceinline__ unsigned short *rep() const { return sm.rep; }
    __device__ __forceinline__ unsigned short *slist() const { return sm.slist; }
    __device__ __forceinline__ int *list() const { return sm.list; }
    __device__ __forceinline__ int &nlist() const { return sm.nlist; }
    __device__ __forceinline__ int &nrep() const { return sm.nrep; }
    __device__ __forceinline__ unsigned long long (*red() const)[3] { return sm.red; }
};

// State of ghost cell craw (< 0 or >= the line length) of line L, in
// global component order, for a sweep with boundary sides: the kind of its
// side at the line's along-side position gives a copy of the nearest cell,
// the mirror image with the normal momentum negated, or the inflow state.
template <int C, int DIR>
__device__ __forceinline__ void side_cell(const SweepArgs &A, long long craw, long long L,
                                          double *u)
{
    constexpr int QN = (DIR == 0) ? 1 : 2;
    const long long nx = A.nx, ny = A.ny, ncell = nx * ny;
    const long long nlen = (DIR == 0) ? nx : ny;
    const SideDev &sd = craw < 0 ? *A.side_lo : *A.side_hi;
    // stage time; dt is not read when the stage sits at t (a lone RHS
    // evaluation may come before any step has set it)
    const double ts =
        A.t_coef != 0.0 ? __dadd_rn(*A.t_dev, __dmul_rn(A.t_coef, *A.dt_time)) : *A.t_dev;
    const double pos = __dmul_rn(__dadd_rn((double)L, 0.5), A.pos_h);
    const bool lo = pos < __dadd_rn(sd.split0, __dmul_rn(sd.rate, ts));
    const int kind = lo ? sd.kind_lo : sd.kind_hi;
    if (kind == SIDE_INFLOW) {
        const double *st = lo ? sd.st_lo : sd.st_hi;
#pragma unroll
        for (int q = 0; q < C; ++q) u[q] = st[q];
        return;
    }
    long long cell;
    if (kind == SIDE_REFLECTIVE) {
        // mirror image; a tile may stage cells further out than any window
        // reaches (lines shorter than the tile), which are kept in the line
        cell = craw < 0 ? -1 - craw : 2 * nlen - 1 - craw;
        cell = cell < 0 ? 0 : (cell >= nlen ? nlen - 1 : cell);
    } else {
        cell = craw < 0 ? 0 : nlen - 1;
    }
    const long long gi = (DIR == 0) ? L * nx + cell : cell * nx + L;
#pragma unroll
    for (int q = 0; q < C; ++q) u[q] = A.U[q * ncell + gi];
    if (kind == SIDE_REFLECTIVE) u[QN] = -u[QN];
}

// Flux of interface x_{k-1/2}, k = x0 + p, of tile line `line` into
// t.Fh(., line, p) (and the selections / field values when requested).
// FLATP: the interface is flat (both sides' centre triples of cell states
// are bitwise equal), e2: its two centre states are bitwise equal.  The
// long path (FLATP false) holds warp votes: all 32 lanes of the warp call
// it together, lanes with valid == false only vote.
// fsel >= 0 (long path, C = 4 only): field-parallel form; lanes 4i .. 4i+3
// of the warp hold one interface and each evaluates field fsel = lane % 4
// only (same operations as the loop over the fields); the four values meet
// at the first lane by shuffles, which alone back-projects and stores.
template <int R, int C, int DIR, int TP, int NL, bool FLATP, class Tile>
__device__ __forceinline__ void interface_flux(const SweepArgs &A, long long x0, long long l0,
                                               const double *sA, const Tile &t, int p, int line,
                                               bool valid, bool e2, int fsel = -1)
{
    constexpr int g = (R + 1) / 2, W = 2 * g - 1, T = Tab<R>::T;
    const long long nlen = (DIR == 0) ? A.nx : A.ny;
    if constexpr (FLATP) {
        if (e2 && !A.ft_out) {
            // Both windows flat on one state U_k (cells k-1 and k bitwise
            // equal): both sides take S(0,0) on it, the Roe state is U_k,
            // f^+ + f^- = l F(U_k) for every field (the alpha terms cancel)
            // and the back-projection returns R L F(U_k) = F(U_k).  The
            // interface flux is the cell's staged physical flux, exactly;
            // the long evaluation differs from it by rounding only.  (A
            // forward pass that records f^+ + f^- for the adjoint takes
            // the long evaluation.)
            const long long nlines = (DIR == 0) ? A.ny : A.nx;
            const long long Lg = l0 + line, k = x0 + p;
            if (A.sel) {
                const long long NI = nlen + 1;
#pragma unroll
                for (int f = 0; f < C; ++f) {
                    A.sel[((0 * C + f) * nlines + Lg) * NI + k] = (uint8_t)(T + 2);
                    A.sel[((1 * C + f) * nlines + Lg) * NI + k] = (uint8_t)(T + 2);
                }
            }
            const int sr = p + g;
#pragma unroll
            for (int q = 0; q < C; ++q) t.Fh(q, line, p) = t.F(q, line, sr);
            return;
        }
    }
    const long long nlines = (DIR == 0) ? A.ny : A.nx;
    const long long Lg = l0 + line;
    const long long k = x0 + p;  // interface x_{k-1/2}, cells k-1 | k
    const int sl = p + g - 1, sr = p + g;

    // Roe average (Sec. 4); for two bitwise-equal states it is that state.
    bool eqLR = true;
#pragma unroll
    for (int q = 0; q < C; ++q)
        eqLR = eqLR && (__double_as_longlong(t.U(q, line, sl)) == __double_as_longlong(t.U(q, line, sr)));
    // sqrt(rho), u_n, u_t, H of the two centre cells: staged per cell, or
    // (views without them) evaluated here by the same operations
    const RoeFace rf = [&]() {
        if constexpr (Tile::kStagedP) {
            return roe_face(eqLR, t.P(0, line, sl), t.P(1, line, sl), t.P(2, line, sl),
                            t.P(3, line, sl), t.P(0, line, sr), t.P(1, line, sr),
                            t.P(2, line, sr), t.P(3, line, sr), C == 4, A.gm1, A.inv_gm1);
        } else {
            const StagedCell<C> cl = stage_cell<C>(t.U(0, line, sl), t.U(1, line, sl),
                                                   (C == 4) ? t.U(2, line, sl) : 0.0,
                                                   t.U(C - 1, line, sl), A.gm1);
            if (eqLR)
                return roe_face(true, cl.sq, cl.un, cl.ut, cl.H, cl.sq, cl.un, cl.ut, cl.H, C == 4,
                                A.gm1, A.inv_gm1);
            const StagedCell<C> cr = stage_cell<C>(t.U(0, line, sr), t.U(1, line, sr),
                                                   (C == 4) ? t.U(2, line, sr) : 0.0,
                                                   t.U(C - 1, line, sr), A.gm1);
            return roe_face(false, cl.sq, cl.un, cl.ut, cl.H, cr.sq, cr.un, cr.ut, cr.H, C == 4,
                            A.gm1, A.inv_gm1);
        }
    }();
    if (valid && fsel <= 0 && !positive(rf.c2)) atomicOr(A.status, ST_NONPHYS_ROE);
    const double uh = rf.uh, vh = rf.vh, Hh = rf.Hh, hq = rf.hq, cs = rf.cs, kap = rf.kap,
                 c2g = rf.c2g, b1 = rf.b1;

    const double *al = A.alpha + 3 * (Lg < nlines ? Lg : nlines - 1);
    const double a_m = al[0], a_0 = al[1], a_p = al[2];

    // Back-projection accumulators.  With phi_f = s_f (f^+ + f^-)_f and the
    // inverse row scalings s = (b1/4, -b1/2, [1/2,] b1/4) (the 1/2 of the
    // splitting included), F = R phi reads
    //   F0 = (phi_0 + phi_a) + phi_1,   F1 = u F0 + c (phi_a - phi_0),
    //   F2 = v F0 + phi_2 (2D),         FE = H (phi_0 + phi_a) + u c (phi_a - phi_0)
    //                                        + hq phi_1 + v phi_2,
    // phi_a being the u+c field.
    double acc_s = 0.0, acc_d = 0.0, ph1 = 0.0, ph2 = 0.0;

    // Scaled left-eigenvector row of field f (a unit entry on E, or on the
    // tangential momentum for the shear field) and the split speed alpha_f.
    auto row = [&](int f, double &l0c, double &l1c, double &alpha) {
        if (C == 4 && f == 2) {
            l0c = -vh;
            l1c = 0.0;
            alpha = a_0;
        } else if (f == 0) {
            l0c = fma(uh, kap, hq);
            l1c = -(uh + kap);
            alpha = a_m;
        } else if (f == C - 1) {
            l0c = fma(-uh, kap, hq);
            l1c = -(uh - kap);
            alpha = a_p;
        } else {
            l0c = hq - c2g;
            l1c = -uh;
            alpha = a_0;
        }
    };
    // w = l U and q = l F of staged cell s (the same operations on every path).
    auto project = [&](int f, int s, double l0c, double l1c, double &w, double &q) {
        if (C == 4 && f == 2) {
            w = fma(l0c, t.U(0, line, s), t.U(2, line, s));
            q = fma(l0c, t.F(0, line, s), t.F(2, line, s));
        } else {
            w = t.U(C - 1, line, s);
            q = t.F(C - 1, line, s);
            if (C == 4) {
                w = fma(-vh, t.U(2, line, s), w);
                q = fma(-vh, t.F(2, line, s), q);
            }
            w = fma(l1c, t.U(1, line, s), w);
            q = fma(l1c, t.F(1, line, s), q);
            w = fma(l0c, t.U(0, line, s), w);
            q = fma(l0c, t.F(0, line, s), q);
        }
    };
    auto accumulate = [&](int f, double ft) {
        if (f == 0) {
            const double ph = 0.25 * b1 * ft;
            acc_s += ph;
            acc_d -= ph;
        } else if (f == C - 1) {
            const double ph = 0.25 * b1 * ft;
            acc_s += ph;
            acc_d += ph;
        } else if (C == 4 && f == 2) {
            ph2 = 0.5 * ft;
        } else {
            ph1 = -0.5 * b1 * ft;
        }
    };

    if (FLATP) {
        // e2: the two centre states are bitwise equal, so are their
        // projections; the second one is not recomputed.
#pragma unroll
        for (int f = 0; f < C; ++f) {
            double l0c, l1c, alpha, w, q;
            row(f, l0c, l1c, alpha);
            project(f, sl, l0c, l1c, w, q);
            const double fp = fma(alpha, w, q);
            if (!e2) project(f, sr, l0c, l1c, w, q);
            const double fm = fma(-alpha, w, q);
            accumulate(f, fp + fm);
            if (A.sel && valid) {
                const long long NI = nlen + 1;
                A.sel[((0 * C + f) * nlines + Lg) * NI + k] = (uint8_t)(T + 2);
                A.sel[((1 * C + f) * nlines + Lg) * NI + k] = (uint8_t)(T + 2);
            }
            if (A.ft_out && valid) A.ft_out[(f * nlines + Lg) * (nlen + 1) + k] = fp + fm;
        }
    } else if (C == 4 && fsel >= 0) {
        const int f = fsel;
        double l0c, l1c, alpha;
        row(f, l0c, l1c, alpha);
        double vp[W], vm[W];
#pragma unroll
        for (int j = 0; j < 2 * g; ++j) {
            double w, q;
            project(f, p + j, l0c, l1c, w, q);
            if (j <= 2 * g - 2) vp[j] = fma(alpha, w, q);
            if (j >= 1) vm[2 * g - 1 - j] = fma(-alpha, w, q);
        }
        int selp, selm;
        double fp, fm;
        if (A.sel_in) {
            const long long NI = nlen + 1;
            selp = A.sel_in[((0 * C + f) * nlines + Lg) * NI + k];
            selm = A.sel_in[((1 * C + f) * nlines + Lg) * NI + k];
            fp = mr_value_forced<R>(vp, sA, selp);
            fm = mr_value_forced<R>(vm, sA, selm);
        } else {
            fp = mr_value<R>(vp, sA, valid, selp);
            fm = mr_value<R>(vm, sA, valid, selm);
        }
        const double ft = fp + fm;
        if (A.sel && valid) {
            const long long NI = nlen + 1;
            A.sel[((0 * C + f) * nlines + Lg) * NI + k] = (uint8_t)selp;
            A.sel[((1 * C + f) * nlines + Lg) * NI + k] = (uint8_t)selm;
        }
        if (A.ft_out && valid) A.ft_out[(f * nlines + Lg) * (nlen + 1) + k] = ft;
        const int first = (threadIdx.x & 31) & ~3;
        double fts[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) fts[q] = __shfl_sync(FULL, ft, first + q);
        if constexpr (C == 4) {
#pragma unroll
            for (int q = 0; q < 4; ++q) accumulate(q, fts[q]);
        }
    } else {
#pragma unroll 1
        for (int f = 0; f < C; ++f) {
            double l0c, l1c, alpha;
            row(f, l0c, l1c, alpha);
            double vp[W], vm[W];
#pragma unroll
            for (int j = 0; j < 2 * g; ++j) {
                double w, q;
                project(f, p + j, l0c, l1c, w, q);
                if (j <= 2 * g - 2) vp[j] = fma(alpha, w, q);       // cell k-1+l, l = j-(g-1)
                if (j >= 1) vm[2 * g - 1 - j] = fma(-alpha, w, q);  // cell k-l,   l = g-j
            }
            int selp, selm;
            double fp, fm;
            if (A.sel_in) {
                // frozen choices (forced per interface): no warp votes here,
                // and the caller gives a uniform A.sel_in to the whole warp
                const long long NI = nlen + 1;
                const long long kk = valid ? k : 0, Lk = valid ? Lg : 0;
                selp = A.sel_in[((0 * C + f) * nlines + Lk) * NI + kk];
                selm = A.sel_in[((1 * C + f) * nlines + Lk) * NI + kk];
                fp = mr_value_forced<R>(vp, sA, selp);
                fm = mr_value_forced<R>(vm, sA, selm);
            } else {
                fp = mr_value<R>(vp, sA, valid, selp);
                fm = mr_value<R>(vm, sA, valid, selm);
            }
            accumulate(f, fp + fm);
            if (A.sel && valid) {
                const long long NI = nlen + 1;
                A.sel[((0 * C + f) * nlines + Lg) * NI + k] = (uint8_t)selp;
                A.sel[((1 * C + f) * nlines + Lg) * NI + k] = (uint8_t)selm;
            }
            if (A.ft_out && valid) A.ft_out[(f * nlines + Lg) * (nlen + 1) + k] = fp + fm;
        }
    }
    double Fh[C];
    Fh[0] = acc_s + ph1;
    Fh[1] = fma(uh, Fh[0], cs * acc_d);
    if (C == 4) Fh[2] = fma(vh, Fh[0], ph2);
    Fh[C - 1] = fma(Hh, acc_s, fma(uh * cs, acc_d, fma(hq, ph1, vh * ph2)));
    // a lane without an interface of its own (it only votes) must not store
    // over the owner's slot; in the field-parallel form the first lane stores
    if (valid && fsel <= 0)
#pragma unroll
        for (int q = 0; q < C; ++q) t.Fh(q, line, p) = Fh[q];
}

// A flat interface that is not on one state (or whose per-field values are
// recorded): projection of its centre cells (interface_flux, FLATP).  Not
// inlined, so that it stays a branch of its caller.
template <int R, int C, int DIR, int TP, int NL, class Tile>
__device__ __noinline__ void flat_projection(const SweepArgs &A, long long x0, long long l0,
                                             const double *sA, const Tile &t, int p, int line,
                                             bool e2)
{
    interface_flux<R, C, DIR, TP, NL, true>(A, x0, l0, sA, t, p, line, true, e2);
}

// Long path of one interface per lane; all 32 lanes call it together.  Not
// inlined, like the other FP64-heavy paths of a tile: kept out of line, its
// code cannot be merged (if-converted) into the per-thread phases of the
// tile, where most lanes would issue it predicated off.
template <int R, int C, int DIR, int TP, int NL, class Tile>
__device__ __noinline__ void long_path(const SweepArgs &A, long long x0, long long l0,
                                       const double *sA, const Tile &t, int p, int line,
                                       bool valid)
{
    interface_flux<R, C, DIR, TP, NL, false>(A, x0, l0, sA, t, p, line, valid, false);
}

// Field-parallel long path of one interface (fsel = lane % 4); all 32 lanes
// call it together.  Not inlined: a second inlined copy of the long path
// would double the sweeps' register spills.
template <int R, int C, int DIR, int TP, int NL, class Tile>
__device__ __noinline__ void long_tail(const SweepArgs &A, long long x0, long long l0,
                                       const double *sA, const Tile &t, int p, int line,
                                       bool valid, int fsel)
{
    interface_flux<R, C, DIR, TP, NL, false>(A, x0, l0, sA, t, p, line, valid, false, fsel);
}

// One tile: NL lines x TP interfaces starting at interface x0 of line l0.
// All threads of the CTA must call it; it ends after its epilogue.
// EXT: the 2D sweep with boundary sides and a body force (SweepArgs'
// side_lo, side_hi, ..., src set); the plain instances leave them unread.
// LM: form of the long path.  LONG_SPLIT: whole warps out of line
// (long_path) and a partly filled last warp of at most LONG_TAIL interfaces
// field-parallel (long_tail).  LONG_FIELDS: as LONG_SPLIT, and a whole list
// of at most eight interfaces per warp field-parallel.  LONG_INLINE: every
// warp inline, interface-parallel.  Measured on 4096^2 (piecewise-constant
// state, order 9 / 17): the row sweep is fastest with LONG_FIELDS (0.76 /
// 1.15 ms), the column sweep with LONG_SPLIT (0.93 / 1.30 ms against 0.97 /
// 1.33 with LONG_FIELDS): its tiles hold four lines, so a front crossing
// them fills its long-path warps better.
enum : int { LONG_INLINE = 0, LONG_SPLIT = 1, LONG_FIELDS = 2 };
template <int DIR>
struct LongForm {
    static constexpr int value = DIR == 0 ? LONG_FIELDS : LONG_SPLIT;
};

template <int R, int C, int DIR, int TP, int NL, bool EXT = false,
          int LM = LongForm<DIR>::value, class Tile>
__device__ __forceinline__ void sweep_tile(const SweepArgs &A, long long x0, long long l0,
                                           const double *sA, const Tile &t)
{
    constexpr int g = (R + 1) / 2, S = TP + 2 * g - 1;
    constexpr int NT = TP * NL;
    constexpr int QN = (DIR == 0) ? 1 : 2;  // normal momentum component
    constexpr int QT = (DIR == 0) ? 2 : 1;  // tangential momentum component (C = 4)
    const long long nx = A.nx, ny = A.ny, ncell = nx * ny;
    const long long nlen = (DIR == 0) ? nx : ny;
    const long long nlines = (DIR == 0) ? ny : nx;
    const int tid = threadIdx.x;

    if (tid == 0) {
        t.nlist() = 0;
        t.nrep() = 0;
    }
    __syncthreads();
    // ---- stage cells, primitives and physical fluxes (normal direction).
    // A staged cell bitwise equal to its predecessor along the line has the
    // same primitives and flux: only representatives (a line's first cell
    // within each warp's 32 staged cells, or one that differs from its
    // predecessor) are evaluated, by whole warps from a compacted list, and
    // the others copy their representative's values.  The staged values are
    // those of evaluating every cell, bit for bit; a piecewise-constant
    // region costs a few evaluations per tile instead of one per cell.
    static_assert(32 % NL == 0, "lines per tile must divide the warp");
    constexpr int NS = NL * S;
    constexpr int PD = (DIR == 0) ? 1 : NL;  // lane distance to the predecessor
    constexpr unsigned CLS = NL == 1 ? 0xffffffffu
                           : NL == 2 ? 0x55555555u
                           : NL == 4 ? 0x11111111u
                           : NL == 8 ? 0x01010101u
                           : NL == 16 ? 0x00010001u : 0x00000001u;  // lanes of one line (DIR 1)
    const int lane = tid & 31;
    bool varies_me = false;  // a cell differs from its predecessor in the same warp
    for (int base = tid & ~31; base < NS; base += NT) {
        const int idx = base + lane;
        const bool act = idx < NS;
        int line = 0, s = 0;
        if (DIR == 0) {
            line = idx / S;
            s = idx - line * S;
        } else {
            s = idx / NL;
            line = idx - s * NL;
        }
        double u[C];
#pragma unroll
        for (int q = 0; q < C; ++q) u[q] = 0.0;
        if (!Tile::kLoads) {
            // cells already staged (and their ghosts filled) in shared memory
            if (act)
#pragma unroll
                for (int q = 0; q < C; ++q) u[q] = t.U(q, line, s);
        } else if (act) {
            long long L = l0 + line;
            if (L >= nlines) L = nlines - 1;
            const long long craw = x0 - g + s;
            if (EXT && (craw < 0 || craw >= nlen)) {
                side_cell<C, DIR>(A, craw, L, u);
            } else {
                const long long cell = ghost(craw, nlen, A.bc);
                const long long gi = (DIR == 0) ? L * nx + cell : cell * nx + L;
#pragma unroll
                for (int q = 0; q < C; ++q) u[q] = A.U[q * ncell + gi];
            }
            t.U(0, line, s) = u[0];
            t.U(1, line, s) = u[QN];
            if (C == 4) t.U(2, line, s) = u[QT];
            t.U(C - 1, line, s) = u[C - 1];
        }
        bool same = lane >= PD && s > 0;
#pragma unroll
        for (int q = 0; q < C; ++q) {
            const double pq = __shfl_up_sync(FULL, u[q], PD);
            same = same && (__double_as_longlong(pq) == __double_as_longlong(u[q]));
        }
        const bool rep = act && !same;
        varies_me = varies_me || (rep && lane >= PD && s > 0);
        const unsigned reps = __ballot_sync(FULL, rep);
        // representative of this cell: the nearest representative lane at or
        // below this one on the same line (a line's first lane is one)
        unsigned m = reps & (lane == 31 ? FULL : ((2u << lane) - 1u));
        if (DIR == 1) m &= CLS << (lane % NL);
        if (act) t.rep()[idx] = (unsigned short)(base + 31 - __clz(m));
        if (reps) {
            int b0 = 0;
            if (lane == 0) b0 = atomicAdd(&t.nrep(), __popc(reps));
            b0 = __shfl_sync(FULL, b0, 0);
            if (rep) t.slist()[b0 + __popc(reps & ((1u << lane) - 1u))] = (unsigned short)idx;
        }
    }
    const bool varies = __syncthreads_or(varies_me) != 0;
    // A tile whose every line holds one state (its halos included): every
    // interface is flat on that line's state, its flux is the cell's flux and
    // every flux difference is exactly zero, so the tile goes straight to
    // its epilogue (most tiles of a piecewise-constant grid).  Only the
    // representatives that start a warp's chunk of cells have not been
    // compared with their predecessor yet.  (Selections or per-field values
    // asked for, or forced choices: the full evaluation.)
    bool constant = false;
    if (!varies && !A.sel && !A.ft_out && !A.sel_in) {
        bool bad = false;
        const int nrep = t.nrep();
        for (int j = tid; j < nrep; j += NT) {
            const int idx = t.slist()[j];
            int line, s;
            if (DIR == 0) {
                line = idx / S;
                s = idx - line * S;
            } else {
                s = idx / NL;
                line = idx - s * NL;
            }
            if (s > 0)
#pragma unroll
                for (int q = 0; q < C; ++q)
                    bad = bad || __double_as_longlong(t.U(q, line, s)) !=
                                     __double_as_longlong(t.U(q, line, s - 1));
        }
        constant = __syncthreads_or(bad) == 0;
    }
    if (!constant) {
    {
        const int nrep = t.nrep();
        for (int b = tid & ~31; b < nrep; b += NT) {
            const int j = b + lane;
            if (j < nrep) {
                const int idx = t.slist()[j];
                int line, s;
                if (DIR == 0) {
                    line = idx / S;
                    s = idx - line * S;
                } else {
                    s = idx / NL;
                    line = idx - s * NL;
                }
                const double u0 = t.U(0, line, s), uE = t.U(C - 1, line, s);
                const StagedCell<C> sc_ = stage_cell<C>(u0, t.U(1, line, s),
                                                        (C == 4) ? t.U(2, line, s) : 0.0, uE, A.gm1);
                if (!positive(u0) || !positive(sc_.p) || !below_1e300(uE))
                    atomicOr(A.status, ST_NONPHYS_CELL);
#pragma unroll
                for (int q = 0; q < C; ++q) t.F(q, line, s) = sc_.F[q];
                if constexpr (Tile::kStagedP) {
                    t.P(0, line, s) = sc_.sq;
                    t.P(1, line, s) = sc_.un;
                    t.P(2, line, s) = sc_.ut;
                    t.P(3, line, s) = sc_.H;
                }
            }
        }
    }
    __syncthreads();
    for (int idx = tid; idx < NS; idx += NT) {
        const int r = t.rep()[idx];
        if (r != idx) {
            int line, s, lr, sr_;
            if (DIR == 0) {
                line = idx / S;
                s = idx - line * S;
                lr = r / S;
                sr_ = r - lr * S;
            } else {
                s = idx / NL;
                line = idx - s * NL;
                sr_ = r / NL;
                lr = r - sr_ * NL;
            }
#pragma unroll
            for (int q = 0; q < C; ++q) t.F(q, line, s) = t.F(q, lr, sr_);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if constexpr (Tile::kStagedP) t.P(q, line, s) = t.P(q, lr, sr_);
        }
    }
    __syncthreads();

    // ---- interface fluxes.  A flat interface (see below) is evaluated by
    // its own thread; the others are appended to a list and evaluated by
    // whole warps, 32 list entries at a time, so that the long path (whose
    // candidate walk is warp-uniform) runs without idle lanes.
    {
        int p, line;
        if (DIR == 0) {
            p = tid % TP;
            line = tid / TP;
        } else {
            line = tid % NL;
            p = tid / NL;
        }
        const bool valid = (l0 + line < nlines) && (x0 + p <= nlen);
        const int sl = p + g - 1, sr = p + g;
        // Flat windows.  If the states of three consecutive cells ending or
        // starting at a side's centre are bitwise equal, every field's
        // projected values there are bitwise equal too, so that side's IS_0
        // is exactly 0, no candidate is tested and minmod returns v(0): only
        // the centre cell needs projecting.  The result is the same as on
        // the long path.
        auto same = [&](int a, int b) {
            bool e = true;
#pragma unroll
            for (int q = 0; q < C; ++q)
                e = e && (__double_as_longlong(t.U(q, line, a)) == __double_as_longlong(t.U(q, line, b)));
            return e;
        };
        const bool e0 = same(sl - 2, sl - 1), e1 = same(sl - 1, sl), e2 = same(sl, sr),
                   e3 = same(sr, sr + 1), e4 = same(sr + 1, sr + 2);
        const bool plus_flat = (e0 && e1) || (e2 && e3);   // centre cell k-1
        const bool minus_flat = (e3 && e4) || (e1 && e2);  // centre cell k (mirrored)
        // with forced (frozen) choices every interface is evaluated in full
        const bool flat = plus_flat && minus_flat && !A.sel_in;
        // One-state flat interfaces (most of a piecewise-constant grid) take
        // the cell's flux inline; the few other flat ones project their centre
        // cells in a separate, non-inlined function, so that the compiler
        // cannot if-convert that FP64 code into this per-thread path (where
        // every one-state lane would issue it predicated off and hold the
        // FP64 pipe for nothing).
        if (valid && flat) {
            if (e2 && !A.ft_out)
                interface_flux<R, C, DIR, TP, NL, true>(A, x0, l0, sA, t, p, line, true, true);
            else
                flat_projection<R, C, DIR, TP, NL>(A, x0, l0, sA, t, p, line, e2);
        }
        // append the other valid interfaces, in lane order within each warp
        const unsigned need = __ballot_sync(FULL, valid && !flat);
        if (need) {
            int base = 0;
            if (lane == 0) base = atomicAdd(&t.nlist(), __popc(need));
            base = __shfl_sync(FULL, base, 0);
            if ((need >> lane) & 1u) t.list()[base + __popc(need & ((1u << lane) - 1u))] = line * TP + p;
        }
    }
    __syncthreads();
    {
        // Whole warps of 32 interfaces each; a last, partly filled warp of at
        // most LONG_TAIL interfaces is evaluated field-parallel instead (four
        // lanes per interface, one field each, eight interfaces per warp):
        // the FP64 pipe is charged per warp instruction, and one field costs
        // about a third of a whole interface, so a few interfaces -- the
        // typical count of a tile crossing a front -- take a third of the
        // pipe time and of the latency.
        const int n = t.nlist();
        int nip = n;
        constexpr int NWARP = NT / 32;
        if constexpr (LM == LONG_INLINE) {
            for (int base = tid & ~31; base < n; base += NT) {
                const int j = base + (tid & 31);
                const bool act = j < n;
                const int e = t.list()[act ? j : base];
                interface_flux<R, C, DIR, TP, NL, false>(A, x0, l0, sA, t, e % TP, e / TP, act,
                                                        false);
            }
            nip = -1;  // done
        } else if constexpr (C == 4) {
            // a list that fits eight interfaces per warp (a tile crossing a
            // front) is evaluated field-parallel as a whole: its FP64 work is
            // spread over every warp, and so over every sub-partition's FP64
            // unit, instead of sitting in one or two warps
            const int r = n & 31;
            if (LM == LONG_FIELDS && n <= 8 * NWARP)
                nip = 0;
            else if (r > 0 && r <= LONG_TAIL)
                nip = n - r;
        }
        for (int base = tid & ~31; base < nip; base += NT) {
            const int j = base + (tid & 31);
            const bool act = j < nip;
            const int e = t.list()[act ? j : base];
            long_path<R, C, DIR, TP, NL>(A, x0, l0, sA, t, e % TP, e / TP, act);
        }
        if (C == 4 && nip >= 0 && nip < n) {
            // the warps without a whole-warp chunk take the tail's chunks
            const int w0 = (nip >> 5) % NWARP, nchunk = (n - nip + 7) >> 3;
            for (int c = ((tid >> 5) - w0 + NWARP) % NWARP; c < nchunk; c += NWARP) {
                const int j = nip + c * 8 + (lane >> 2);
                const bool act = j < n;
                const int e = t.list()[act ? j : nip];
                long_tail<R, C, DIR, TP, NL>(A, x0, l0, sA, t, e % TP, e / TP, act, lane & 3);
            }
        }
    }
    __syncthreads();
    }  // !constant

    const int p = (DIR == 0) ? tid % TP : tid / NL;
    const int line = (DIR == 0) ? tid / TP : tid % NL;
    const long long Lg = l0 + line;

    // ---- flux difference and epilogue for the TP-1 cells of the tile
    unsigned long long ws[3] = {0, 0, 0};
    if (p < TP - 1 && Lg < nlines) {
        const long long i = x0 + p;
        if (i < nlen) {
            const long long gi = (DIR == 0) ? Lg * nx + i : i * nx + Lg;
            const int sc = p + g;  // staged index of cell i
            double o[C];
            auto cell = [&](auto M, auto P, auto Z) {
#pragma unroll
                for (int q = 0; q < C; ++q) {
                    // map line component back to the state component
                    const int qs = (q == 1) ? QN : ((C == 4 && q == 2) ? QT : q);
                    double dF = 0.0;  // constant tile: exactly zero
                    if constexpr (!decltype(Z)::value) dF = t.Fh(q, line, p + 1) - t.Fh(q, line, p);
                    double S = 0.0;
                    if constexpr (EXT) {
                        // body force (0, rho g_n, rho g_t, m_n g_n + m_t g_t)
                        const double rho = t.U(0, line, sc);
                        if (q == 1) S = __dmul_rn(rho, A.g_n);
                        if (C == 4 && q == 2) S = __dmul_rn(rho, A.g_t);
                        if (q == C - 1)
                            S = (C == 4) ? __dadd_rn(__dmul_rn(t.U(1, line, sc), A.g_n),
                                                     __dmul_rn(t.U(2, line, sc), A.g_t))
                                         : __dmul_rn(t.U(1, line, sc), A.g_n);
                    }
                    o[q] = epilogue_form<decltype(M)::value, decltype(P)::value != 0,
                                         decltype(Z)::value != 0>(
                        A.epi, qs * ncell + gi, dF, A.inv_h, t.U(q, line, sc), EXT && A.src != 0,
                        S);
                }
            };
            auto tile_form = [&](auto M, auto P) {
                if (constant)
                    cell(M, P, IC<1>{});
                else
                    cell(M, P, IC<0>{});
            };
            // the 2D row sweep always stores its partial right-hand side
            // (its launchers refuse any other epilogue)
            if constexpr (DIR == 0 && C == 4)
                tile_form(IC<EPI_STORE>{}, IC<0>{});
            else
                with_epilogue_form(A.epi, tile_form);
            if (C == 3 && A.alpha_next) {
                double w3[3];
                wave_speeds3(o[0], o[1], o[2], A.gm1, A.gamma, w3, A.status);
#pragma unroll
                for (int k3 = 0; k3 < 3; ++k3) ws[k3] = __double_as_longlong(w3[k3]);
            }
        }
    }
    if (C == 3 && A.alpha_next) {
        // CTA maximum of the new state's wave speeds -> the next stage's alpha
#pragma unroll
        for (int k3 = 0; k3 < 3; ++k3) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                unsigned long long w = __shfl_xor_sync(FULL, ws[k3], o);
                ws[k3] = ws[k3] > w ? ws[k3] : w;
            }
        }
        if ((tid & 31) == 0)
            for (int k3 = 0; k3 < 3; ++k3) t.red()[tid >> 5][k3] = ws[k3];
        __syncthreads();
        if (tid < 3) {
            unsigned long long m = 0;
            for (int wi = 0; wi < NT / 32; ++wi) m = m > t.red()[wi][tid] ? m : t.red()[wi][tid];
            atomicMax((unsigned long long *)(A.alpha_next + tid), m);
        }
    }
}

// Resident sweep threads per SM: 1280 (40 warps, five 256-thread CTAs,
// which is also what the shared memory of the 2D tiles allows) caps the
// registers at 48.  The flat interfaces, most of a typical grid, need few
// registers and hide the FP64 latency with more warps: measured on the
// 4096^2 Riemann workload, 16 -> 24 -> 32 -> 40 warps gave 3.07 -> 3.40 ->
// 3.57 -> 3.70 G cell-updates/s at order 9 (orders 5-17 alike).  The long
// path spills to local memory (L1) and keeps its speed on the smooth vortex
// (within 0.5 %).
constexpr int SWEEP_THREADS_PER_SM = SWEEP_HIGH_THREADS_PER_SM;
// The low-occupancy instances (MINB = SWEEP_LOW_CTAS CTAs of 256 threads per
// SM, 128 registers per thread) keep the long path's windows in registers
// without spilling; they serve launches of few tiles, whose speed is set by
// the latency of one tile rather than by the number of warps in flight.
constexpr int SWEEP_LOW_CTAS = 2;

// The 2D row sweeps compile only the plain-store epilogue: their partial
// right-hand side goes to a buffer that the column sweep adds.  Their
// launchers refuse any other.
inline bool row_epilogue_ok(const SweepArgs &a)
{
    return a.epi.mode == EPI_STORE && a.epi.Dprev == nullptr;
}

template <int R, int C, int DIR, int TP, int NL, bool EXT = false,
          int MINB = SWEEP_THREADS_PER_SM / (TP * NL), int LM = LongForm<DIR>::value>
__global__ void __launch_bounds__(TP *NL, MINB) k_sweep(SweepArgs A)
{
    constexpr int g = (R + 1) / 2, W = 2 * g - 1, T = Tab<R>::T;
    __shared__ SweepSmem<R, C, TP, NL> sm;
    __shared__ double sA[T * W];
    load_a_table<R>(sA, threadIdx.x, TP * NL);
    const long long x0 = (long long)((DIR == 0) ? blockIdx.x : blockIdx.y) * (TP - 1);
    const long long l0 = (long long)((DIR == 0) ? blockIdx.y : blockIdx.x) * NL;
    sweep_tile<R, C, DIR, TP, NL, EXT, LM>(A, x0, l0, sA, ClassicTile<R, C, DIR, TP, NL>{sm});
}

// ---------------------------------------------------------------------------
// Batched 1D Euler: one persistent launch per RK stage over a table of
// (problem, first interface) tiles of many independent problems of uneven
// size.  Each tile runs the same interface arithmetic as the single-problem
// sweep, so results are bitwise those of one problem at a time.
// ---------------------------------------------------------------------------
template <int R, int TP>
__global__ void __launch_bounds__(TP) k_batch_stage(BatchArgs B)
{
    constexpr int g = (R + 1) / 2, W = 2 * g - 1, T = Tab<R>::T;
    __shared__ SweepSmem<R, 3, TP, 1> sm;
    __shared__ double sA[T * W];
    load_a_table<R>(sA, threadIdx.x, TP);
    // work items of tiles_per_item consecutive tiles (each thread evaluates
    // that many interfaces per item), strided over the persistent grid
    const int k = B.tiles_per_item;
    const long long nitem = (B.ntiles + k - 1) / k;
    for (long long t = 0, w = blockIdx.x, j = 0; w < nitem;) {
        t = w * k + j;
        if (++j == k) {
            j = 0;
            w += gridDim.x;
        }
        if (t >= B.ntiles) continue;
        __syncthreads();  // the previous tile is done with shared memory
        const BatchTile tl = B.tiles[t];
        const int pr = tl.prob;
        const long long base = B.base[pr];
        SweepArgs A;
        A.U = B.Us + base;
        A.nx = B.n[pr];
        A.ny = 1;
        A.bc = B.bc;
        A.gm1 = B.gm1;
        A.inv_gm1 = B.inv_gm1;
        A.gamma = B.gamma;
        A.inv_h = B.inv_dx[pr];
        A.alpha = B.alpha + 3 * pr;
        A.alpha_next = B.alpha_next ? B.alpha_next + 3 * pr : nullptr;
        A.sel = nullptr;
        A.sel_in = nullptr;
        A.ft_out = nullptr;
        A.status = B.status;
        A.epi.mode = EPI_STAGE;
        A.epi.c0 = B.c0;
        A.epi.c1 = B.c1;
        A.epi.dt_dev = B.dt + pr;
        A.epi.Un = B.Un + base;
        A.epi.Dprev = nullptr;
        A.epi.out = B.out + base;
        sweep_tile<R, 3, 0, TP, 1>(A, tl.x0, 0, sA, ClassicTile<R, 3, 0, TP, 1>{sm});
    }
}

}  // namespace enomr
