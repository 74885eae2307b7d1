// enomr_vjp.cuh -- vector-Jacobian product of the ENO-MR right-hand side with
// the forward pass's discrete choices frozen (selected stencil or minmod
// branch at every interface, field and side; the cell attaining each
// per-line alpha).  With those frozen the RHS is a smooth function of U and
// this is its exact transpose Jacobian applied to a cotangent.
//
// Per tile, every interface re-runs the forward computation of
// enomr_kernels.cuh (same operations, same selections) and then walks it
// backwards: flux difference -> back-projection -> reconstruction on the
// chosen stencil -> Lax-Friedrichs split -> characteristic projection of
// U and F -> Roe average -> primitive variables.  Contributions to the
// window cells are written per interface to shared memory and gathered per
// cell (field by field), so no atomics are used inside a tile; cells shared
// with a neighbouring tile are added to the output with atomicAdd.  The
// derivative with respect to alpha is summed per line and applied to the
// frozen argmax cell by k_alpha_vjp.
#pragma once

#include "enomr_sweep.cuh"

namespace enomr {

// Reverse of the primitives (sqrt(rho), u_n, u_t, H) of one cell with respect
// to its conserved state (rho, m_n, m_t, E): adds to ub[].
template <int C>
__device__ __forceinline__ void prim_bar(double rho, double un, double ut, double H, double sq,
                                         double sq_b, double un_b, double ut_b, double H_b,
                                         double gm1, double gamma, double *ub)
{
    const double ir = 1.0 / rho;
    const double q2 = (C == 4) ? un * un + ut * ut : un * un;
    ub[0] += sq_b * 0.5 / sq - (un_b * un + ((C == 4) ? ut_b * ut : 0.0)) * ir +
             H_b * (0.5 * gm1 * q2 - H) * ir;
    ub[1] += (un_b - H_b * gm1 * un) * ir;
    if (C == 4) ub[2] += (ut_b - H_b * gm1 * ut) * ir;
    ub[C - 1] += H_b * gamma * ir;
}

template <int R, int C, int DIR, int TP, int NL>
__global__ void __launch_bounds__(TP *NL) k_sweep_vjp(VjpArgs A)
{
    constexpr int g = (R + 1) / 2, W = 2 * g - 1, S = TP + 2 * g - 1, T = Tab<R>::T;
    constexpr int NT = TP * NL;
    constexpr int QN = (DIR == 0) ? 1 : 2;
    constexpr int QT = (DIR == 0) ? 2 : 1;
    constexpr int CPT = (NL * S + NT - 1) / NT;  // staged cells per thread in the gather
    __shared__ double sU[C][NL][S];
    __shared__ double sF[C][NL][S];
    __shared__ double sP[4][NL][S];  // sqrt(rho), u_n, u_t, H
    __shared__ double sLb[C][NL][TP + 1];
    __shared__ double sWB[NL][TP][2 * g];
    __shared__ double sQB[NL][TP][2 * g];
    __shared__ double sRow[NL][TP][3];
    __shared__ double sRowA[NL][TP][4];
    __shared__ double sRoeB[NL][TP][2][C];
    __shared__ double sA[T * W];

    const long long nx = A.nx, ny = A.ny, ncell = nx * ny;
    const long long nlen = (DIR == 0) ? nx : ny;
    const long long nlines = (DIR == 0) ? ny : nx;
    const long long x0 = (long long)((DIR == 0) ? blockIdx.x : blockIdx.y) * (TP - 1);
    const long long l0 = (long long)((DIR == 0) ? blockIdx.y : blockIdx.x) * NL;
    const int tid = threadIdx.x;
    load_a_table<R>(sA, tid, NT);

    // ---- stage cells (as the forward sweep) and the cotangent of L
    for (int idx = tid; idx < NL * S; idx += NT) {
        int line, s;
        if (DIR == 0) {
            line = idx / S;
            s = idx - line * S;
        } else {
            s = idx / NL;
            line = idx - s * NL;
        }
        long long L = l0 + line;
        if (L >= nlines) L = nlines - 1;
        const long long cell = ghost(x0 - g + s, nlen, A.bc);
        const long long gi = (DIR == 0) ? L * nx + cell : cell * nx + L;
        double u[C];
#pragma unroll
        for (int q = 0; q < C; ++q) u[q] = A.U[q * ncell + gi];
        const StagedCell<C> sc_ = stage_cell<C>(u[0], u[QN], (C == 4) ? u[QT] : 0.0, u[C - 1], A.gm1);
        sU[0][line][s] = u[0];
        sU[1][line][s] = u[QN];
        if (C == 4) sU[2][line][s] = u[QT];
        sU[C - 1][line][s] = u[C - 1];
#pragma unroll
        for (int q = 0; q < C; ++q) sF[q][line][s] = sc_.F[q];
        sP[0][line][s] = sc_.sq;
        sP[1][line][s] = sc_.un;
        sP[2][line][s] = sc_.ut;
        sP[3][line][s] = sc_.H;
    }
    for (int idx = tid; idx < NL * (TP + 1); idx += NT) {
        const int line = idx / (TP + 1), j = idx - line * (TP + 1);
        const long long L = l0 + line;
        const long long cell = x0 - 1 + j;  // cells x0-1 .. x0+TP-1
#pragma unroll
        for (int q = 0; q < C; ++q) {
            double v = 0.0;
            if (L < nlines && cell >= 0 && cell < nlen) {
                const int qs = (q == 1) ? QN : ((C == 4 && q == 2) ? QT : q);
                const long long gi = (DIR == 0) ? L * nx + cell : cell * nx + L;
                v = A.Lbar[qs * ncell + gi];
            }
            sLb[q][line][j] = v;
        }
    }
    __syncthreads();

    int p, line;
    if (DIR == 0) {
        p = tid % TP;
        line = tid / TP;
    } else {
        line = tid % NL;
        p = tid / NL;
    }
    const long long Lg = l0 + line;
    const long long k = x0 + p;  // interface x_{k-1/2}
    const bool valid = (Lg < nlines) && (k <= nlen);
    // each interface is owned by one tile (overlapping tiles share one)
    const bool owned = valid && (p < TP - 1 || k == nlen);
    const int sl = p + g - 1, sr = p + g;

    // cotangent of the interface flux: F_k enters L_{k-1} (-1/h) and L_k (+1/h)
    const double scale = A.scale_dev ? A.scale * *A.scale_dev : A.scale;
    double Fb[C];
#pragma unroll
    for (int q = 0; q < C; ++q)
        Fb[q] = owned ? scale * (sLb[q][line][p + 1] - sLb[q][line][p]) * A.inv_h : 0.0;

    // ---- forward: Roe average and scaled eigenvectors (as the forward sweep)
    bool eqLR = true;
#pragma unroll
    for (int q = 0; q < C; ++q)
        eqLR = eqLR && (__double_as_longlong(sU[q][line][sl]) == __double_as_longlong(sU[q][line][sr]));
    const double qL = sP[0][line][sl], qR = sP[0][line][sr];
    const double rs = 1.0 / (qL + qR);
    const RoeFace rf = roe_face(eqLR, qL, sP[1][line][sl], sP[2][line][sl], sP[3][line][sl], qR,
                                sP[1][line][sr], sP[2][line][sr], sP[3][line][sr], C == 4,
                                A.gm1, A.inv_gm1);
    const double uh = rf.uh, vh = rf.vh, Hh = rf.Hh, hq = rf.hq, c2 = rf.c2, ic = rf.ic,
                 cs = rf.cs, kap = rf.kap, c2g = rf.c2g, b1 = rf.b1;
    const double *al = A.alpha + 3 * (Lg < nlines ? Lg : nlines - 1);
    const double a_m = al[0], a_0 = al[1], a_p = al[2];

    // ---- reverse of the back-projection, part independent of the fields
    const double FbE = Fb[C - 1];
    const double F0b = Fb[0] + Fb[1] * uh + ((C == 4) ? Fb[2] * vh : 0.0);
    const double acc_s_b = F0b + FbE * Hh;
    const double acc_d_b = (Fb[1] + FbE * uh) * cs;
    const double ph1_b = F0b + FbE * hq;
    const double ph2_b = (C == 4) ? Fb[2] + FbE * vh : 0.0;
    const double ph0_b = acc_s_b - acc_d_b, pha_b = acc_s_b + acc_d_b;

    double ftv[C];
    double hq_b = 0.0, uh_b = 0.0, vh_b = 0.0, kap_b = 0.0, c2g_b = 0.0;
    double ab[3] = {0.0, 0.0, 0.0};
    // per staged cell: accumulated U and F cotangents (this thread's cells)
    double cUb[CPT][C], cFb[CPT][C];
#pragma unroll
    for (int c = 0; c < CPT; ++c)
#pragma unroll
        for (int q = 0; q < C; ++q) cUb[c][q] = cFb[c][q] = 0.0;

#pragma unroll 1
    for (int f = 0; f < C; ++f) {
        const bool shear = (C == 4 && f == 2);
        double l0c, l1c, alpha;
        int aidx;
        if (shear) {
            l0c = -vh;
            l1c = 0.0;
            alpha = a_0;
            aidx = 1;
        } else if (f == 0) {
            l0c = fma(uh, kap, hq);
            l1c = -(uh + kap);
            alpha = a_m;
            aidx = 0;
        } else if (f == C - 1) {
            l0c = fma(-uh, kap, hq);
            l1c = -(uh - kap);
            alpha = a_p;
            aidx = 2;
        } else {
            l0c = hq - c2g;
            l1c = -uh;
            alpha = a_0;
            aidx = 1;
        }
        auto project_w = [&](int s) {
            if (shear) return fma(l0c, sU[0][line][s], sU[2][line][s]);
            double w = sU[C - 1][line][s];
            if (C == 4) w = fma(-vh, sU[2][line][s], w);
            w = fma(l1c, sU[1][line][s], w);
            return fma(l0c, sU[0][line][s], w);
        };
        auto project_q = [&](int s) {
            if (shear) return fma(l0c, sF[0][line][s], sF[2][line][s]);
            double q = sF[C - 1][line][s];
            if (C == 4) q = fma(-vh, sF[2][line][s], q);
            q = fma(l1c, sF[1][line][s], q);
            return fma(l0c, sF[0][line][s], q);
        };
        // forward: frozen selection and value (given, or recomputed)
        int selp, selm;
        if (A.sel_in) {
            const long long NI = nlen + 1;
            const long long kc = k <= nlen ? k : nlen;
            const long long lc = Lg < nlines ? Lg : nlines - 1;
            selp = A.sel_in[((0 * C + f) * nlines + lc) * NI + kc];
            selm = A.sel_in[((1 * C + f) * nlines + lc) * NI + kc];
            ftv[f] = A.ft_in[(f * nlines + lc) * NI + kc];
        } else {
            double vp[W], vm[W];
#pragma unroll
            for (int j = 0; j < 2 * g; ++j) {
                const double w = project_w(p + j), q = project_q(p + j);
                if (j <= 2 * g - 2) vp[j] = fma(alpha, w, q);
                if (j >= 1) vm[2 * g - 1 - j] = fma(-alpha, w, q);
            }
            const double fp = mr_value<R>(vp, sA, valid, selp);
            const double fm = mr_value<R>(vm, sA, valid, selm);
            ftv[f] = fp + fm;
        }
        // cotangent of this field's f^+ + f^-
        double ftb;
        if (f == 0) ftb = 0.25 * b1 * ph0_b;
        else if (f == C - 1) ftb = 0.25 * b1 * pha_b;
        else if (shear) ftb = 0.5 * ph2_b;
        else ftb = -0.5 * b1 * ph1_b;
        // effective reconstruction weights of the frozen choice, times ftb
        constexpr int c0 = g - 1;
        double wp[W], wm[W];
#pragma unroll
        for (int j = 0; j < W; ++j) {
            wp[j] = (selp < T) ? sA[selp * W + j] * ftb : 0.0;
            wm[j] = (selm < T) ? sA[selm * W + j] * ftb : 0.0;
        }
        if (selp == T) { wp[c0] = 0.5 * ftb; wp[c0 + 1] = 0.5 * ftb; }
        if (selp == T + 1) { wp[c0] = 1.5 * ftb; wp[c0 - 1] = -0.5 * ftb; }
        if (selp == T + 2) wp[c0] = ftb;
        if (selm == T) { wm[c0] = 0.5 * ftb; wm[c0 + 1] = 0.5 * ftb; }
        if (selm == T + 1) { wm[c0] = 1.5 * ftb; wm[c0 - 1] = -0.5 * ftb; }
        if (selm == T + 2) wm[c0] = ftb;
        // reverse of split and projection, per window cell.  With d = P - M
        // the cotangents are w_bar = alpha d and q_bar = P + M; the sums
        // S[q] = sum_j d_j U_j[q] give both the U part of the row-coefficient
        // cotangents (alpha S) and the alpha cotangent sum_j d_j w_j = l . S.
        double S0 = 0.0, S1 = 0.0, ST = 0.0, SE = 0.0, Q0 = 0.0, Q1 = 0.0, QT = 0.0;
#pragma unroll
        for (int j = 0; j < 2 * g; ++j) {
            const int s = p + j;
            const double P = (j <= 2 * g - 2) ? wp[j] : 0.0;
            const double M = (j >= 1) ? wm[2 * g - 1 - j] : 0.0;
            const double qb = P + M, d = P - M;
            sWB[line][p][j] = d;  // alpha is folded into the gather's row
            sQB[line][p][j] = qb;
            S0 = fma(d, sU[0][line][s], S0);
            Q0 = fma(qb, sF[0][line][s], Q0);
            if (C == 4) ST = fma(d, sU[2][line][s], ST);
            if (!shear) {
                S1 = fma(d, sU[1][line][s], S1);
                SE = fma(d, sU[C - 1][line][s], SE);
                Q1 = fma(qb, sF[1][line][s], Q1);
                if (C == 4) QT = fma(qb, sF[2][line][s], QT);
            }
        }
        double l0b, l1b = 0.0, ltb = 0.0;
        l0b = fma(alpha, S0, Q0);
        if (shear) {
            ab[aidx] += fma(l0c, S0, ST);
        } else {
            l1b = fma(alpha, S1, Q1);
            if (C == 4) ltb = fma(alpha, ST, QT);
            double a = fma(l0c, S0, SE);
            a = fma(l1c, S1, a);
            if (C == 4) a = fma(-vh, ST, a);
            ab[aidx] += a;
        }
        // gather rows: U part scaled by alpha (it multiplies d), F part not
        sRow[line][p][0] = l0c;
        sRow[line][p][1] = l1c;
        sRow[line][p][2] = (C == 4) ? -vh : 0.0;
        sRowA[line][p][0] = alpha * l0c;
        sRowA[line][p][1] = alpha * l1c;
        sRowA[line][p][2] = (C == 4) ? -alpha * vh : 0.0;
        sRowA[line][p][3] = alpha;
        // row coefficients -> Roe scalars
        if (shear) {
            vh_b -= l0b;
        } else if (f == 0) {
            hq_b += l0b;
            uh_b += l0b * kap - l1b;
            kap_b += l0b * uh - l1b;
            vh_b -= ltb;
        } else if (f == C - 1) {
            hq_b += l0b;
            uh_b -= l0b * kap + l1b;
            kap_b += l1b - l0b * uh;
            vh_b -= ltb;
        } else {
            hq_b += l0b;
            c2g_b -= l0b;
            uh_b -= l1b;
            vh_b -= ltb;
        }
        __syncthreads();
        // gather: staged cell s receives wb l and qb l from interfaces p' = s - j
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const int idx = tid + c * NT;
            if (idx < NL * S) {
                int gl, s;
                if (DIR == 0) {
                    gl = idx / S;
                    s = idx - gl * S;
                } else {
                    s = idx / NL;
                    gl = idx - s * NL;
                }
                for (int j = 0; j < 2 * g; ++j) {
                    const int pp = s - j;
                    if (pp < 0 || pp >= TP) continue;
                    const double d = sWB[gl][pp][j], qb = sQB[gl][pp][j];
                    const double r0 = sRow[gl][pp][0], a0 = sRowA[gl][pp][0];
                    const double al_ = sRowA[gl][pp][3];
                    if (shear) {
                        cUb[c][0] += d * a0;
                        cUb[c][2] += d * al_;
                        cFb[c][0] += qb * r0;
                        cFb[c][2] += qb;
                    } else {
                        const double r1 = sRow[gl][pp][1], rt = sRow[gl][pp][2];
                        const double a1 = sRowA[gl][pp][1], at = sRowA[gl][pp][2];
                        cUb[c][0] += d * a0;
                        cUb[c][1] += d * a1;
                        cUb[c][C - 1] += d * al_;
                        cFb[c][0] += qb * r0;
                        cFb[c][1] += qb * r1;
                        cFb[c][C - 1] += qb;
                        if (C == 4) {
                            cUb[c][2] += d * at;
                            cFb[c][2] += qb * rt;
                        }
                    }
                }
            }
        }
        __syncthreads();
    }

    // ---- reverse of the back-projection terms that need the field values
    {
        const double ph0 = 0.25 * b1 * ftv[0], pha = 0.25 * b1 * ftv[C - 1];
        const double ph1 = -0.5 * b1 * ftv[1], ph2 = (C == 4) ? 0.5 * ftv[2] : 0.0;
        const double acc_s = ph0 + pha, acc_d = pha - ph0;
        const double F0 = acc_s + ph1;
        double Hh_b = FbE * acc_s;
        uh_b += FbE * cs * acc_d + Fb[1] * F0;
        double cs_b = (FbE * uh + Fb[1]) * acc_d;
        hq_b += FbE * ph1;
        if (C == 4) vh_b += FbE * ph2 + Fb[2] * F0;
        const double b1_b = 0.25 * ftv[0] * ph0_b + 0.25 * ftv[C - 1] * pha_b - 0.5 * ftv[1] * ph1_b;
        // Roe scalars
        double ic_b = b1_b * 2.0 * A.gm1 * ic;
        double c2_b = c2g_b * A.inv_gm1;
        cs_b += kap_b * A.inv_gm1;
        c2_b += cs_b * ic;
        ic_b += cs_b * c2;
        c2_b += -0.5 * ic_b * ic * ic * ic;
        Hh_b += A.gm1 * c2_b;
        hq_b -= A.gm1 * c2_b;
        uh_b += hq_b * uh;
        vh_b += hq_b * vh;
        // Roe average (weights sqrt(rho))
        const double WL = qL * rs, WR = qR * rs;
        const double uL = sP[1][line][sl], uR = sP[1][line][sr];
        const double vL = sP[2][line][sl], vR = sP[2][line][sr];
        const double HL = sP[3][line][sl], HR = sP[3][line][sr];
        const double qL_b = (uh_b * (uL - uh) + ((C == 4) ? vh_b * (vL - vh) : 0.0) + Hh_b * (HL - Hh)) * rs;
        const double qR_b = (uh_b * (uR - uh) + ((C == 4) ? vh_b * (vR - vh) : 0.0) + Hh_b * (HR - Hh)) * rs;
        double ubL[C], ubR[C];
#pragma unroll
        for (int q = 0; q < C; ++q) ubL[q] = ubR[q] = 0.0;
        prim_bar<C>(sU[0][line][sl], uL, vL, HL, qL, qL_b, uh_b * WL, vh_b * WL, Hh_b * WL, A.gm1,
                    A.gamma, ubL);
        prim_bar<C>(sU[0][line][sr], uR, vR, HR, qR, qR_b, uh_b * WR, vh_b * WR, Hh_b * WR, A.gm1,
                    A.gamma, ubR);
#pragma unroll
        for (int q = 0; q < C; ++q) {
            sRoeB[line][p][0][q] = owned ? ubL[q] : 0.0;
            sRoeB[line][p][1][q] = owned ? ubR[q] : 0.0;
        }
    }
    // alpha cotangents of this line: warp sum over lanes of the same line
    // (x sweeps: a warp lies in one line; y sweeps: lines interleave with period NL)
    constexpr int OMIN = (DIR == 0) ? 1 : NL;
#pragma unroll
    for (int a3 = 0; a3 < 3; ++a3) {
        double v = owned ? ab[a3] : 0.0;
        for (int o = 16; o >= OMIN; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
        ab[a3] = v;
    }
    if ((tid & 31) < OMIN && Lg < nlines) {
        for (int a3 = 0; a3 < 3; ++a3)
            if (ab[a3] != 0.0) atomicAdd(A.alpha_bar + 3 * Lg + a3, ab[a3]);
    }
    __syncthreads();

    // ---- per staged cell: Roe contributions, flux Jacobian transpose, output
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
        const int idx = tid + c * NT;
        if (idx >= NL * S) continue;
        int gl, s;
        if (DIR == 0) {
            gl = idx / S;
            s = idx - gl * S;
        } else {
            s = idx / NL;
            gl = idx - s * NL;
        }
        const long long L = l0 + gl;
        if (L >= nlines) continue;
        double ub[C];
#pragma unroll
        for (int q = 0; q < C; ++q) ub[q] = cUb[c][q];
        const int pl = s - g + 1, pr = s - g;  // interfaces with s as left / right cell
        if (pl >= 0 && pl < TP)
#pragma unroll
            for (int q = 0; q < C; ++q) ub[q] += sRoeB[gl][pl][0][q];
        if (pr >= 0 && pr < TP)
#pragma unroll
            for (int q = 0; q < C; ++q) ub[q] += sRoeB[gl][pr][1][q];
        // F = (m, m u + p, m_t u, (E + p) u), p = (gamma-1)(E - (m^2 + m_t^2)/(2 rho))
        const double rho = sU[0][gl][s], m = sU[1][gl][s], E = sU[C - 1][gl][s];
        const double mt = (C == 4) ? sU[2][gl][s] : 0.0;
        const double u = sP[1][gl][s], v = sP[2][gl][s];
        const double pr_ = rho * sP[3][gl][s] - E;  // p = rho H - E
        const double a0 = cFb[c][0], a1 = cFb[c][1], a3v = cFb[c][C - 1];
        const double a2 = (C == 4) ? cFb[c][2] : 0.0;
        const double u_b = a1 * m + a2 * mt + a3v * (E + pr_);
        const double p_b = a1 + a3v * u;
        const double ir = 1.0 / rho;
        ub[0] += -u_b * u * ir + p_b * 0.5 * A.gm1 * (u * u + v * v);
        ub[1] += a0 + a1 * u + u_b * ir - p_b * A.gm1 * u;
        if (C == 4) ub[2] += a2 * u - p_b * A.gm1 * v;
        ub[C - 1] += a3v * u + p_b * A.gm1;
        const long long cell = ghost(x0 - g + s, nlen, A.bc);
        const long long gi = (DIR == 0) ? L * nx + cell : cell * nx + L;
#pragma unroll
        for (int q = 0; q < C; ++q) {
            const int qs = (q == 1) ? QN : ((C == 4 && q == 2) ? QT : q);
            if (ub[q] != 0.0) atomicAdd(A.Ubar + qs * ncell + gi, ub[q]);
        }
    }
}

// Scalar advection: F_k = MR(a u) on the upwind side, frozen choice; the
// transpose scatters a * weight * F_bar_k to the window cells.
template <int R, int TP>
__global__ void __launch_bounds__(TP) k_advection_vjp(AdvArgs A, const double *Lbar, double *Ubar,
                                                     double factor, const double *factor_dev)
{
    const double scale = factor_dev ? factor * *factor_dev : factor;
    constexpr int g = (R + 1) / 2, W = 2 * g - 1, S = TP + 2 * g - 1, T = Tab<R>::T;
    __shared__ double sf[S];
    __shared__ double sA[T * W];
    const int p = threadIdx.x;
    const long long x0 = (long long)blockIdx.x * (TP - 1);
    load_a_table<R>(sA, p, TP);
    for (int s = p; s < S; s += TP) sf[s] = A.a * A.U[ghost(x0 - g + s, A.n, A.bc)];
    __syncthreads();
    const long long k = x0 + p;
    const bool valid = k <= A.n;
    const bool owned = valid && (p < TP - 1 || k == A.n);
    double v[W];
    const bool plus = A.a >= 0.0;
#pragma unroll
    for (int j = 0; j < W; ++j) v[j] = plus ? sf[p + j] : sf[p + 2 * g - 1 - j];
    int sel;
    mr_value<R>(v, sA, valid, sel);
    if (!owned) return;
    const double Lk = (k < A.n) ? Lbar[k] : 0.0;
    const double Lk1 = (k >= 1) ? Lbar[k - 1] : 0.0;
    const double fb = scale * (Lk - Lk1) * A.inv_h * A.a;
    constexpr int c0 = g - 1;
    for (int j = 0; j < W; ++j) {
        double w = (sel < T) ? sA[sel * W + j] : 0.0;
        if (sel == T) w = (j == c0 || j == c0 + 1) ? 0.5 : 0.0;
        if (sel == T + 1) w = (j == c0) ? 1.5 : ((j == c0 - 1) ? -0.5 : 0.0);
        if (sel == T + 2) w = (j == c0) ? 1.0 : 0.0;
        if (w == 0.0) continue;
        const int s = plus ? p + j : p + 2 * g - 1 - j;
        atomicAdd(Ubar + ghost(x0 - g + s, A.n, A.bc), w * fb);
    }
}

}  // namespace enomr
