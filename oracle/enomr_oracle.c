/*
 * enomr_oracle.c -- plain, slow FP64 CPU oracle for the ENO-MR semi-discrete
 * right-hand side and its Runge-Kutta time integrators.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or generator
 * with the CUDA path.
 *
 * Written from: "An efficient class of increasingly high-order ENO schemes
 * with multi-resolution" (arXiv 2311.15504).
 *   Sec. 2.1  Eq. (1DWENOFD) conservative finite-difference form,
 *             Eq. (LF_Flux_Split) global Lax-Friedrichs splitting.
 *   Sec. 2.2  Eq. (Polynomial_Construction), Eq. (ReconstructedFlux).
 *   Sec. 2.3  Eq. (TVD3rdRK) SSP-RK3, Eq. (lSSPRK)/(lSSPRK_Coe) linear SSP-RK.
 *   Sec. 3.1  Eq. (Candidates) candidate stencils, Tables 1-2 (a_l),
 *             Tables 3-4 (b_l).
 *   Sec. 3.2  Steps 1-3: baseline indicator IS_0 (Eq. Baseline_IS),
 *             candidate indicator (Eq. CurrentIS / ISCoe), ordered test,
 *             minmod fallback.
 *   Sec. 4    Roe-averaged characteristic decomposition for Euler; 1D and
 *             2D Euler equations.
 *
 * Readings of places where the paper is silent or garbled:
 *   - Candidate list for order R = 2r-1 < 17: the entries of Eq. (Candidates)
 *     with m <= r-1 and n <= r-1, kept in the printed order.
 *   - "smaller than" is strict; equality falls through.
 *   - Only candidates with m >= 1 and n >= 1 are tested; S(0,1), S(1,0),
 *     S(0,0) are reached through the minmod rule only.
 *   - b_l are the signed binomials (-1)^(n-l) C(m+n, n-l) (Table 3 prints
 *     -3423 twice where the binomial is -3432).
 *   - f^- uses the mirror image of the f^+ formulae about x_{j+1/2}:
 *     v(l) = f^-_{j+1-l}.
 *   - minmod's "ab > 0" is evaluated as a sign test (same sign, both
 *     nonzero), which is the mathematical meaning and avoids underflow.
 *   - For systems, alpha is taken per characteristic field k as
 *     max_i |lambda_k(U_i)| over the interior cells of the line, from the
 *     cell states of the stage being evaluated.
 *   - Linear SSP-RK coefficients: alpha_{m,m-1} = (2/m) alpha_{m-1,m-2}.
 *   - Non-reflecting boundaries: zeroth-order extrapolation into the ghosts.
 *
 * Arithmetic: plain C, compiled with -ffp-contract=off; every sum runs in the
 * order written in the paper (increasing l).  L = R^{-1} is obtained by a
 * numerical Gauss-Jordan inverse, not a closed form.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENONPHYS 4

#define MAXG 9
#define MAXW (2 * MAXG - 1)
#define NCAND 29

/* ------------------------------------------------------------------------- */
/* Tables 1 and 2: a_l for f^+_{j+1/2} on the 29 stencils S_{j-m}^{j+n}, in   */
/* the order of Eq. (Candidates).  num[] runs over l = -m .. n; the value is  */
/* num/den.                                                                  */
/* ------------------------------------------------------------------------- */
typedef struct {
    int m, n;
    long den;
    long num[17];
} stencil_t;

static const stencil_t CAND[NCAND] = {
    {8, 8, 12252240L, {56, -1015, 8777, -48343, 191561, -588127, 1491041, -3409855, 8842385,
                       7481025, -2320767, 797985, -241599, 58281, -10263, 1161, -63}},
    {7, 8, 720720L, {-7, 121, -999, 5273, -20207, 61329, -162895, 477745, 477745, -162895, 61329,
                     -20207, 5273, -999, 121, -7}},
    {8, 7, 720720L, {7, -119, 961, -4919, 18013, -50783, 117385, -242975, 567835, 397665, -106839,
                     30753, -7467, 1353, -159, 9}},
    {7, 7, 360360L, {-7, 113, -867, 4229, -14881, 41175, -98965, 261395, 216350, -63930, 20154,
                     -5326, 1044, -132, 8}},
    {8, 6, 360360L, {8, -127, 953, -4507, 15149, -38905, 81215, -150445, 312875, 176310, -39906,
                     9234, -1686, 204, -12}},
    {6, 7, 360360L, {15, -230, 1681, -7874, 27161, -77944, 237371, 237371, -77944, 27161, -7874,
                     1681, -230, 15}},
    {7, 6, 360360L, {-15, 225, -1595, 7141, -22889, 57191, -122989, 288851, 192326, -47914, 12146,
                     -2414, 316, -20}},
    {6, 6, 360360L, {30, -425, 2851, -12164, 37886, -97249, 263111, 211631, -58639, 16436, -3584,
                     511, -35}},
    {7, 5, 360360L, {-35, 485, -3155, 12861, -37189, 82931, -157309, 323171, 166586, -33614, 6426,
                     -854, 56}},
    {5, 6, 27720L, {-5, 67, -428, 1772, -5653, 18107, 18107, -5653, 1772, -428, 67, -5}},
    {6, 5, 27720L, {5, -65, 397, -1528, 4247, -9613, 22727, 14147, -3178, 672, -98, 7}},
    {5, 5, 27720L, {-10, 122, -703, 2597, -7303, 20417, 15797, -4003, 947, -153, 12}},
    {6, 4, 27720L, {12, -142, 782, -2683, 6557, -12847, 25961, 11837, -2023, 287, -21}},
    {4, 5, 2520L, {2, -23, 127, -473, 1627, 1627, -473, 127, -23, 2}},
    {5, 4, 2520L, {-2, 22, -113, 367, -893, 2131, 1207, -233, 37, -3}},
    {4, 4, 2520L, {4, -41, 199, -641, 1879, 1375, -305, 55, -5}},
    {5, 3, 2520L, {-5, 49, -221, 619, -1271, 2509, 955, -125, 10}},
    {3, 4, 840L, {-3, 29, -139, 533, 533, -139, 29, -3}},
    {4, 3, 840L, {3, -27, 113, -307, 743, 365, -55, 5}},
    {3, 3, 420L, {-3, 25, -101, 319, 214, -38, 4}},
    {2, 3, 60L, {1, -8, 37, 37, -8, 1}},
    {3, 2, 60L, {-1, 7, -23, 57, 22, -2}},
    {2, 2, 60L, {2, -13, 47, 27, -3}},
    {1, 2, 12L, {-1, 7, 7, -1}},
    {2, 1, 12L, {1, -5, 13, 3}},
    {1, 1, 6L, {-1, 5, 2}},
    {0, 1, 2L, {1, 1}},
    {1, 0, 2L, {-1, 3}},
    {0, 0, 1L, {1}},
};

/* Per-order view: the tested candidates (m>=1, n>=1) in Eq. (Candidates)
 * order, restricted to m,n <= g-1, with a_l and b_l as doubles. */
typedef struct {
    int R, g, T;
    int m[NCAND], n[NCAND];
    double a[NCAND][17];
    double b[NCAND][17];
} order_t;

static order_t ORDERS[7];
static int orders_ready = 0;

static double binom(int n, int k)
{
    double c = 1.0;
    int i;
    if (k < 0 || k > n) return 0.0;
    for (i = 1; i <= k; ++i) c = c * (double)(n - k + i) / (double)i;
    return c;
}

static void build_orders(void)
{
    int oi, s, l;
    if (orders_ready) return;
    for (oi = 0; oi < 7; ++oi) {
        order_t *o = &ORDERS[oi];
        o->R = 5 + 2 * oi;
        o->g = (o->R + 1) / 2;
        o->T = 0;
        for (s = 0; s < NCAND; ++s) {
            const stencil_t *st = &CAND[s];
            if (st->m > o->g - 1 || st->n > o->g - 1) continue;
            if (st->m < 1 || st->n < 1) continue;
            o->m[o->T] = st->m;
            o->n[o->T] = st->n;
            for (l = 0; l <= st->m + st->n; ++l) {
                int ll = l - st->m; /* stencil offset */
                int k = st->n - ll;
                double c = binom(st->m + st->n, k);
                o->a[o->T][l] = (double)st->num[l] / (double)st->den;
                o->b[o->T][l] = (k % 2) ? -c : c;
            }
            o->T++;
        }
    }
    orders_ready = 1;
}

static const order_t *get_order(int R)
{
    build_orders();
    if (R < 5 || R > 17 || (R % 2) == 0) return NULL;
    return &ORDERS[(R - 5) / 2];
}

/* ------------------------------------------------------------------------- */
/* Sec. 3.2: the ENO-MR reconstruction of one value f_{j+1/2}.               */
/* v points at v(0) = f_j; v[-(g-1)] .. v[g-1] are read.                    */
/* Selection id: t in [0,T) for the t-th tested candidate; T, T+1, T+2 for   */
/* the minmod outcomes S(0,1), S(1,0), S(0,0).                               */
/* ------------------------------------------------------------------------- */
static double dabs(double x) { return x < 0 ? -x : x; }
static double dmax(double x, double y) { return x > y ? x : y; }
static double dmin(double x, double y) { return x < y ? x : y; }

static double recon(const order_t *o, int t, const double *v)
{
    int l;
    double s = 0.0;
    if (t < o->T) {
        for (l = -o->m[t]; l <= o->n[t]; ++l) s = s + o->a[t][l + o->m[t]] * v[l];
        return s;
    }
    /* Step 3.2: f = f_j + 1/2 minmod(f_{j+1}-f_j, f_j-f_{j-1}) */
    if (t == o->T) return v[0] + 0.5 * (v[1] - v[0]);
    if (t == o->T + 1) return v[0] + 0.5 * (v[0] - v[-1]);
    return v[0];
}

static double cand_is(const order_t *o, int t, const double *v)
{
    int l;
    double s = 0.0;
    for (l = -o->m[t]; l <= o->n[t]; ++l) s = s + o->b[t][l + o->m[t]] * v[l];
    return dabs(s);
}

static double baseline_is(const double *v)
{
    double isl = dmax(dabs(v[0] - v[-1]), dabs(v[0] - 2.0 * v[-1] + v[-2]));
    double isr = dmax(dabs(v[0] - v[1]), dabs(v[0] - 2.0 * v[1] + v[2]));
    return dmin(isl, isr);
}

static int minmod_choice(const order_t *o, const double *v)
{
    double a = v[1] - v[0], b = v[0] - v[-1];
    int same_sign = (a > 0 && b > 0) || (a < 0 && b < 0);
    if (!same_sign) return o->T + 2;           /* minmod = 0 -> S(0,0) */
    return dabs(a) <= dabs(b) ? o->T : o->T + 1;
}

static int select_stencil(const order_t *o, const double *v, int *ntested)
{
    int t;
    double is0 = baseline_is(v);                    /* Step 1 */
    for (t = 0; t < o->T; ++t) {                    /* Steps 2 and 3.1 */
        if (ntested) (*ntested)++;
        if (cand_is(o, t, v) < is0) return t;
    }
    return minmod_choice(o, v);                      /* Step 3.2 */
}

static double mr(const order_t *o, const double *v, int forced, int *sel, long *ntested)
{
    int t, nt = 0;
    if (forced >= 0)
        t = forced;
    else
        t = select_stencil(o, v, &nt);
    if (ntested) *ntested += nt;
    if (sel) *sel = t;
    return recon(o, t, v);
}

/* ------------------------------------------------------------------------- */
/* Exported table and single-window entry points (for the pin tests).        */
/* ------------------------------------------------------------------------- */
int orc_num_tested(int R)
{
    const order_t *o = get_order(R);
    return o ? o->T : -1;
}

/* m, n of tested candidate t; a_l and b_l for l=-m..n written to a[], b[]. */
int orc_candidate(int R, int t, int *m, int *n, double *a, double *b)
{
    const order_t *o = get_order(R);
    int l;
    if (!o || t < 0 || t >= o->T) return ORC_EINVAL;
    *m = o->m[t];
    *n = o->n[t];
    for (l = 0; l <= o->m[t] + o->n[t]; ++l) {
        a[l] = o->a[t][l];
        b[l] = o->b[t][l];
    }
    return ORC_OK;
}

/* The printed 29-entry list of Eq. (Candidates): m, n and a_l = num/den. */
int orc_paper_stencil(int s, int *m, int *n, long *den, long *num)
{
    int l;
    if (s < 0 || s >= NCAND) return ORC_EINVAL;
    *m = CAND[s].m;
    *n = CAND[s].n;
    *den = CAND[s].den;
    for (l = 0; l <= CAND[s].m + CAND[s].n; ++l) num[l] = CAND[s].num[l];
    return ORC_OK;
}

/* window w[0 .. 2g-2] with w[g-1] = f_j */
double orc_mr(int R, const double *w, int forced, int *sel)
{
    const order_t *o = get_order(R);
    if (!o) return NAN;
    return mr(o, w + (o->g - 1), forced, sel, NULL);
}

/* Diagnostics for one window: IS_0 and the indicator of every tested
 * candidate, together with the magnitudes sum |b_l v_l| and the IS_0 terms'
 * magnitude (used to judge near-ties). */
int orc_mr_indicators(int R, const double *w, double *is0, double *mag0, double *is,
                      double *mag)
{
    const order_t *o = get_order(R);
    const double *v;
    int t, l;
    if (!o) return ORC_EINVAL;
    v = w + (o->g - 1);
    *is0 = baseline_is(v);
    *mag0 = dabs(v[0]) + 2.0 * dabs(v[-1]) + dabs(v[-2]) + 2.0 * dabs(v[1]) + dabs(v[2]);
    for (t = 0; t < o->T; ++t) {
        double m = 0.0;
        is[t] = cand_is(o, t, v);
        for (l = -o->m[t]; l <= o->n[t]; ++l) m += dabs(o->b[t][l + o->m[t]] * v[l]);
        mag[t] = m;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Boundary conditions (ghost fill).  bc = 0 periodic, 1 transmissive.       */
/* ------------------------------------------------------------------------- */
static long ghost_index(long i, long N, int bc)
{
    if (bc == 0) {
        long r = i % N;
        return r < 0 ? r + N : r;
    }
    if (i < 0) return 0;
    if (i >= N) return N - 1;
    return i;
}

/* ------------------------------------------------------------------------- */
/* Scalar conservation law, f(u) = a u (linear advection).                   */
/* Eq. (1DWENOFD) with Eq. (LF_Flux_Split); alpha = |a|.                      */
/* Interface k (k = 0..N) is x_{k-1/2}, between cells k-1 and k.             */
/* sel layout: [side][interface], side 0 = f^+, 1 = f^-.                     */
/* win layout: [side][interface][2g-1].                                      */
/* ------------------------------------------------------------------------- */
/* Shared by the scalar equations: MR values of the split fluxes fp, fm
 * (given on cells -g..N+g-1, index j+g), fhat = f^+ + f^- per interface and
 * the flux difference of Eq. (1DWENOFD). */
static void scalar_mr_rhs(const order_t *o, long N, const double *fp, const double *fm, double h,
                          const uint8_t *forced, uint8_t *sel_out, double *win_out, double *rhs,
                          long *ntested_out)
{
    const int g = o->g;
    long k, j;
    long ntested = 0;
    double *fhat = (double *)malloc(sizeof(double) * (N + 1));
#pragma omp parallel for schedule(static) reduction(+ : ntested)
    for (k = 0; k <= N; ++k) {
        long i = k - 1; /* interface i+1/2 */
        double vp[MAXW], vm[MAXW];
        int l, sp, sm, fsp = -1, fsm = -1;
        for (l = -(g - 1); l <= g - 1; ++l) {
            vp[l + g - 1] = fp[i + l + g];
            vm[l + g - 1] = fm[i + 1 - l + g];
        }
        if (forced) {
            fsp = forced[k];
            fsm = forced[(N + 1) + k];
        }
        {
            double hp = mr(o, vp + g - 1, fsp, &sp, &ntested);
            double hm = mr(o, vm + g - 1, fsm, &sm, &ntested);
            fhat[k] = hp + hm;
        }
        if (sel_out) {
            sel_out[k] = (uint8_t)sp;
            sel_out[(N + 1) + k] = (uint8_t)sm;
        }
        if (win_out) {
            for (l = 0; l < 2 * g - 1; ++l) {
                win_out[k * (2 * g - 1) + l] = vp[l];
                win_out[((N + 1) + k) * (2 * g - 1) + l] = vm[l];
            }
        }
    }
    for (j = 0; j < N; ++j) rhs[j] = -(fhat[j + 1] - fhat[j]) / h;
    if (ntested_out) *ntested_out = ntested;
    free(fhat);
}

int orc_rhs_advection(long N, const double *u, double h, int R, int bc, double a,
                      const uint8_t *forced, uint8_t *sel_out, double *win_out, double *rhs,
                      long *ntested_out)
{
    const order_t *o = get_order(R);
    long j;
    int g;
    double alpha;
    double *fp, *fm;
    if (!o || N < 1 || !(h > 0)) return ORC_EINVAL;
    g = o->g;
    if (bc == 0 && N < 2 * g) return ORC_EINVAL;
    alpha = dabs(a);
    fp = (double *)malloc(sizeof(double) * (N + 2 * g));
    fm = (double *)malloc(sizeof(double) * (N + 2 * g));
    for (j = -g; j < N + g; ++j) {
        double uj = u[ghost_index(j, N, bc)];
        double f = a * uj;
        fp[j + g] = 0.5 * (f + alpha * uj);
        fm[j + g] = 0.5 * (f - alpha * uj);
    }
    scalar_mr_rhs(o, N, fp, fm, h, forced, sel_out, win_out, rhs, ntested_out);
    free(fp);
    free(fm);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Inviscid Burgers equation u_t + (u^2/2)_x = 0 (Sec. 4.2).                  */
/* f'(u) = u.  Where f' keeps one sign over the line (all u >= 0, or all      */
/* u <= 0) the flux needs no splitting (the paper's remark for its test):    */
/* f^+ = f, f^- = 0 (or f^+ = 0, f^- = f).  Otherwise the global             */
/* Lax-Friedrichs split of Eq. (LF_Flux_Split) with alpha = max |u|.          */
/* Layouts as orc_rhs_advection.                                             */
/* ------------------------------------------------------------------------- */
int orc_rhs_burgers(long N, const double *u, double h, int R, int bc, const uint8_t *forced,
                    uint8_t *sel_out, double *win_out, double *rhs, long *ntested_out)
{
    const order_t *o = get_order(R);
    long j;
    int g, mode;
    double umin, umax, alpha = 0.0;
    double *fp, *fm;
    if (!o || N < 1 || !(h > 0)) return ORC_EINVAL;
    g = o->g;
    if (bc == 0 && N < 2 * g) return ORC_EINVAL;
    umin = u[0];
    umax = u[0];
    for (j = 0; j < N; ++j) {
        if (!(u[j] == u[j])) return ORC_ENONPHYS;
        umin = u[j] < umin ? u[j] : umin;
        umax = u[j] > umax ? u[j] : umax;
        alpha = dmax(alpha, dabs(u[j]));
    }
    mode = (umin >= 0.0) ? 0 : ((umax <= 0.0) ? 1 : 2);
    fp = (double *)malloc(sizeof(double) * (N + 2 * g));
    fm = (double *)malloc(sizeof(double) * (N + 2 * g));
    for (j = -g; j < N + g; ++j) {
        double uj = u[ghost_index(j, N, bc)];
        double f = 0.5 * (uj * uj);
        if (mode == 0) {
            fp[j + g] = f;
            fm[j + g] = 0.0;
        } else if (mode == 1) {
            fp[j + g] = 0.0;
            fm[j + g] = f;
        } else {
            fp[j + g] = 0.5 * (f + alpha * uj);
            fm[j + g] = 0.5 * (f - alpha * uj);
        }
    }
    scalar_mr_rhs(o, N, fp, fm, h, forced, sel_out, win_out, rhs, ntested_out);
    free(fp);
    free(fm);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Euler equations, ideal gas.  A "line" holds c = 3 (1D: rho, m, E) or      */
/* c = 4 (2D sweep: rho, m_normal, m_tangential, E) components.              */
/* ------------------------------------------------------------------------- */
typedef struct {
    double rho, un, ut, p, c, H;
} prim_t;

static int primitive(int c, double gamma, const double *U, prim_t *P)
{
    double rho = U[0];
    double un = U[1] / rho;
    double ut = (c == 4) ? U[2] / rho : 0.0;
    double E = U[c - 1];
    double p = (gamma - 1.0) * (E - 0.5 * rho * (un * un + ut * ut));
    if (!(rho > 0) || !(p > 0) || !isfinite(E) || !isfinite(un) || !isfinite(ut))
        return ORC_ENONPHYS;
    P->rho = rho;
    P->un = un;
    P->ut = ut;
    P->p = p;
    P->c = sqrt(gamma * p / rho);
    P->H = (E + p) / rho;
    return ORC_OK;
}

/* Physical flux in the normal direction. */
static void phys_flux(int c, const double *U, const prim_t *P, double *F)
{
    F[0] = U[1];
    F[1] = U[1] * P->un + P->p;
    if (c == 4) {
        F[2] = U[2] * P->un;
        F[3] = (U[3] + P->p) * P->un;
    } else {
        F[2] = (U[2] + P->p) * P->un;
    }
}

/* Roe average at the face between UL and UR, and the right eigenvectors
 * (columns) for the fields u-c, u, [shear], u+c. */
static int roe_eigen(int c, double gamma, const double *UL, const double *UR, double Rm[4][4],
                     double *lam)
{
    prim_t L, R;
    double sL, sR, u, v, H, q2, c2, cs;
    if (primitive(c, gamma, UL, &L) || primitive(c, gamma, UR, &R)) return ORC_ENONPHYS;
    sL = sqrt(L.rho);
    sR = sqrt(R.rho);
    u = (sL * L.un + sR * R.un) / (sL + sR);
    v = (sL * L.ut + sR * R.ut) / (sL + sR);
    H = (sL * L.H + sR * R.H) / (sL + sR);
    q2 = u * u + v * v;
    c2 = (gamma - 1.0) * (H - 0.5 * q2);
    if (!(c2 > 0)) return ORC_ENONPHYS;
    cs = sqrt(c2);
    memset(Rm, 0, sizeof(double) * 16);
    if (c == 3) {
        Rm[0][0] = 1.0;         Rm[0][1] = 1.0;      Rm[0][2] = 1.0;
        Rm[1][0] = u - cs;      Rm[1][1] = u;        Rm[1][2] = u + cs;
        Rm[2][0] = H - u * cs;  Rm[2][1] = 0.5 * q2; Rm[2][2] = H + u * cs;
        lam[0] = u - cs; lam[1] = u; lam[2] = u + cs;
    } else {
        Rm[0][0] = 1.0;        Rm[0][1] = 1.0;      Rm[0][2] = 0.0; Rm[0][3] = 1.0;
        Rm[1][0] = u - cs;     Rm[1][1] = u;        Rm[1][2] = 0.0; Rm[1][3] = u + cs;
        Rm[2][0] = v;          Rm[2][1] = v;        Rm[2][2] = 1.0; Rm[2][3] = v;
        Rm[3][0] = H - u * cs; Rm[3][1] = 0.5 * q2; Rm[3][2] = v;   Rm[3][3] = H + u * cs;
        lam[0] = u - cs; lam[1] = u; lam[2] = u; lam[3] = u + cs;
    }
    return ORC_OK;
}

/* Gauss-Jordan inverse with partial pivoting of a c x c matrix. */
static int invert(int c, double A[4][4], double Ainv[4][4])
{
    double M[4][8];
    int i, j, k;
    for (i = 0; i < c; ++i)
        for (j = 0; j < 2 * c; ++j) M[i][j] = (j < c) ? A[i][j] : (j - c == i ? 1.0 : 0.0);
    for (k = 0; k < c; ++k) {
        int piv = k;
        double best = dabs(M[k][k]), f;
        for (i = k + 1; i < c; ++i)
            if (dabs(M[i][k]) > best) {
                best = dabs(M[i][k]);
                piv = i;
            }
        if (!(best > 0)) return ORC_ENONPHYS;
        if (piv != k)
            for (j = 0; j < 2 * c; ++j) {
                double t = M[k][j];
                M[k][j] = M[piv][j];
                M[piv][j] = t;
            }
        f = M[k][k];
        for (j = 0; j < 2 * c; ++j) M[k][j] = M[k][j] / f;
        for (i = 0; i < c; ++i) {
            if (i == k) continue;
            f = M[i][k];
            for (j = 0; j < 2 * c; ++j) M[i][j] = M[i][j] - f * M[k][j];
        }
    }
    for (i = 0; i < c; ++i)
        for (j = 0; j < c; ++j) Ainv[i][j] = M[i][j + c];
    return ORC_OK;
}

int orc_euler_eigen(int c, double gamma, const double *UL, const double *UR, double *Rout,
                    double *Lout, double *lam)
{
    double Rm[4][4], Lm[4][4];
    int i, j, st;
    if (c != 3 && c != 4) return ORC_EINVAL;
    st = roe_eigen(c, gamma, UL, UR, Rm, lam);
    if (st) return st;
    st = invert(c, Rm, Lm);
    if (st) return st;
    for (i = 0; i < c; ++i)
        for (j = 0; j < c; ++j) {
            Rout[i * c + j] = Rm[i][j];
            Lout[i * c + j] = Lm[i][j];
        }
    return ORC_OK;
}

/* Per-field alpha over the interior cells of a line (reading of
 * Eq. LF_Flux_Split for systems): alpha_k = max_i |lambda_k(U_i)| with
 * lambda = (u-c, u, [u], u+c).  amax (optional) receives the first cell
 * attaining each maximum. */
static int line_alpha(int c, double gamma, long N, const double *Ul /* [N][c] */, double *alpha,
                      int *amax)
{
    long i;
    int k;
    for (k = 0; k < c; ++k) {
        alpha[k] = 0.0;
        if (amax) amax[k] = 0;
    }
    for (i = 0; i < N; ++i) {
        prim_t P;
        double lam[4];
        if (primitive(c, gamma, Ul + i * c, &P)) return ORC_ENONPHYS;
        lam[0] = P.un - P.c;
        lam[1] = P.un;
        lam[2] = (c == 4) ? P.un : P.un + P.c;
        lam[3] = P.un + P.c;
        for (k = 0; k < c; ++k)
            if (dabs(lam[k]) > alpha[k]) {
                alpha[k] = dabs(lam[k]);
                if (amax) amax[k] = (int)i;
            }
    }
    return ORC_OK;
}

/* The same alpha with the maximising cells given (frozen): alpha_k =
 * |lambda_k(U_{amax[k]})|.  Used to differentiate the scheme with all its
 * discrete choices held fixed. */
static int line_alpha_frozen(int c, double gamma, const double *Ul, const int *amax,
                             double *alpha)
{
    int k;
    for (k = 0; k < c; ++k) {
        prim_t P;
        double lam;
        if (primitive(c, gamma, Ul + (long)amax[k] * c, &P)) return ORC_ENONPHYS;
        if (k == 0)
            lam = P.un - P.c;
        else if (k == c - 1)
            lam = P.un + P.c;
        else
            lam = P.un;
        alpha[k] = dabs(lam);
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Boundary sides (the 2D problems of Sec. 4.4).  A side is described by 12  */
/* doubles: kind below and above a split position along the side, the split  */
/* position s0 + rate * t, and a conserved state (rho, rho u, rho v, E) for   */
/* each part.  Kinds: 1 transmissive (copy of the nearest cell), 2 reflective */
/* (mirror image, normal momentum negated), 3 inflow (the given state).       */
/* Along-side coordinate of a line: the cell centre of the row (x sides) or  */
/* of the column (y sides), from the lower-left corner of the domain.        */
/* ------------------------------------------------------------------------- */
enum { SIDE_TRANSMISSIVE = 1, SIDE_REFLECTIVE = 2, SIDE_INFLOW = 3 };

typedef struct {
    const double *d; /* 12 doubles, or NULL: transmissive */
    double pos, t;   /* along-side coordinate of the line, time */
    int normal;      /* global component of the normal momentum (1: x, 2: y) */
} side_t;

/* Ghost cell j (< 0 or >= N) of a line of c components (line order rho,
 * m_n, [m_t], E) into G. */
static void side_ghost(const side_t *sd, int c, long j, long N, const double *Ul, double *G)
{
    int kind = SIDE_TRANSMISSIVE, q;
    const double *st = NULL;
    if (sd && sd->d) {
        const int lo = sd->pos < sd->d[2] + sd->d[3] * sd->t;
        kind = (int)(lo ? sd->d[0] : sd->d[1]);
        st = sd->d + (lo ? 4 : 8);
    }
    if (kind == SIDE_REFLECTIVE) {
        const long m = j < 0 ? -1 - j : 2 * N - 1 - j;
        for (q = 0; q < c; ++q) G[q] = Ul[m * c + q];
        G[1] = -G[1];
    } else if (kind == SIDE_INFLOW) {
        /* global (rho, m_x, m_y, E) -> line (rho, m_n, [m_t], E) */
        G[0] = st[0];
        G[1] = st[sd->normal];
        if (c == 4) G[2] = st[sd->normal == 1 ? 2 : 1];
        G[c - 1] = st[3];
    } else {
        const long m = j < 0 ? 0 : N - 1;
        for (q = 0; q < c; ++q) G[q] = Ul[m * c + q];
    }
}

/* One 1D sweep over a line of N cells (cell-major, Ul[i*c + comp]).
 * Writes the numerical fluxes fhat[(N+1)*c] at interfaces k = 0..N.
 * sel/win (optional) for this line: sel[side][field][N+1],
 * win[side][field][N+1][2g-1]; forced likewise. */
static int sweep_line(int c, double gamma, const order_t *o, int bc, long N, const double *Ul,
                      const double *alpha_fixed, const int *amax_in, int *amax_out,
                      const uint8_t *forced, uint8_t *sel_out,
                      double *win_out, double *fhat, double *alpha_out, long *ntested,
                      const side_t *lo, const side_t *hi)
{
    int g = o->g, st, q, k, l;
    long i, j;
    double alpha[4];
    double *Ug = (double *)malloc(sizeof(double) * (N + 2 * g) * c);
    double *Fg = (double *)malloc(sizeof(double) * (N + 2 * g) * c);
    const long NI = N + 1;
    if (alpha_fixed) {
        for (k = 0; k < c; ++k) alpha[k] = alpha_fixed[k];
        st = ORC_OK;
    } else {
        st = amax_in ? line_alpha_frozen(c, gamma, Ul, amax_in, alpha)
                     : line_alpha(c, gamma, N, Ul, alpha, amax_out);
    }
    if (alpha_out)
        for (k = 0; k < c; ++k) alpha_out[k] = alpha[k];
    /* ghost fill and physical flux per cell */
    for (j = -g; j < N + g && !st; ++j) {
        prim_t P;
        double Gs[4];
        const double *U = Ul + ghost_index(j, N, bc) * c;
        if ((lo || hi) && (j < 0 || j >= N)) {
            side_ghost(j < 0 ? lo : hi, c, j, N, Ul, Gs);
            U = Gs;
        }
        for (q = 0; q < c; ++q) Ug[(j + g) * c + q] = U[q];
        if (primitive(c, gamma, U, &P)) {
            st = ORC_ENONPHYS;
            break;
        }
        phys_flux(c, U, &P, Fg + (j + g) * c);
    }
    for (k = 0; k <= N && !st; ++k) {
        long ii = k - 1; /* interface ii+1/2 between cells ii and ii+1 */
        double Rm[4][4], Lm[4][4], lam[4];
        double gp[4][2 * MAXG], gm[4][2 * MAXG];
        double fsum[4];
        long cell;
        if (roe_eigen(c, gamma, Ug + (ii + g) * c, Ug + (ii + 1 + g) * c, Rm, lam) ||
            invert(c, Rm, Lm)) {
            st = ORC_ENONPHYS;
            break;
        }
        /* characteristic projection of the 2g-cell window and LF split */
        for (l = 0; l < 2 * g; ++l) {
            cell = ii - g + 1 + l;
            for (q = 0; q < c; ++q) {
                double w = 0.0, f = 0.0;
                int r;
                for (r = 0; r < c; ++r) {
                    w = w + Lm[q][r] * Ug[(cell + g) * c + r];
                    f = f + Lm[q][r] * Fg[(cell + g) * c + r];
                }
                gp[q][l] = 0.5 * (f + alpha[q] * w);
                gm[q][l] = 0.5 * (f - alpha[q] * w);
            }
        }
        for (q = 0; q < c; ++q) {
            double vp[MAXW], vm[MAXW];
            int sp, sm, fsp = -1, fsm = -1;
            for (l = -(g - 1); l <= g - 1; ++l) {
                vp[l + g - 1] = gp[q][(l) + g - 1];       /* cell ii + l       */
                vm[l + g - 1] = gm[q][(1 - l) + g - 1];   /* cell ii + 1 - l   */
            }
            if (forced) {
                fsp = forced[(0 * c + q) * NI + k];
                fsm = forced[(1 * c + q) * NI + k];
            }
            fsum[q] = mr(o, vp + g - 1, fsp, &sp, ntested) + mr(o, vm + g - 1, fsm, &sm, ntested);
            if (sel_out) {
                sel_out[(0 * c + q) * NI + k] = (uint8_t)sp;
                sel_out[(1 * c + q) * NI + k] = (uint8_t)sm;
            }
            if (win_out)
                for (l = 0; l < 2 * g - 1; ++l) {
                    win_out[((0 * c + q) * NI + k) * (2 * g - 1) + l] = vp[l];
                    win_out[((1 * c + q) * NI + k) * (2 * g - 1) + l] = vm[l];
                }
        }
        /* back-projection F = R (f^+ + f^-) */
        for (q = 0; q < c; ++q) {
            double s = 0.0;
            int r;
            for (r = 0; r < c; ++r) s = s + Rm[q][r] * fsum[r];
            fhat[k * c + q] = s;
        }
    }
    (void)i;
    free(Ug);
    free(Fg);
    return st;
}

/* 1D Euler: U is [3][N] (component-major).  sel/win as in sweep_line. */
static int rhs_euler1d(long N, const double *U, double h, int R, int bc, double gamma,
                       const int *amax_in, int *amax_out, const uint8_t *forced,
                       uint8_t *sel_out, double *win_out, double *rhs, double *alpha_out,
                       long *ntested_out)
{
    const order_t *o = get_order(R);
    double *Ul, *fhat;
    long i;
    int q, st;
    long ntested = 0;
    if (!o || N < 1 || !(h > 0) || !(gamma > 1)) return ORC_EINVAL;
    if (bc == 0 && N < 2 * o->g) return ORC_EINVAL;
    Ul = (double *)malloc(sizeof(double) * N * 3);
    fhat = (double *)malloc(sizeof(double) * (N + 1) * 3);
    for (i = 0; i < N; ++i)
        for (q = 0; q < 3; ++q) Ul[i * 3 + q] = U[q * N + i];
    st = sweep_line(3, gamma, o, bc, N, Ul, NULL, amax_in, amax_out, forced, sel_out, win_out,
                    fhat, alpha_out, &ntested, NULL, NULL);
    if (!st)
        for (i = 0; i < N; ++i)
            for (q = 0; q < 3; ++q) rhs[q * N + i] = -(fhat[(i + 1) * 3 + q] - fhat[i * 3 + q]) / h;
    if (ntested_out) *ntested_out = ntested;
    free(Ul);
    free(fhat);
    return st;
}

int orc_rhs_euler1d(long N, const double *U, double h, int R, int bc, double gamma,
                    const uint8_t *forced, uint8_t *sel_out, double *win_out, double *rhs,
                    double *alpha_out, long *ntested_out)
{
    return rhs_euler1d(N, U, h, R, bc, gamma, NULL, NULL, forced, sel_out, win_out, rhs,
                       alpha_out, ntested_out);
}

/* 1D Euler with every discrete choice given: the stencils (forced) and the
 * cell maximising each alpha (amax[3]).  amax_out (optional) receives the
 * maximising cells of the plain scheme when amax_in is NULL. */
int orc_rhs_euler1d_frozen(long N, const double *U, double h, int R, int bc, double gamma,
                           const uint8_t *forced, const int *amax_in, int *amax_out, double *rhs)
{
    return rhs_euler1d(N, U, h, R, bc, gamma, amax_in, amax_out, forced, NULL, NULL, rhs, NULL,
                       NULL);
}

/* 2D Euler, dimension by dimension.  U is [4][ny][nx] with components
 * (rho, rho u, rho v, E).  rhs = x part + y part, where
 * x part = -(F_{i+1/2} - F_{i-1/2})/dx on each row and
 * y part = -(G_{j+1/2} - G_{j-1/2})/dy on each column.
 * sel/win layout: x sweep first, [side][field][row][nx+1], then the y sweep,
 * [side][field][col][ny+1]; win has a trailing [2g-1]. */
static int rhs_euler2d(long nx, long ny, const double *U, double dx, double dy, int R, int bc,
                       double gamma, const double *afx, const double *afy,
                       const int *amx_in, const int *amy_in, int *amx_out,
                       int *amy_out, const uint8_t *forced, uint8_t *sel_out, double *win_out,
                       double *rhs, double *alpha_x, double *alpha_y, long *ntested_out,
                       const double *sides, double t, double gx, double gy)
{
    const order_t *o = get_order(R);
    const long ncell = nx * ny;
    const int W = o ? 2 * o->g - 1 : 0;
    const long xsel = 2L * 4 * ny * (nx + 1);
    double *xpart;
    long y, x;
    int st = ORC_OK;
    long ntested = 0;
    if (!o || nx < 1 || ny < 1 || !(dx > 0) || !(dy > 0) || !(gamma > 1)) return ORC_EINVAL;
    if (bc == 0 && (nx < 2 * o->g || ny < 2 * o->g)) return ORC_EINVAL;
    xpart = (double *)malloc(sizeof(double) * ncell * 4);

    /* x sweep, row by row */
#pragma omp parallel for schedule(dynamic) reduction(+ : ntested)
    for (y = 0; y < ny; ++y) {
        double *Ul = (double *)malloc(sizeof(double) * nx * 4);
        double *fh = (double *)malloc(sizeof(double) * (nx + 1) * 4);
        uint8_t *fl = NULL, *sl = NULL;
        double *wl = NULL;
        long i, nt = 0;
        int q, r, lst;
        for (i = 0; i < nx; ++i)
            for (q = 0; q < 4; ++q) Ul[i * 4 + q] = U[q * ncell + y * nx + i];
        if (forced) fl = (uint8_t *)malloc(8 * (nx + 1));
        if (sel_out) sl = (uint8_t *)malloc(8 * (nx + 1));
        if (win_out) wl = (double *)malloc(sizeof(double) * 8 * (nx + 1) * W);
        if (forced)
            for (r = 0; r < 8; ++r)
                memcpy(fl + r * (nx + 1), forced + ((long)r * ny + y) * (nx + 1), nx + 1);
        {
            const side_t slo = {sides, (y + 0.5) * dy, t, 1};
            const side_t shi = {sides ? sides + 12 : NULL, (y + 0.5) * dy, t, 1};
            lst = sweep_line(4, gamma, o, bc, nx, Ul, afx ? afx + y * 4 : NULL,
                             amx_in ? amx_in + y * 4 : NULL,
                             amx_out ? amx_out + y * 4 : NULL, fl, sl, wl, fh,
                             alpha_x ? alpha_x + y * 4 : NULL, &nt, sides ? &slo : NULL,
                             sides ? &shi : NULL);
        }
        ntested += nt;
        if (lst) {
#pragma omp critical
            st = lst;
        } else {
            for (i = 0; i < nx; ++i)
                for (q = 0; q < 4; ++q)
                    xpart[q * ncell + y * nx + i] = -(fh[(i + 1) * 4 + q] - fh[i * 4 + q]) / dx;
            for (r = 0; r < 8; ++r) {
                if (sel_out) memcpy(sel_out + ((long)r * ny + y) * (nx + 1), sl + r * (nx + 1), nx + 1);
                if (win_out)
                    memcpy(win_out + ((long)r * ny + y) * (nx + 1) * W, wl + (long)r * (nx + 1) * W,
                           sizeof(double) * (nx + 1) * W);
            }
        }
        free(Ul);
        free(fh);
        free(fl);
        free(sl);
        free(wl);
    }
    if (st) {
        free(xpart);
        return st;
    }
    /* y sweep, column by column: normal momentum is rho v */
#pragma omp parallel for schedule(dynamic) reduction(+ : ntested)
    for (x = 0; x < nx; ++x) {
        double *Ul = (double *)malloc(sizeof(double) * ny * 4);
        double *fh = (double *)malloc(sizeof(double) * (ny + 1) * 4);
        uint8_t *fl = NULL, *sl = NULL;
        double *wl = NULL;
        long j, nt = 0;
        int r, lst;
        const long ysel_off = xsel;
        for (j = 0; j < ny; ++j) {
            long idx = j * nx + x;
            Ul[j * 4 + 0] = U[0 * ncell + idx];
            Ul[j * 4 + 1] = U[2 * ncell + idx];
            Ul[j * 4 + 2] = U[1 * ncell + idx];
            Ul[j * 4 + 3] = U[3 * ncell + idx];
        }
        if (forced) fl = (uint8_t *)malloc(8 * (ny + 1));
        if (sel_out) sl = (uint8_t *)malloc(8 * (ny + 1));
        if (win_out) wl = (double *)malloc(sizeof(double) * 8 * (ny + 1) * W);
        if (forced)
            for (r = 0; r < 8; ++r)
                memcpy(fl + r * (ny + 1), forced + ysel_off + ((long)r * nx + x) * (ny + 1), ny + 1);
        {
            const side_t slo = {sides ? sides + 24 : NULL, (x + 0.5) * dx, t, 2};
            const side_t shi = {sides ? sides + 36 : NULL, (x + 0.5) * dx, t, 2};
            lst = sweep_line(4, gamma, o, bc, ny, Ul, afy ? afy + x * 4 : NULL,
                             amy_in ? amy_in + x * 4 : NULL,
                             amy_out ? amy_out + x * 4 : NULL, fl, sl, wl, fh,
                             alpha_y ? alpha_y + x * 4 : NULL, &nt, sides ? &slo : NULL,
                             sides ? &shi : NULL);
        }
        ntested += nt;
        if (lst) {
#pragma omp critical
            st = lst;
        } else {
            for (j = 0; j < ny; ++j) {
                long idx = j * nx + x;
                /* line components (rho, rho v, rho u, E) back to (rho, rho u, rho v, E) */
                double g0 = -(fh[(j + 1) * 4 + 0] - fh[j * 4 + 0]) / dy;
                double g1 = -(fh[(j + 1) * 4 + 2] - fh[j * 4 + 2]) / dy;
                double g2 = -(fh[(j + 1) * 4 + 1] - fh[j * 4 + 1]) / dy;
                double g3 = -(fh[(j + 1) * 4 + 3] - fh[j * 4 + 3]) / dy;
                rhs[0 * ncell + idx] = xpart[0 * ncell + idx] + g0;
                rhs[1 * ncell + idx] = xpart[1 * ncell + idx] + g1;
                rhs[2 * ncell + idx] = xpart[2 * ncell + idx] + g2;
                rhs[3 * ncell + idx] = xpart[3 * ncell + idx] + g3;
                if (gx != 0.0 || gy != 0.0) {
                    /* body force (gx, gy): S = (0, rho gx, rho gy, rho u gx + rho v gy) */
                    const double rho = U[0 * ncell + idx], mx = U[1 * ncell + idx];
                    const double my = U[2 * ncell + idx];
                    rhs[1 * ncell + idx] = rhs[1 * ncell + idx] + rho * gx;
                    rhs[2 * ncell + idx] = rhs[2 * ncell + idx] + rho * gy;
                    rhs[3 * ncell + idx] = rhs[3 * ncell + idx] + (my * gy + mx * gx);
                }
            }
            for (r = 0; r < 8; ++r) {
                if (sel_out)
                    memcpy(sel_out + ysel_off + ((long)r * nx + x) * (ny + 1), sl + r * (ny + 1), ny + 1);
                if (win_out)
                    memcpy(win_out + (ysel_off + ((long)r * nx + x) * (ny + 1)) * W,
                           wl + (long)r * (ny + 1) * W, sizeof(double) * (ny + 1) * W);
            }
        }
        free(Ul);
        free(fh);
        free(fl);
        free(sl);
        free(wl);
    }
    free(xpart);
    if (ntested_out) *ntested_out = ntested;
    return st;
}

int orc_rhs_euler2d(long nx, long ny, const double *U, double dx, double dy, int R, int bc,
                    double gamma, const uint8_t *forced, uint8_t *sel_out, double *win_out,
                    double *rhs, double *alpha_x, double *alpha_y, long *ntested_out)
{
    return rhs_euler2d(nx, ny, U, dx, dy, R, bc, gamma, NULL, NULL, NULL, NULL, NULL, NULL, forced,
                       sel_out, win_out, rhs, alpha_x, alpha_y, ntested_out, NULL, 0.0, 0.0, 0.0);
}

/* 2D Euler on [0, nx dx] x [0, ny dy] with boundary sides (4 x 12 doubles:
 * x low, x high, y low, y high; see side_t) at time t and a body force
 * (gx, gy).  bc must be transmissive; sel as orc_rhs_euler2d. */
int orc_rhs_euler2d_ext(long nx, long ny, const double *U, double dx, double dy, int R,
                        double gamma, const double *sides, double t, double gx, double gy,
                        const uint8_t *forced, uint8_t *sel_out, double *win_out, double *rhs)
{
    /* a reflective side mirrors the g cells next to it: its lines (rows for
     * the x sides, columns for the y sides) must hold at least g cells */
    const order_t *o = get_order(R);
    int sd;
    if (!o) return ORC_EINVAL;
    for (sd = 0; sides && sd < 4; ++sd) {
        const double *d = sides + 12 * sd;
        const long len = sd < 2 ? nx : ny;
        if (((int)d[0] == SIDE_REFLECTIVE || (int)d[1] == SIDE_REFLECTIVE) && len < o->g)
            return ORC_EINVAL;
    }
    return rhs_euler2d(nx, ny, U, dx, dy, R, 1, gamma, NULL, NULL, NULL, NULL, NULL, NULL, forced,
                       sel_out, win_out, rhs, NULL, NULL, NULL, sides, t, gx, gy);
}

/* 2D Euler with every discrete choice given (stencils and, per row and per
 * column, the cell maximising each field's alpha: amx[ny][4], amy[nx][4]);
 * with amx_in NULL the plain scheme runs and its maximising cells are
 * written to amx_out/amy_out. */
int orc_rhs_euler2d_frozen(long nx, long ny, const double *U, double dx, double dy, int R, int bc,
                           double gamma, const uint8_t *forced, const int *amx_in,
                           const int *amy_in, int *amx_out, int *amy_out, double *rhs)
{
    return rhs_euler2d(nx, ny, U, dx, dy, R, bc, gamma, NULL, NULL, amx_in, amy_in, amx_out,
                       amy_out, forced, NULL, NULL, rhs, NULL, NULL, NULL, NULL, 0.0, 0.0, 0.0);
}

/* 2D Euler with the stencils forced and the split speeds given as values
 * (alpha_x[ny][4], alpha_y[nx][4]): used to differentiate with respect to
 * alpha alone. */
int orc_rhs_euler2d_alpha(long nx, long ny, const double *U, double dx, double dy, int R, int bc,
                          double gamma, const uint8_t *forced, const double *alpha_x,
                          const double *alpha_y, double *rhs)
{
    return rhs_euler2d(nx, ny, U, dx, dy, R, bc, gamma, alpha_x, alpha_y, NULL, NULL, NULL, NULL,
                       forced, NULL, NULL, rhs, NULL, NULL, NULL, NULL, 0.0, 0.0, 0.0);
}

/* ------------------------------------------------------------------------- */
/* Generic RHS dispatcher used by the time integrators.                      */
/* eq: 0 advection (uses a), 1 Euler 1D, 2 Euler 2D, 3 Burgers.              */
/* ------------------------------------------------------------------------- */
typedef struct {
    int eq, R, bc;
    long nx, ny;
    double dx, dy, gamma, a;
} problem_t;

static long prob_size(const problem_t *P)
{
    if (P->eq == 0 || P->eq == 3) return P->nx;
    if (P->eq == 1) return 3 * P->nx;
    return 4 * P->nx * P->ny;
}

static int prob_rhs(const problem_t *P, const double *U, double *rhs)
{
    if (P->eq == 0)
        return orc_rhs_advection(P->nx, U, P->dx, P->R, P->bc, P->a, NULL, NULL, NULL, rhs, NULL);
    if (P->eq == 3)
        return orc_rhs_burgers(P->nx, U, P->dx, P->R, P->bc, NULL, NULL, NULL, rhs, NULL);
    if (P->eq == 1)
        return orc_rhs_euler1d(P->nx, U, P->dx, P->R, P->bc, P->gamma, NULL, NULL, NULL, rhs, NULL,
                               NULL);
    return orc_rhs_euler2d(P->nx, P->ny, U, P->dx, P->dy, P->R, P->bc, P->gamma, NULL, NULL, NULL,
                           rhs, NULL, NULL, NULL);
}

/* Public RHS with the same dispatch (U and rhs hold prob_size doubles). */
int orc_rhs(int eq, long nx, long ny, double dx, double dy, int R, int bc, double gamma, double a,
            const double *U, double *rhs)
{
    problem_t P = {eq, R, bc, nx, ny, dx, dy, gamma, a};
    return prob_rhs(&P, U, rhs);
}

/* CFL time step: 1D dt = cfl*h / max(|u|+c) (advection: cfl*h/|a|;
 * Burgers: cfl*h/max|u|); 2D dt = cfl / max((|u|+c)/dx + (|v|+c)/dy). */
int orc_cfl_dt(int eq, long nx, long ny, double dx, double dy, double gamma, double a,
               const double *U, double cfl, double *dt)
{
    long i, n = (eq == 2) ? nx * ny : nx;
    double smax = 0.0;
    if (eq == 0) {
        if (!(dabs(a) > 0)) return ORC_EINVAL;
        *dt = cfl * dx / dabs(a);
        return ORC_OK;
    }
    if (eq == 3) {
        for (i = 0; i < nx; ++i) smax = dmax(smax, dabs(U[i]));
        if (!(smax > 0)) return ORC_EINVAL;
        *dt = cfl * dx / smax;
        return ORC_OK;
    }
    for (i = 0; i < n; ++i) {
        prim_t P;
        double Uc[4], s;
        if (eq == 1) {
            Uc[0] = U[i]; Uc[1] = U[n + i]; Uc[2] = U[2 * n + i];
            if (primitive(3, gamma, Uc, &P)) return ORC_ENONPHYS;
            s = dabs(P.un) + P.c;
        } else {
            double sx, sy;
            Uc[0] = U[i]; Uc[1] = U[n + i]; Uc[2] = U[2 * n + i]; Uc[3] = U[3 * n + i];
            if (primitive(4, gamma, Uc, &P)) return ORC_ENONPHYS;
            sx = (dabs(P.un) + P.c) / dx;
            sy = (dabs(P.ut) + P.c) / dy;
            s = sx + sy;
        }
        smax = dmax(smax, s);
    }
    *dt = (eq == 1) ? cfl * dx / smax : cfl / smax;
    return ORC_OK;
}

/* Eq. (TVD3rdRK): one SSP-RK3 step, in the paper's written form. */
int orc_step_ssprk3(int eq, long nx, long ny, double dx, double dy, int R, int bc, double gamma,
                    double a, double *U, double dt)
{
    problem_t P = {eq, R, bc, nx, ny, dx, dy, gamma, a};
    long n = prob_size(&P), i;
    double *L = (double *)malloc(sizeof(double) * n);
    double *U1 = (double *)malloc(sizeof(double) * n);
    double *U2 = (double *)malloc(sizeof(double) * n);
    int st = prob_rhs(&P, U, L);
    if (!st) {
        for (i = 0; i < n; ++i) U1[i] = U[i] + dt * L[i];
        st = prob_rhs(&P, U1, L);
    }
    if (!st) {
        for (i = 0; i < n; ++i) U2[i] = 0.75 * U[i] + 0.25 * (U1[i] + dt * L[i]);
        st = prob_rhs(&P, U2, L);
    }
    if (!st)
        for (i = 0; i < n; ++i) U[i] = (1.0 / 3.0) * U[i] + (2.0 / 3.0) * (U2[i] + dt * L[i]);
    free(L);
    free(U1);
    free(U2);
    return st;
}

/* Eq. (TVD3rdRK) for 2D Euler with boundary sides and a body force: the
 * stage right-hand sides are taken at t, t + dt and t + dt/2. */
int orc_step_ssprk3_euler2d_ext(long nx, long ny, double dx, double dy, int R, double gamma,
                                const double *sides, double t, double gx, double gy, double *U,
                                double dt)
{
    long n = 4 * nx * ny, i;
    double *L = (double *)malloc(sizeof(double) * n);
    double *U1 = (double *)malloc(sizeof(double) * n);
    double *U2 = (double *)malloc(sizeof(double) * n);
    int st = orc_rhs_euler2d_ext(nx, ny, U, dx, dy, R, gamma, sides, t, gx, gy, NULL, NULL, NULL, L);
    if (!st) {
        for (i = 0; i < n; ++i) U1[i] = U[i] + dt * L[i];
        st = orc_rhs_euler2d_ext(nx, ny, U1, dx, dy, R, gamma, sides, t + dt, gx, gy, NULL, NULL,
                                 NULL, L);
    }
    if (!st) {
        for (i = 0; i < n; ++i) U2[i] = 0.75 * U[i] + 0.25 * (U1[i] + dt * L[i]);
        st = orc_rhs_euler2d_ext(nx, ny, U2, dx, dy, R, gamma, sides, t + 0.5 * dt, gx, gy, NULL,
                                 NULL, NULL, L);
    }
    if (!st)
        for (i = 0; i < n; ++i) U[i] = (1.0 / 3.0) * U[i] + (2.0 / 3.0) * (U2[i] + dt * L[i]);
    free(L);
    free(U1);
    free(U2);
    return st;
}

/* Eq. (lSSPRK_Coe) with the reading alpha_{m,m-1} = (2/m) alpha_{m-1,m-2}:
 * coefficients alpha_{m,0..m-1} written to out[0..m-1]. */
int orc_lssp_coeffs(int m, double *out)
{
    double prev[32], cur[32];
    int mm, k;
    if (m < 2 || m > 31) return ORC_EINVAL;
    prev[0] = 0.0;
    prev[1] = 1.0;
    for (mm = 3; mm <= m; ++mm) {
        double s = 0.0;
        for (k = 1; k <= mm - 2; ++k) cur[k] = (2.0 / k) * prev[k - 1];
        cur[mm - 1] = (2.0 / mm) * prev[mm - 2];
        for (k = 1; k <= mm - 1; ++k) s = s + cur[k];
        cur[0] = 1.0 - s;
        for (k = 0; k < mm; ++k) prev[k] = cur[k];
    }
    for (k = 0; k < m; ++k) out[k] = prev[k];
    return ORC_OK;
}

/* Eq. (lSSPRK): one l-SSP-RK(m, m-1) step. */
int orc_step_lssp(int m, int eq, long nx, long ny, double dx, double dy, int R, int bc,
                  double gamma, double a, double *U, double dt)
{
    problem_t P = {eq, R, bc, nx, ny, dx, dy, gamma, a};
    long n = prob_size(&P), i;
    double alpha[32];
    double *stage = (double *)malloc(sizeof(double) * n * m); /* u^(0..m-1) */
    double *L = (double *)malloc(sizeof(double) * n);
    int s, k, st = orc_lssp_coeffs(m, alpha);
    if (!st) memcpy(stage, U, sizeof(double) * n);
    for (s = 1; s <= m - 1 && !st; ++s) {
        st = prob_rhs(&P, stage + (s - 1) * n, L);
        if (!st)
            for (i = 0; i < n; ++i) stage[s * n + i] = stage[(s - 1) * n + i] + 0.5 * dt * L[i];
    }
    if (!st) st = prob_rhs(&P, stage + (m - 1) * n, L);
    if (!st)
        for (i = 0; i < n; ++i) {
            double acc = 0.0;
            for (k = 0; k <= m - 2; ++k) acc = acc + alpha[k] * stage[k * n + i];
            U[i] = acc + alpha[m - 1] * (stage[(m - 1) * n + i] + 0.5 * dt * L[i]);
        }
    free(stage);
    free(L);
    return st;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
