/* Test driver: runs the oracle's entry points on small, edge-case inputs in
 * one process built with AddressSanitizer and UndefinedBehaviorSanitizer
 * (tests/test_oracle_sanitize.py compiles and runs it).  Every buffer is a
 * malloc of exactly the size the entry point's contract names, so a read or
 * write past it, a use of freed memory, a leak or undefined arithmetic on
 * integers aborts the run.  Status codes other than success are allowed
 * where the contract rejects the input (too short a periodic line, a
 * non-physical state); results are not checked here: the other oracle tests
 * do that.
 *
 * The oracle is compiled into this translation unit, without OpenMP. */
#include <stdio.h>

#include "oracle/enomr_oracle.c"

static unsigned long long rng_state = 0x9e3779b97f4a7c15ULL;

static double urand(void) /* in [0, 1) */
{
    rng_state = rng_state * 6364136223846793005ULL + 1442695040888963407ULL;
    return (double)(rng_state >> 11) * (1.0 / 9007199254740992.0);
}

static double *dalloc(long n)
{
    return (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
}

static uint8_t *balloc(long n)
{
    return (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
}

/* a primitive state -> conserved components at cell i of an n-cell field */
static void put_state(double *U, long n, long i, int c, double rho, double u, double v, double p,
                      double gamma)
{
    U[i] = rho;
    U[n + i] = rho * u;
    if (c == 4) {
        U[2 * n + i] = rho * v;
        U[3 * n + i] = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v);
    } else {
        U[2 * n + i] = p / (gamma - 1.0) + 0.5 * rho * u * u;
    }
}

/* piecewise-constant with a smooth part: runs of equal cells and varying ones */
static void euler_field(double *U, long n, int c, double gamma)
{
    long i;
    for (i = 0; i < n; ++i) {
        if ((i / 5) % 3 == 0)
            put_state(U, n, i, c, 1.0, 0.3, -0.2, 1.0, gamma);
        else
            put_state(U, n, i, c, 0.5 + urand(), urand() - 0.5, urand() - 0.5, 0.2 + urand(),
                      gamma);
    }
}

static int scalar_cases(int R)
{
    const int g = (R + 1) / 2, W = 2 * g - 1;
    const long sizes[4] = {1, 2 * g, 2 * g + 1, 37};
    int k, bc, st = 0;
    for (k = 0; k < 4; ++k) {
        for (bc = 0; bc < 2; ++bc) {
            const long N = sizes[k];
            double *u = dalloc(N), *rhs = dalloc(N), *win = dalloc(2 * (N + 1) * W);
            uint8_t *sel = balloc(2 * (N + 1)), *forced = balloc(2 * (N + 1));
            long cnt = 0, i;
            double dt = 0.0;
            for (i = 0; i < N; ++i) u[i] = (i % 4 == 0) ? 1.0 : urand() - 0.5;
            if (orc_rhs_advection(N, u, 0.1, R, bc, 1.0, NULL, sel, win, rhs, &cnt) == ORC_OK) {
                memcpy(forced, sel, (size_t)(2 * (N + 1)));
                orc_rhs_advection(N, u, 0.1, R, bc, 1.0, forced, NULL, NULL, rhs, NULL);
            }
            if (orc_rhs_burgers(N, u, 0.1, R, bc, NULL, sel, win, rhs, &cnt) == ORC_OK) {
                memcpy(forced, sel, (size_t)(2 * (N + 1)));
                orc_rhs_burgers(N, u, 0.1, R, bc, forced, NULL, NULL, rhs, NULL);
            }
            orc_step_ssprk3(0, N, 1, 0.1, 0.1, R, bc, 1.4, 1.0, u, 0.01);
            if (orc_cfl_dt(3, N, 1, 0.1, 0.1, 1.4, 0.0, u, 0.5, &dt) == ORC_OK)
                orc_step_ssprk3(3, N, 1, 0.1, 0.1, R, bc, 1.4, 0.0, u, dt);
            orc_step_lssp(3, 0, N, 1, 0.1, 0.1, R, bc, 1.4, 1.0, u, 0.1);
            free(u);
            free(rhs);
            free(win);
            free(sel);
            free(forced);
        }
    }
    return st;
}

static void window_cases(int R)
{
    const int g = (R + 1) / 2, W = 2 * g - 1, T = orc_num_tested(R);
    double *w = dalloc(W), *is = dalloc(T), *mag = dalloc(T);
    double is0, mag0, a[17], b[17];
    int t, sel, m, n, j;
    for (t = 0; t < T; ++t) orc_candidate(R, t, &m, &n, a, b);
    for (j = 0; j < 20; ++j) {
        int l;
        for (l = 0; l < W; ++l) w[l] = (j % 3 == 0) ? 1.0 : urand();
        orc_mr_indicators(R, w, &is0, &mag0, is, &mag[0]);
        for (t = -1; t < T + 3; ++t) orc_mr(R, w, t, &sel);
    }
    free(w);
    free(is);
    free(mag);
}

static void euler1d_cases(int R, double gamma)
{
    const int g = (R + 1) / 2, W = 2 * g - 1;
    const long sizes[5] = {1, 2, 3, 2 * g, 40};
    int k, bc;
    for (k = 0; k < 5; ++k) {
        for (bc = 0; bc < 2; ++bc) {
            const long N = sizes[k];
            double *U = dalloc(3 * N), *rhs = dalloc(3 * N), *win = dalloc(2 * 3 * (N + 1) * W);
            double alpha[3], dt = 0.0;
            uint8_t *sel = balloc(2 * 3 * (N + 1));
            int amax[3];
            long cnt = 0;
            euler_field(U, N, 3, gamma);
            if (orc_rhs_euler1d(N, U, 0.1, R, bc, gamma, NULL, sel, win, rhs, alpha, &cnt) ==
                ORC_OK) {
                orc_rhs_euler1d_frozen(N, U, 0.1, R, bc, gamma, sel, NULL, amax, rhs);
                orc_rhs_euler1d_frozen(N, U, 0.1, R, bc, gamma, sel, amax, NULL, rhs);
            }
            if (orc_cfl_dt(1, N, 1, 0.1, 0.1, gamma, 0.0, U, 0.5, &dt) == ORC_OK) {
                orc_step_ssprk3(1, N, 1, 0.1, 0.1, R, bc, gamma, 0.0, U, dt);
                orc_step_lssp(2, 1, N, 1, 0.1, 0.1, R, bc, gamma, 0.0, U, 0.5 * dt);
            }
            free(U);
            free(rhs);
            free(win);
            free(sel);
        }
    }
}

static void euler2d_cases(int R, double gamma)
{
    const int g = (R + 1) / 2, W = 2 * g - 1;
    const long shapes[5][2] = {{1, 37}, {37, 1}, {2, 3}, {13, 11}, {2 * g, 2 * g}};
    int k, bc;
    for (k = 0; k < 5; ++k) {
        for (bc = 0; bc < 2; ++bc) {
            const long nx = shapes[k][0], ny = shapes[k][1], n = nx * ny;
            const long nsel = 8 * ny * (nx + 1) + 8 * nx * (ny + 1);
            double *U = dalloc(4 * n), *rhs = dalloc(4 * n), *win = dalloc(nsel * W);
            double *ax = dalloc(4 * ny), *ay = dalloc(4 * nx), *al = dalloc(4 * ny),
                   *aly = dalloc(4 * nx);
            int *amx = (int *)malloc(sizeof(int) * 4 * ny), *amy = (int *)malloc(sizeof(int) * 4 * nx);
            uint8_t *sel = balloc(nsel);
            long cnt = 0, i;
            double dt = 0.0;
            euler_field(U, n, 4, gamma);
            if (orc_rhs_euler2d(nx, ny, U, 0.1, 0.2, R, bc, gamma, NULL, sel, win, rhs, ax, ay,
                                &cnt) == ORC_OK) {
                orc_rhs_euler2d_frozen(nx, ny, U, 0.1, 0.2, R, bc, gamma, sel, NULL, NULL, amx,
                                       amy, rhs);
                orc_rhs_euler2d_frozen(nx, ny, U, 0.1, 0.2, R, bc, gamma, sel, amx, amy, NULL,
                                       NULL, rhs);
                for (i = 0; i < 4 * ny; ++i) al[i] = ax[i];
                for (i = 0; i < 4 * nx; ++i) aly[i] = ay[i];
                orc_rhs_euler2d_alpha(nx, ny, U, 0.1, 0.2, R, bc, gamma, sel, al, aly, rhs);
            }
            if (orc_cfl_dt(2, nx, ny, 0.1, 0.2, gamma, 0.0, U, 0.5, &dt) == ORC_OK)
                orc_step_ssprk3(2, nx, ny, 0.1, 0.2, R, bc, gamma, 0.0, U, dt);
            free(U);
            free(rhs);
            free(win);
            free(ax);
            free(ay);
            free(al);
            free(aly);
            free(amx);
            free(amy);
            free(sel);
        }
    }
}

static void set_side(double *s, int kind_lo, int kind_hi, double split0, double rate,
                     const double *lo, const double *hi)
{
    int q;
    s[0] = kind_lo;
    s[1] = kind_hi;
    s[2] = split0;
    s[3] = rate;
    for (q = 0; q < 4; ++q) {
        s[4 + q] = lo ? lo[q] : 0.0;
        s[8 + q] = hi ? hi[q] : 0.0;
    }
}

static void euler2d_side_cases(int R, double gamma)
{
    const int g = (R + 1) / 2, W = 2 * g - 1;
    const long shapes[3][2] = {{12, 10}, {3, 20}, {2 * g, 2 * g + 1}};
    double inflow[4];
    int k;
    put_state(inflow, 1, 0, 4, 1.4, 0.5, 0.1, 1.0, gamma);
    for (k = 0; k < 3; ++k) {
        const long nx = shapes[k][0], ny = shapes[k][1], n = nx * ny;
        const long nsel = 8 * ny * (nx + 1) + 8 * nx * (ny + 1);
        double *U = dalloc(4 * n), *rhs = dalloc(4 * n), *win = dalloc(nsel * W);
        double sides[48];
        uint8_t *sel = balloc(nsel);
        euler_field(U, n, 4, gamma);
        set_side(sides + 0, 3, 1, 1e300, 0.0, inflow, NULL);          /* x low: inflow */
        set_side(sides + 12, 1, 2, 0.05 * ny, 0.0, NULL, NULL);       /* x high */
        set_side(sides + 24, 1, 2, 0.03 * nx, 2.0, NULL, NULL);       /* y low: moving split */
        set_side(sides + 36, 2, 3, 0.05 * nx, 1.0, NULL, inflow);     /* y high */
        if (orc_rhs_euler2d_ext(nx, ny, U, 0.1, 0.1, R, gamma, sides, 0.1, 0.0, 1.0, NULL, sel,
                                win, rhs) == ORC_OK)
            orc_rhs_euler2d_ext(nx, ny, U, 0.1, 0.1, R, gamma, sides, 0.1, 0.0, 1.0, sel, NULL,
                                NULL, rhs);
        orc_step_ssprk3_euler2d_ext(nx, ny, 0.1, 0.1, R, gamma, sides, 0.0, 0.3, -0.2, U, 1e-3);
        free(U);
        free(rhs);
        free(win);
        free(sel);
    }
}

int main(void)
{
    int R;
    double c[8];
    for (R = 5; R <= 17; R += 2) {
        window_cases(R);
        scalar_cases(R);
        euler1d_cases(R, 1.4);
        euler2d_cases(R, 1.4);
        euler2d_side_cases(R, 5.0 / 3.0);
    }
    for (R = 1; R <= 8; ++R) orc_lssp_coeffs(R, c);
    /* rejected inputs */
    orc_num_tested(4);
    orc_num_tested(19);
    printf("ok\n");
    return 0;
}
