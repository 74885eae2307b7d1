// enomr_common.cuh -- device helpers shared by the alpha reduction and the
// sweep epilogues, so that both take the same operations on a cell state.
#pragma once

#include "enomr_internal.h"

namespace enomr {

// x > 0 (+inf included, NaN excluded) and |x| < 1e300, tested on the
// integer ALU: for doubles the IEEE bit pattern, read as an int64, orders
// like the value on the non-negative half-line.
__device__ __forceinline__ bool positive(double x)
{
    const long long b = __double_as_longlong(x);
    return b > 0 && b <= 0x7ff0000000000000LL;
}

__device__ __forceinline__ bool below_1e300(double x)
{
    return (__double_as_longlong(x) & 0x7fffffffffffffffLL) < 0x7e37e43c8800759cLL;
}

struct CellWaves {
    double u, v, c;  // normal and tangential velocity, sound speed
};

// The helpers below are written with explicitly rounded operations
// (__dmul_rn, __fma_rn, ...), which the compiler never contracts or
// re-associates.  Every kernel that needs the same quantity of the same
// state -- the alpha reduction, the argmax search of the adjoint, the
// stage epilogues, the forward sweeps and their recomputation in the
// adjoint -- therefore obtains the same bits.

// Primitive velocity and sound speed of one cell (ideal gas); flags a
// non-physical state in the status word.
template <int C>
__device__ __forceinline__ CellWaves cell_waves(double rho, double mx, double my, double E,
                                                double gm1, double gamma, int *status)
{
    const double ir = 1.0 / rho;  // IEEE division: never contracted
    const double u = __dmul_rn(mx, ir);
    const double v = (C == 4) ? __dmul_rn(my, ir) : 0.0;
    // u^2 + v^2 in a form symmetric in u and v, so that a state symmetric
    // under x <-> y (with u <-> v) has bitwise equal x- and y-line speeds
    const double ke = (C == 4) ? __dadd_rn(__dmul_rn(u, u), __dmul_rn(v, v)) : __dmul_rn(u, u);
    const double p = __dmul_rn(gm1, __fma_rn(-0.5 * rho, ke, E));
    if (!positive(rho) || !positive(p) || !below_1e300(E)) atomicOr(status, ST_NONPHYS_CELL);
    const double c2 = __dmul_rn(__dmul_rn(gamma, p), ir);
    CellWaves w;
    w.u = u;
    w.v = v;
    w.c = __dmul_rn(c2, rsqrt(c2));
    return w;
}

// |u - c|, |u|, |u + c| of a 1D cell: the per-field speeds whose line maxima
// are the split speeds alpha_k.
__device__ __forceinline__ void wave_speeds3(double rho, double m, double E, double gm1,
                                             double gamma, double *out, int *status)
{
    const CellWaves w = cell_waves<3>(rho, m, 0.0, E, gm1, gamma, status);
    out[0] = fabs(__dsub_rn(w.u, w.c));
    out[1] = fabs(w.u);
    out[2] = fabs(__dadd_rn(w.u, w.c));
}

// Staged quantities of one cell for a sweep whose normal momentum is mn:
// sqrt(rho), u_n, u_t, H and the normal flux (m_n, m_n u_n + p, m_t u_n,
// (E + p) u_n).
template <int C>
struct StagedCell {
    double sq, un, ut, H, p;
    double F[C];
};

template <int C>
__device__ __forceinline__ StagedCell<C> stage_cell(double rho, double mn, double mt, double E,
                                                    double gm1)
{
    StagedCell<C> o;
    const double rr = rsqrt(rho);
    const double ir = __dmul_rn(rr, rr);
    o.un = __dmul_rn(mn, ir);
    o.ut = (C == 4) ? __dmul_rn(mt, ir) : 0.0;
    const double ke = (C == 4) ? __fma_rn(o.un, o.un, __dmul_rn(o.ut, o.ut)) : __dmul_rn(o.un, o.un);
    o.p = __dmul_rn(gm1, __fma_rn(-0.5 * rho, ke, E));
    const double Ep = __dadd_rn(E, o.p);
    o.sq = __dmul_rn(rho, rr);
    o.H = __dmul_rn(Ep, ir);
    o.F[0] = mn;
    o.F[1] = __fma_rn(mn, o.un, o.p);
    if (C == 4) o.F[2] = __dmul_rn(mt, o.un);
    o.F[C - 1] = __dmul_rn(Ep, o.un);
    return o;
}

// Roe-averaged state at a face and the quantities of the scaled
// eigenvectors (c, c/(gamma-1), c^2/(gamma-1), (gamma-1)/c^2).
struct RoeFace {
    double uh, vh, Hh, hq, c2, ic, cs, kap, c2g, b1;
};

__device__ __forceinline__ RoeFace roe_face(bool equal, double qL, double uL, double vL,
                                            double HL, double qR, double uR, double vR,
                                            double HR, bool twod, double gm1, double inv_gm1)
{
    RoeFace r;
    if (equal) {
        r.uh = uL;
        r.vh = twod ? vL : 0.0;
        r.Hh = HL;
    } else {
        const double rs = 1.0 / __dadd_rn(qL, qR);
        r.uh = __dmul_rn(__fma_rn(qL, uL, __dmul_rn(qR, uR)), rs);
        r.vh = twod ? __dmul_rn(__fma_rn(qL, vL, __dmul_rn(qR, vR)), rs) : 0.0;
        r.Hh = __dmul_rn(__fma_rn(qL, HL, __dmul_rn(qR, HR)), rs);
    }
    r.hq = __dmul_rn(0.5, __fma_rn(r.uh, r.uh, __dmul_rn(r.vh, r.vh)));
    r.c2 = __dmul_rn(gm1, __dsub_rn(r.Hh, r.hq));
    r.ic = rsqrt(r.c2);
    r.cs = __dmul_rn(r.c2, r.ic);
    r.kap = __dmul_rn(r.cs, inv_gm1);
    r.c2g = __dmul_rn(r.c2, inv_gm1);
    r.b1 = __dmul_rn(gm1, __dmul_rn(r.ic, r.ic));
    return r;
}

}  // namespace enomr
