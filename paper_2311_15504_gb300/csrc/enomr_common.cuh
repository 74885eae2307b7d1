// enomr_common.cuh -- device helpers shared by the alpha reduction and the
// sweep epilogues, so that both take the same operations on a cell state.
#pragma once

#include "enomr_internal.h"

namespace enomr {

struct CellWaves {
    double u, v, c;  // normal and tangential velocity, sound speed
};

// Primitive velocity and sound speed of one cell (ideal gas); flags a
// non-physical state in the status word.
template <int C>
__device__ __forceinline__ CellWaves cell_waves(double rho, double mx, double my, double E,
                                                double gm1, double gamma, int *status)
{
    const double ir = 1.0 / rho;
    const double u = mx * ir;
    const double v = (C == 4) ? my * ir : 0.0;
    const double ke = (C == 4) ? fma(u, u, v * v) : u * u;
    const double p = gm1 * (E - 0.5 * rho * ke);
    if (!(rho > 0.0) || !(p > 0.0) || !(fabs(E) < 1e300)) atomicOr(status, ST_NONPHYS_CELL);
    const double c2 = gamma * p * ir;
    CellWaves w;
    w.u = u;
    w.v = v;
    w.c = c2 * rsqrt(c2);
    return w;
}

// |u - c|, |u|, |u + c| of a 1D cell: the per-field speeds whose line maxima
// are the split speeds alpha_k.
__device__ __forceinline__ void wave_speeds3(double rho, double m, double E, double gm1,
                                             double gamma, double *out, int *status)
{
    const CellWaves w = cell_waves<3>(rho, m, 0.0, E, gm1, gamma, status);
    out[0] = fabs(w.u - w.c);
    out[1] = fabs(w.u);
    out[2] = fabs(w.u + w.c);
}

}  // namespace enomr
