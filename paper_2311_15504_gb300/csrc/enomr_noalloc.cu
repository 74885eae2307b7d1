// enomr_noalloc.cu -- a 2D Euler right-hand side that allocates nothing.
//
// Some callers cannot call cudaMalloc: host frameworks that reserve the
// device memory for their own caching allocator (a stray cudaMalloc then
// fails or fragments their pool), applications with a fixed device-memory
// budget, and latency-sensitive loops where cudaMalloc/cudaFree would
// synchronise the device.  For them, enomr_rhs_euler2d_noalloc() needs no
// context and no allocation: its only scratch (the per-line alpha maxima and
// a status word) lives in the file-scope device array below, which every GPU
// that loads this library holds until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "../../include/enomr.h"
#include "enomr_internal.h"

namespace {

// Largest nx and ny accepted (lines per direction).
constexpr long long kMaxLines = ENOMR_NOALLOC_MAX_LINES;
// alpha_x [kMaxLines][3], alpha_y [kMaxLines][3], status word (padded).
constexpr long long kScratchDoubles = 6 * kMaxLines + 32;

static __device__ __align__(256) double g_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double *g_scratch_addr[kMaxDevices] = {};  // device address of g_scratch, per device

// Device address of g_scratch on the current device.  In host code the name
// g_scratch is only a host-side stand-in, so the address is looked up with
// that device current.  It is looked up again on every call made outside
// stream capture (a device reset reloads the module, and the array may then
// sit elsewhere); during capture the address cached by the last call outside
// capture on that device is used, so the first call on a device must come
// before any capture.
cudaError_t scratch_address(cudaStream_t s, double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (cs == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<double *>(p);
    } else if (!g_scratch_addr[dev]) {
        return cudaErrorStreamCaptureUnsupported;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

template <int R> cudaError_t run_x(const enomr::SweepArgs &a, cudaStream_t s)
{
    return enomr::launch_euler2d_x<R>(a, false, s);
}
template <int R> cudaError_t run_y(const enomr::SweepArgs &a, cudaStream_t s)
{
    return enomr::launch_euler2d_y<R>(a, false, s);
}

cudaError_t sweep(bool ysweep, int R, const enomr::SweepArgs &a, cudaStream_t s)
{
    switch (R) {
    case 5: return ysweep ? run_y<5>(a, s) : run_x<5>(a, s);
    case 7: return ysweep ? run_y<7>(a, s) : run_x<7>(a, s);
    case 9: return ysweep ? run_y<9>(a, s) : run_x<9>(a, s);
    case 11: return ysweep ? run_y<11>(a, s) : run_x<11>(a, s);
    case 13: return ysweep ? run_y<13>(a, s) : run_x<13>(a, s);
    case 15: return ysweep ? run_y<15>(a, s) : run_x<15>(a, s);
    case 17: return ysweep ? run_y<17>(a, s) : run_x<17>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

extern "C" ENOMR_API enomr_status enomr_rhs_euler2d_noalloc(const double *U, double *dUdt,
                                                            int64_t nx, int64_t ny, double dx,
                                                            double dy, int order, double gamma,
                                                            int bc, void *stream)
{
    if (!U || !dUdt || (const double *)dUdt == U) return ENOMR_EINVAL;
    if (order < 5 || order > 17 || (order % 2) == 0) return ENOMR_EINVAL;
    if (bc != ENOMR_PERIODIC && bc != ENOMR_TRANSMISSIVE) return ENOMR_EINVAL;
    if (nx < 1 || ny < 1 || !(dx > 0.0) || !(dy > 0.0) || !(gamma > 1.0)) return ENOMR_EINVAL;
    if (nx > kMaxLines || ny > kMaxLines) return ENOMR_EINVAL;  // beyond the static scratch
    const int g = (order + 1) / 2;
    if (bc == ENOMR_PERIODIC && (nx < 2 * g || ny < 2 * g)) return ENOMR_EINVAL;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double *base = nullptr;
    if (scratch_address(s, &base) != cudaSuccess) return ENOMR_ECUDA;
    double *ax = base;                 // [ny][3]
    double *ay = base + 3 * kMaxLines; // [nx][3]
    int *status = reinterpret_cast<int *>(base + 6 * kMaxLines);

    // the maxima accumulate with atomicMax and must start at zero
    if (cudaMemsetAsync(ax, 0, sizeof(double) * 3 * ny, s) != cudaSuccess ||
        cudaMemsetAsync(ay, 0, sizeof(double) * 3 * nx, s) != cudaSuccess ||
        cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess)
        return ENOMR_ECUDA;

    enomr::AlphaArgs aa;
    aa.U = U;
    aa.nx = nx;
    aa.ny = ny;
    aa.gm1 = gamma - 1.0;
    aa.gamma = gamma;
    aa.inv_dx = 1.0 / dx;
    aa.inv_dy = 1.0 / dy;
    aa.ax = ax;
    aa.ay = ay;
    aa.smax = nullptr;
    aa.status = status;
    if (enomr::launch_alpha(4, aa, s) != cudaSuccess) return ENOMR_ECUDA;

    enomr::SweepArgs a;
    memset(&a, 0, sizeof(a));
    a.U = U;
    a.nx = nx;
    a.ny = ny;
    a.bc = bc;
    a.gamma = gamma;
    a.gm1 = gamma - 1.0;
    a.inv_gm1 = 1.0 / (gamma - 1.0);
    a.status = status;
    a.sel = nullptr;
    // x sweep: its flux difference goes straight into dUdt ...
    a.inv_h = 1.0 / dx;
    a.alpha = ax;
    a.epi.mode = enomr::EPI_STORE;
    a.epi.out = dUdt;
    if (sweep(false, order, a, s) != cudaSuccess) return ENOMR_ECUDA;
    // ... and the y sweep adds its own to it, cell by cell, in place
    a.inv_h = 1.0 / dy;
    a.alpha = ay;
    a.epi.Dprev = dUdt;
    if (sweep(true, order, a, s) != cudaSuccess) return ENOMR_ECUDA;
    return ENOMR_OK;
}
