// Convergence sums of a caller-owned population array without any device
// allocation: the reduction's scratch (one row of five partial sums per block
// and the five totals) is a fixed array in the library's own device memory.
//
// Who needs this: callers that cannot let a library call cudaMalloc while they
// run -- an application whose device memory is all handed out by its own pool
// or arena, a loop that must not pay (or risk failing) an allocation between
// steps, or code that records its work into a CUDA graph, where an allocation
// call cannot be recorded.  They pass their device buffers in and get the sums
// back in a device buffer of their own.
#include <math.h>
#include <string.h>

#include "lbm_internal.h"

namespace lbm {

namespace {

// Partial-sum rows: one 256-thread block per 256 cells writes one row of five
// sums, then one more block adds the rows into the caller's buffer.  The array
// holds LBM_NOALLOC_MAX_PARTIALS rows (2.5 MiB), hence at most
// LBM_NOALLOC_MAX_CELLS cells per call; every GPU that loads the library keeps
// it until the process exits.
constexpr int kRows = LBM_NOALLOC_MAX_PARTIALS;
constexpr int kCellsPerRow = 256;
static __device__ __align__(256) double g_scratch[(size_t)kRows * 5];

constexpr int kMaxDevices = 64;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

}  // namespace

}  // namespace lbm

using namespace lbm;

extern "C" lbm_status lbm_residual_sums_noalloc(const lbm_population_desc *d, const void *f_dev, double *snap_ux_dev,
                                                double *snap_uy_dev, double *sums_dev, void *stream)
{
    if (!d || !f_dev || !snap_ux_dev || !snap_uy_dev || !sums_dev)
        return set_error(LBM_ERR_INVALID, "lbm_residual_sums_noalloc: null argument");
    if (d->nx < 1 || d->ny < 1 || d->pitch < d->nx || d->storage < 0 || d->storage > 3 || !(d->gamma > 0.0))
        return set_error(LBM_ERR_INVALID, "lbm_residual_sums_noalloc: bad descriptor (nx, ny >= 1, pitch >= nx, "
                                          "storage 0..3, gamma > 0)");
    const long long cells = (long long)d->nx * d->ny;
    if (cells > LBM_NOALLOC_MAX_CELLS)
        return set_error(LBM_ERR_INVALID, "lbm_residual_sums_noalloc: nx*ny exceeds LBM_NOALLOC_MAX_CELLS "
                                          "(the fixed scratch holds 65536 partial rows of 256 cells)");

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return set_error(LBM_ERR_CUDA, "lbm_residual_sums_noalloc: no usable CUDA device");
    }
    // Set-up, once per device, with that device current: the device address of
    // the scratch array (its name in host code is only a host-side stand-in).
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return set_error(LBM_ERR_CUDA, "lbm_residual_sums_noalloc: cudaGetSymbolAddress failed");
        }
        g_scratch_ptr[dev] = static_cast<double *>(ptr);
    }
    double *partials = g_scratch_ptr[dev];

    StepParams p;
    memset(&p, 0, sizeof(p));
    p.nx = d->nx;
    p.ny = d->ny;
    p.pitch = d->pitch;
    p.plane = (long long)d->pitch * d->ny;
    p.gamma = d->gamma;
    p.Fx = d->fx;
    p.Fy = d->fy;
    p.solid = d->solid_dev;
    const int nblocks = (int)((cells + kCellsPerRow - 1) / kCellsPerRow);
    // every partial row is written before the second pass reads it: nothing in
    // the scratch has to start at zero
    cudaError_t e = launch_residual(p, d->storage, f_dev, snap_ux_dev, snap_uy_dev, partials, nblocks, sums_dev,
                                    (cudaStream_t)stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(LBM_ERR_CUDA, std::string("lbm_residual_sums_noalloc: ") + cudaGetErrorString(e));
    }
    return LBM_OK;
}
