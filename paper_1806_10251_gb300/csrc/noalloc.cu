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
#include <cudaTypedefs.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "lbm_internal.h"

namespace lbm {

namespace {

// Partial-sum rows: each block of the first pass takes lattice rows with a
// stride of the grid size (the grid of lbm_residual: one block per row, at most
// 1024) and writes one row of five sums; one more block adds the rows into the
// caller's buffer.  The array holds LBM_NOALLOC_MAX_PARTIALS rows (2.5 MiB);
// every GPU that loads the library keeps it until the process exits.
constexpr int kRows = LBM_NOALLOC_MAX_PARTIALS;
static __device__ __align__(256) double g_scratch[(size_t)kRows * 5];

// Device address of g_scratch per device, with the id of the CUDA context it
// was looked up in (a cudaDeviceReset ends that context; the next call then
// looks the address up again).  Filled under a mutex, so first calls from
// several host threads at once are safe.
constexpr int kMaxDevices = 64;
struct ScratchSlot {
    unsigned long long ctx_id;
    double *ptr;
};
std::mutex g_scratch_mu;
ScratchSlot g_scratch_slot[kMaxDevices] = {};

template <typename Fn>
Fn driver_fn(const char *name)
{
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return reinterpret_cast<Fn>(f);
}

// Id of the calling thread's current context (false if there is none or the
// driver does not provide the calls).
bool current_context_id(unsigned long long *id)
{
    static const PFN_cuCtxGetCurrent_v4000 get_current = driver_fn<PFN_cuCtxGetCurrent_v4000>("cuCtxGetCurrent");
    static const PFN_cuCtxGetId_v12000 get_id = driver_fn<PFN_cuCtxGetId_v12000>("cuCtxGetId");
    CUcontext c = nullptr;
    if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c) return false;
    return get_id(c, id) == CUDA_SUCCESS;
}

// The device address of g_scratch on device dev (current), looked up once per
// context with that device current: in host code the array's name is only a
// host-side stand-in, which a kernel must never be given.
cudaError_t scratch_address(int dev, double **out)
{
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    unsigned long long id = 0;
    bool have_id = current_context_id(&id);
    ScratchSlot &slot = g_scratch_slot[dev];
    if (slot.ptr && have_id && slot.ctx_id == id) {
        *out = slot.ptr;
        return cudaSuccess;
    }
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
    if (e != cudaSuccess || !ptr) {
        cudaGetLastError();
        return e != cudaSuccess ? e : cudaErrorInvalidSymbol;
    }
    if (!have_id) have_id = current_context_id(&id);  // the lookup made the context current
    slot.ctx_id = have_id ? id : 0;
    slot.ptr = have_id ? static_cast<double *>(ptr) : nullptr;  // no id: look up on every call
    *out = static_cast<double *>(ptr);
    return cudaSuccess;
}

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
                                          "(16777216 cells), the largest domain this entry point accepts");

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return set_error(LBM_ERR_CUDA, "lbm_residual_sums_noalloc: no usable CUDA device");
    }
    // set-up, once per device and context, with that device current
    double *partials = nullptr;
    if (scratch_address(dev, &partials) != cudaSuccess)
        return set_error(LBM_ERR_CUDA, "lbm_residual_sums_noalloc: cudaGetSymbolAddress failed");

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
    const int nblocks = residual_blocks(p);
    static_assert(1024 <= kRows, "the residual grid fits the scratch rows");
    // every partial row of the launch is written before the second pass reads
    // it: nothing in the scratch has to start at zero
    cudaError_t e = launch_residual(p, d->storage, f_dev, snap_ux_dev, snap_uy_dev, partials, nblocks, sums_dev,
                                    (cudaStream_t)stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(LBM_ERR_CUDA, std::string("lbm_residual_sums_noalloc: ") + cudaGetErrorString(e));
    }
    return LBM_OK;
}
