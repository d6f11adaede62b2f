// Run-time choice of the step- and batch-kernel variant for a launch (the
// variants themselves are compiled in variants.cu).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "variants.h"

namespace lbm {

namespace {

bool is_forced(const StepParams &p) { return p.force != nullptr || p.Fx != 0.0 || p.Fy != 0.0; }

// FP64 storage carries the guard as a run-time flag (no GUARD variants).
template <typename ST> constexpr bool has_guard_variants() { return sizeof(ST) != 8; }

template <typename ST, int MODE>
cudaError_t step_mode(bool forced, const StepParams &p, const CUtensorMap &tin, const CUtensorMap &tout,
                      const void *fin, void *fout, int grid, cudaStream_t s)
{
    return forced ? step_variant_launch<ST, MODE, true, false, false>(p, tin, tout, fin, fout, grid, s)
                  : step_variant_launch<ST, MODE, false, false, false>(p, tin, tout, fin, fout, grid, s);
}

template <typename ST>
cudaError_t launch_step_t(const StepParams &p, const CUtensorMap &tin, const CUtensorMap &tout, const void *fin,
                          void *fout, int grid, cudaStream_t s)
{
    constexpr bool G = has_guard_variants<ST>();
    const bool forced = is_forced(p);
    if (p.fd_iso && p.gi_mode == LBM_GI_FULL) {
        // the density gradient enters the full kernel only; the isotropic
        // variant carries the guard and leaves it to the context's flag
        return forced ? step_variant_launch<ST, LBM_GI_FULL, true, G, true>(p, tin, tout, fin, fout, grid, s)
                      : step_variant_launch<ST, LBM_GI_FULL, false, G, true>(p, tin, tout, fin, fout, grid, s);
    }
    if (G && p.guard && p.gi_mode == LBM_GI_FULL) {
        // the guard acts in the full kernel only (the strain solve)
        return forced ? step_variant_launch<ST, LBM_GI_FULL, true, G, false>(p, tin, tout, fin, fout, grid, s)
                      : step_variant_launch<ST, LBM_GI_FULL, false, G, false>(p, tin, tout, fin, fout, grid, s);
    }
    switch (p.gi_mode) {
    case LBM_GI_UNCORRECTED: return step_mode<ST, LBM_GI_UNCORRECTED>(forced, p, tin, tout, fin, fout, grid, s);
    case LBM_GI_CUBIC_ONLY: return step_mode<ST, LBM_GI_CUBIC_ONLY>(forced, p, tin, tout, fin, fout, grid, s);
    default: return step_mode<ST, LBM_GI_FULL>(forced, p, tin, tout, fin, fout, grid, s);
    }
}

int min3(int a, int b, int c) { return a < b ? (a < c ? a : c) : (b < c ? b : c); }

// Resident blocks per SM of the step-kernel variant a launch with these
// settings uses; for the full kernel, the minimum over its guard and
// isotropic-gradient variants, which get their shared-memory attribute too.
template <typename ST>
int blocks_per_sm_t(int gi_mode, bool forced)
{
    constexpr bool G = has_guard_variants<ST>();
    switch (gi_mode) {
    case LBM_GI_UNCORRECTED:
        return forced ? step_variant_blocks<ST, LBM_GI_UNCORRECTED, true, false, false>()
                      : step_variant_blocks<ST, LBM_GI_UNCORRECTED, false, false, false>();
    case LBM_GI_CUBIC_ONLY:
        return forced ? step_variant_blocks<ST, LBM_GI_CUBIC_ONLY, true, false, false>()
                      : step_variant_blocks<ST, LBM_GI_CUBIC_ONLY, false, false, false>();
    default:
        if (forced)
            return min3(step_variant_blocks<ST, LBM_GI_FULL, true, false, false>(),
                        step_variant_blocks<ST, LBM_GI_FULL, true, G, false>(),
                        step_variant_blocks<ST, LBM_GI_FULL, true, G, true>());
        return min3(step_variant_blocks<ST, LBM_GI_FULL, false, false, false>(),
                    step_variant_blocks<ST, LBM_GI_FULL, false, G, false>(),
                    step_variant_blocks<ST, LBM_GI_FULL, false, G, true>());
    }
}

template <typename ST>
cudaError_t launch_batch_t(int gi_mode, bool forced, const BatchArgs &a, int grid, cudaStream_t s)
{
    switch (gi_mode) {
    case LBM_GI_UNCORRECTED:
        return forced ? batch_variant_launch<ST, LBM_GI_UNCORRECTED, true>(a, grid, s)
                      : batch_variant_launch<ST, LBM_GI_UNCORRECTED, false>(a, grid, s);
    case LBM_GI_CUBIC_ONLY:
        return forced ? batch_variant_launch<ST, LBM_GI_CUBIC_ONLY, true>(a, grid, s)
                      : batch_variant_launch<ST, LBM_GI_CUBIC_ONLY, false>(a, grid, s);
    default:
        return forced ? batch_variant_launch<ST, LBM_GI_FULL, true>(a, grid, s)
                      : batch_variant_launch<ST, LBM_GI_FULL, false>(a, grid, s);
    }
}

template <typename ST>
int batch_blocks_t(int gi_mode, bool forced)
{
    switch (gi_mode) {
    case LBM_GI_UNCORRECTED:
        return forced ? batch_variant_blocks<ST, LBM_GI_UNCORRECTED, true>()
                      : batch_variant_blocks<ST, LBM_GI_UNCORRECTED, false>();
    case LBM_GI_CUBIC_ONLY:
        return forced ? batch_variant_blocks<ST, LBM_GI_CUBIC_ONLY, true>()
                      : batch_variant_blocks<ST, LBM_GI_CUBIC_ONLY, false>();
    default:
        return forced ? batch_variant_blocks<ST, LBM_GI_FULL, true>() : batch_variant_blocks<ST, LBM_GI_FULL, false>();
    }
}

}  // namespace

#define LBM_STORAGE_ENTRY(TAG, ST)                                                                             \
    cudaError_t launch_step_##TAG(const StepParams &p, const CUtensorMap &tin, const CUtensorMap &tout,       \
                                  const void *fin, void *fout, int grid, cudaStream_t s)                       \
    {                                                                                                          \
        return launch_step_t<ST>(p, tin, tout, fin, fout, grid, s);                                            \
    }                                                                                                          \
    int blocks_per_sm_##TAG(int gi_mode, bool forced) { return blocks_per_sm_t<ST>(gi_mode, forced); }         \
    cudaError_t launch_batch_##TAG(int gi_mode, bool forced, const BatchArgs &a, int grid, cudaStream_t s)    \
    {                                                                                                          \
        return launch_batch_t<ST>(gi_mode, forced, a, grid, s);                                                \
    }                                                                                                          \
    int batch_blocks_##TAG(int gi_mode, bool forced) { return batch_blocks_t<ST>(gi_mode, forced); }

LBM_STORAGE_ENTRY(f32, float)
LBM_STORAGE_ENTRY(f16, __half)
LBM_STORAGE_ENTRY(bf16, __nv_bfloat16)
LBM_STORAGE_ENTRY(f64, double)

bool batch_persistent_supported(int storage, int gi_mode)
{
    return storage != LBM_STORAGE_F64 && gi_mode == LBM_GI_FULL;
}

cudaError_t launch_batch_persistent(int storage, bool forced, const BatchArgs &a, int k0, int nsteps, int grid,
                                    cudaStream_t s)
{
#define LBM_PERSISTENT(ST) \
    (forced ? batch_persistent_variant_launch<ST, true>(a, k0, nsteps, grid, s) \
            : batch_persistent_variant_launch<ST, false>(a, k0, nsteps, grid, s))
    switch (storage) {
    case LBM_STORAGE_F16: return LBM_PERSISTENT(__half);
    case LBM_STORAGE_BF16: return LBM_PERSISTENT(__nv_bfloat16);
    case LBM_STORAGE_F32: return LBM_PERSISTENT(float);
    default: return cudaErrorNotSupported;
    }
#undef LBM_PERSISTENT
}

int batch_persistent_blocks_per_sm(int storage, bool forced)
{
    switch (storage) {
    case LBM_STORAGE_F16:
        return forced ? batch_persistent_variant_blocks<__half, true>() : batch_persistent_variant_blocks<__half, false>();
    case LBM_STORAGE_BF16:
        return forced ? batch_persistent_variant_blocks<__nv_bfloat16, true>()
                      : batch_persistent_variant_blocks<__nv_bfloat16, false>();
    case LBM_STORAGE_F32:
        return forced ? batch_persistent_variant_blocks<float, true>() : batch_persistent_variant_blocks<float, false>();
    default: return 0;
    }
}

}  // namespace lbm
