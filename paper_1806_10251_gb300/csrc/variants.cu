// Definitions of the kernel-variant launchers declared in variants.h.
//
// Built once per (LBM_VARIANT_STORAGE, LBM_VARIANT_PART) by build.py: the
// storage type selects the kernel family (packed two-cells-per-lane kernels for
// FP32/FP16/BF16, the one-cell-per-lane kernel for FP64) and the part selects
// which group of variants this object instantiates (parts 0-3: step and batch
// kernels; part 4, packed storages only: the persistent batch kernel).  Every
// variant is instantiated in exactly one part.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "variants.h"

#ifndef LBM_VARIANT_STORAGE
#define LBM_VARIANT_STORAGE 0
#endif
#ifndef LBM_VARIANT_PART
#define LBM_VARIANT_PART 0
#endif

#if LBM_VARIANT_STORAGE == 3
#include "stream_collide.cuh"
#else
#include "stream_collide_x2.cuh"
#endif

namespace lbm {

#if LBM_VARIANT_STORAGE == 3
// FP64 storage: one cell per lane, staged TMA stores (tout), guard at run time.
template <typename ST, int MODE, bool FORCED, bool GUARD, bool ISO>
cudaError_t step_variant_launch(const StepParams &p, const CUtensorMap &tin, const CUtensorMap &tout,
                                const void *fin, void *, int grid, cudaStream_t s)
{
    stream_collide_kernel<ST, MODE, FORCED, ISO><<<grid, THREADS, Tile<ST>::SMEM_BYTES, s>>>(
        p, tin, tout, static_cast<const ST *>(fin));
    return cudaGetLastError();
}

template <typename KernelFn>
static int occupancy_of(KernelFn fn, int smem)
{
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, THREADS, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

template <typename ST, int MODE, bool FORCED, bool GUARD, bool ISO>
int step_variant_blocks()
{
    return occupancy_of(stream_collide_kernel<ST, MODE, FORCED, ISO>, Tile<ST>::SMEM_BYTES);
}

template <typename ST, int MODE, bool FORCED>
cudaError_t batch_variant_launch(const BatchArgs &a, int grid, cudaStream_t s)
{
    stream_collide_batch_kernel<ST, MODE, FORCED><<<grid, THREADS, Tile<ST>::SMEM_BYTES, s>>>(a);
    return cudaGetLastError();
}

template <typename ST, int MODE, bool FORCED>
int batch_variant_blocks()
{
    return occupancy_of(stream_collide_batch_kernel<ST, MODE, FORCED>, Tile<ST>::SMEM_BYTES);
}
using VST = double;
#else
// FP32 / FP16 / BF16 storage: two cells per lane, stores straight from registers.
template <typename ST, int MODE, bool FORCED, bool GUARD, bool ISO>
cudaError_t step_variant_launch(const StepParams &p, const CUtensorMap &tin, const CUtensorMap &,
                                const void *fin, void *fout, int grid, cudaStream_t s)
{
    stream_collide_x2_kernel<ST, MODE, FORCED, GUARD, ISO><<<grid, THREADS, Tile2<ST>::SMEM_BYTES, s>>>(
        p, tin, static_cast<const ST *>(fin), static_cast<ST *>(fout));
    return cudaGetLastError();
}

template <typename ST, int MODE, bool FORCED, bool GUARD, bool ISO>
int step_variant_blocks()
{
    return occupancy_of(stream_collide_x2_kernel<ST, MODE, FORCED, GUARD, ISO>, Tile2<ST>::SMEM_BYTES);
}

template <typename ST, int MODE, bool FORCED>
cudaError_t batch_variant_launch(const BatchArgs &a, int grid, cudaStream_t s)
{
    stream_collide_x2_batch_kernel<ST, MODE, FORCED><<<grid, THREADS, Tile2<ST>::SMEM_BYTES, s>>>(a);
    return cudaGetLastError();
}

template <typename ST, int MODE, bool FORCED>
int batch_variant_blocks()
{
    return occupancy_of(stream_collide_x2_batch_kernel<ST, MODE, FORCED>, Tile2<ST>::SMEM_BYTES);
}

template <typename ST, bool FORCED>
cudaError_t batch_persistent_variant_launch(const BatchArgs &a, int k0, int nsteps, int grid, cudaStream_t s)
{
    void *args[] = {const_cast<BatchArgs *>(&a), &k0, &nsteps};
    return cudaLaunchCooperativeKernel(
        reinterpret_cast<const void *>(&stream_collide_x2_batch_persistent_kernel<ST, LBM_GI_FULL, FORCED>), grid,
        THREADS, args, Tile2<ST>::SMEM_BYTES, s);
}

template <typename ST, bool FORCED>
int batch_persistent_variant_blocks()
{
    return occupancy_of(stream_collide_x2_batch_persistent_kernel<ST, LBM_GI_FULL, FORCED>, Tile2<ST>::SMEM_BYTES);
}
#if LBM_VARIANT_STORAGE == 1
using VST = __half;
#elif LBM_VARIANT_STORAGE == 2
using VST = __nv_bfloat16;
#else
using VST = float;
#endif
#endif

#define LBM_STEP_VARIANT(M, F, G, I)                                                                           \
    template cudaError_t step_variant_launch<VST, M, F, G, I>(const StepParams &, const CUtensorMap &,        \
                                                              const CUtensorMap &, const void *, void *, int,   \
                                                              cudaStream_t);                                    \
    template int step_variant_blocks<VST, M, F, G, I>();
#define LBM_BATCH_VARIANT(M, F)                                                                                \
    template cudaError_t batch_variant_launch<VST, M, F>(const BatchArgs &, int, cudaStream_t);               \
    template int batch_variant_blocks<VST, M, F>();

constexpr int U_ = LBM_GI_UNCORRECTED, C_ = LBM_GI_CUBIC_ONLY, F_ = LBM_GI_FULL;

#if LBM_VARIANT_PART == 0
LBM_STEP_VARIANT(U_, false, false, false)
LBM_STEP_VARIANT(U_, true, false, false)
LBM_STEP_VARIANT(C_, false, false, false)
LBM_STEP_VARIANT(C_, true, false, false)
#elif LBM_VARIANT_PART == 1
LBM_STEP_VARIANT(F_, false, false, false)
LBM_STEP_VARIANT(F_, true, false, false)
#if LBM_VARIANT_STORAGE == 3
LBM_STEP_VARIANT(F_, false, false, true)
LBM_STEP_VARIANT(F_, true, false, true)
#else
LBM_STEP_VARIANT(F_, false, true, false)
LBM_STEP_VARIANT(F_, true, true, false)
#endif
#elif LBM_VARIANT_PART == 2
#if LBM_VARIANT_STORAGE != 3
LBM_STEP_VARIANT(F_, false, true, true)
LBM_STEP_VARIANT(F_, true, true, true)
#endif
LBM_BATCH_VARIANT(U_, false)
LBM_BATCH_VARIANT(U_, true)
#elif LBM_VARIANT_PART == 3
LBM_BATCH_VARIANT(C_, false)
LBM_BATCH_VARIANT(C_, true)
LBM_BATCH_VARIANT(F_, false)
LBM_BATCH_VARIANT(F_, true)
#elif LBM_VARIANT_STORAGE != 3
// part 4 (packed storages only): the persistent batch kernel
template cudaError_t batch_persistent_variant_launch<VST, false>(const BatchArgs &, int, int, int, cudaStream_t);
template cudaError_t batch_persistent_variant_launch<VST, true>(const BatchArgs &, int, int, int, cudaStream_t);
template int batch_persistent_variant_blocks<VST, false>();
template int batch_persistent_variant_blocks<VST, true>();
#endif

}  // namespace lbm
