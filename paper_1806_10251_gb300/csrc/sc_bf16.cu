// Step kernel instantiations for the __nv_bfloat16 population storage.
#include "stream_collide.cuh"

namespace lbm {

cudaError_t launch_step_bf16(const StepParams &p, const CUtensorMap &tin, const CUtensorMap &tout, const void *fin,
                           int grid, cudaStream_t s)
{
    return launch_step_t<__nv_bfloat16>(p, tin, tout, fin, grid, s);
}

cudaError_t launch_batch_bf16(int gi_mode, const BatchArgs &a, int grid, cudaStream_t s)
{
    return launch_batch_t<__nv_bfloat16>(gi_mode, a, grid, s);
}

int batch_blocks_bf16(int gi_mode) { return batch_blocks_t<__nv_bfloat16>(gi_mode); }

int blocks_per_sm_bf16(int gi_mode) { return blocks_per_sm_t<__nv_bfloat16>(gi_mode); }

}  // namespace lbm
