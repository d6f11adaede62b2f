// Step kernel instantiations for the __nv_bfloat16 population storage (two cells per lane).
#include "stream_collide_x2.cuh"

namespace lbm {

cudaError_t launch_step_bf16(const StepParams &p, const CUtensorMap &tin, const CUtensorMap &, const void *fin,
                           void *fout, int grid, cudaStream_t s)
{
    return launch_step_x2_t<__nv_bfloat16>(p, tin, fin, fout, grid, s);
}

cudaError_t launch_batch_bf16(int gi_mode, bool forced, const BatchArgs &a, int grid, cudaStream_t s)
{
    return launch_batch_x2_t<__nv_bfloat16>(gi_mode, forced, a, grid, s);
}

int batch_blocks_bf16(int gi_mode, bool forced) { return batch_blocks_x2_t<__nv_bfloat16>(gi_mode, forced); }

int blocks_per_sm_bf16(int gi_mode, bool forced) { return blocks_per_sm_x2_t<__nv_bfloat16>(gi_mode, forced); }

}  // namespace lbm
