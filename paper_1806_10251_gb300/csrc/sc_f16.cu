// Step kernel instantiations for the __half population storage.
#include "stream_collide.cuh"

namespace lbm {

cudaError_t launch_step_f16(const StepParams &p, const CUtensorMap &tin, const CUtensorMap &tout, const void *fin,
                           int grid, cudaStream_t s)
{
    return launch_step_t<__half>(p, tin, tout, fin, grid, s);
}

cudaError_t launch_batch_f16(int gi_mode, const BatchArgs &a, int grid, cudaStream_t s)
{
    return launch_batch_t<__half>(gi_mode, a, grid, s);
}

int batch_blocks_f16(int gi_mode) { return batch_blocks_t<__half>(gi_mode); }

int blocks_per_sm_f16(int gi_mode) { return blocks_per_sm_t<__half>(gi_mode); }

}  // namespace lbm
