// Step kernel instantiations for the double population storage.
#include "stream_collide.cuh"

namespace lbm {

cudaError_t launch_step_f64(const StepParams &p, const CUtensorMap &tin, const CUtensorMap &tout, const void *fin,
                           void *, int grid, cudaStream_t s)
{
    return launch_step_t<double>(p, tin, tout, fin, grid, s);
}

cudaError_t launch_batch_f64(int gi_mode, bool forced, const BatchArgs &a, int grid, cudaStream_t s)
{
    return launch_batch_t<double>(gi_mode, forced, a, grid, s);
}

int batch_blocks_f64(int gi_mode, bool forced) { return batch_blocks_t<double>(gi_mode, forced); }

int blocks_per_sm_f64(int gi_mode, bool forced) { return blocks_per_sm_t<double>(gi_mode, forced); }

}  // namespace lbm
