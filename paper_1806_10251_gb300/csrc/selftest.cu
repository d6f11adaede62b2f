// Self-test of the failure path of the bounded waits (the paper has no
// counterpart).  Every mbarrier wait of the step kernels gives up after a time
// limit, raises the context's device error flag and lets its warp return, so a
// lost copy ends the launch with an error status instead of a hang.  This
// kernel drives that path on purpose without any fault: one thread initialises
// an mbarrier that expects one arrival, nothing ever arrives, and the thread
// waits on it with the step kernels' own bounded wait (mbar_wait_bounded, same
// limit), then raises the flag exactly as a step kernel does.
#include "stream_collide.cuh"

namespace lbm {

__global__ void bounded_wait_selftest_kernel(int *error, unsigned long long *waited_ns)
{
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x == 0) {
        const uint32_t b = smem_u32(&bar);
        mbar_init(b, 1);
        fence_mbar_init();
        const unsigned long long t0 = globaltimer();
        // phase 0 of a fresh barrier never completes: the wait runs to its limit
        if (!mbar_wait_bounded(b, 0u)) atomicExch(error, 1);
        *waited_ns = globaltimer() - t0;
    }
}

cudaError_t launch_bounded_wait_selftest(int *error, unsigned long long *waited_ns, cudaStream_t s)
{
    bounded_wait_selftest_kernel<<<1, 32, 0, s>>>(error, waited_ns);
    return cudaGetLastError();
}

}  // namespace lbm
