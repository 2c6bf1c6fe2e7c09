// Self-test of the device time-out path (swdft2d_selftest_wait_timeout): one thread waits on
// a shared-memory mbarrier that nothing arrives on, at most `polls` polls of at most about
// 1 ms each, and records the time-out in this file's device word, which
// swdft2d_check_device reads beside the tensor-core kernels' word.  No fault, no hang.
#include "sm100_ptx.cuh"
#include "swdft_internal.h"

namespace swdft {

__device__ int g_probe_status;  // 0 = ok; 1 = the self-test's wait timed out

__global__ void __launch_bounds__(32) wait_timeout_probe(uint32_t polls) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait(&bar, 0, polls)) atomicExch(&g_probe_status, 1);
}

cudaError_t launch_wait_timeout_probe(uint32_t polls, cudaStream_t s) {
    wait_timeout_probe<<<1, 32, 0, s>>>(polls);
    return cudaGetLastError();
}

cudaError_t probe_status(int *status, bool reset) {
    cudaError_t e = cudaMemcpyFromSymbol(status, g_probe_status, sizeof(int));
    if (e == cudaSuccess && reset) {
        const int zero = 0;
        e = cudaMemcpyToSymbol(g_probe_status, &zero, sizeof(int));
    }
    return e;
}

}  // namespace swdft
