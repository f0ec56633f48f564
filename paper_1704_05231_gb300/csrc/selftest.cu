// Failure-detection self-test: the bounded mbarrier wait of the tensor-core kernels, run on
// a barrier that is (or is not) signalled, so the timeout path can be exercised on a GPU
// without a hang: the wait gives up, records a code in the handle's status word, returns.
#include "internal.h"
#include "tc_common.cuh"

namespace gb {

constexpr int kSelftestTimeoutCode = 90;

__global__ void k_wait_selftest(int *status, int signal, unsigned long long limit_ns)
{
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (signal) mbar_arrive(&bar);
        if (!mbar_wait_for(&bar, 0, &abort_flag, limit_ns)) atomicExch(status, kSelftestTimeoutCode);
    }
    __syncthreads();
}

cudaError_t launch_wait_selftest(int *status, int signal, unsigned long long limit_ns, cudaStream_t st)
{
    k_wait_selftest<<<1, 32, 0, st>>>(status, signal, limit_ns);
    return cudaGetLastError();
}

}  // namespace gb
