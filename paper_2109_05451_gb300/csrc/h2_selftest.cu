// h2_selftest.cu -- self-test of the bounded device waits (no paper counterpart).
//
// Every wait of the pipelined kernels is bounded: after a budget of clock cycles without
// progress the waiting thread records the failure in a device flag and returns, so a stalled
// pipeline ends its kernel instead of hanging the GPU. This entry point exercises that path on
// purpose and harmlessly: one thread waits on a shared-memory barrier nothing arrives on, with
// a short budget, and the host reads the flag.
#include <cuda_runtime.h>

#include "../../include/h2.h"
#include "h2_pipe.cuh"

namespace {

__global__ void k_wait_timeout(long long budget, int *err)
{
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        h2p::mbar_init(&bar, 1);
        abort_flag = 0;
        h2p::fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) h2p::mbar_wait_for(&bar, 0, &abort_flag, err, budget);  // no arrival ever comes
}

}  // namespace

extern "C" int h2_selftest_wait_timeout(int64_t budget_cycles)
{
    if (budget_cycles < 1 || budget_cycles > 4000000000LL) return H2_EINVAL;
    int *err = nullptr;
    if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return H2_ENOMEM;
    }
    int flag = 0;
    cudaError_t e = cudaMemset(err, 0, sizeof(int));
    if (e == cudaSuccess) {
        k_wait_timeout<<<1, 32>>>(budget_cycles, err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&flag, err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(err);
    if (e != cudaSuccess) return H2_ECUDA;
    return flag ? H2_ETIMEOUT : H2_OK;
}
