// h2_selftest.cu -- self-tests and measurements of the device (no paper counterpart).
//
// 1. Bounded device waits. Every wait of the pipelined kernels is bounded: after a budget of
//    clock cycles without progress the waiting thread records the failure in a device flag and
//    returns, so a stalled pipeline ends its kernel instead of hanging the GPU. The self-test
//    exercises that path on purpose and harmlessly: one thread waits on a shared-memory barrier
//    nothing arrives on, with a short budget, and the host reads the flag. The warp sweeps'
//    waits on node flags in global memory are exercised the same way: two warps wait on flags
//    nothing sets; the first gives up after the budget and raises the launch's abort word, and
//    the second, whose own budget is fifty times longer, must leave on that abort word.
// 2. Arithmetic peaks. The FP64 product is bound by the FP64 fused multiply-add rate, the FP32
//    multi-vector product on the CUDA cores by the FP32 one, and the matrix-free product by the
//    special-function unit; their rooflines need those rates as this device delivers them, not
//    as a datasheet states them. Each is measured with register-resident chains of one
//    instruction kind (32 warps per SM, every SM busy), timed with CUDA events around the
//    launch after a calibration run; nothing else runs in the kernel, and the chains' results
//    feed a store the compiler cannot prove dead.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/h2.h"
#include "h2_pipe.cuh"
#include "h2_warpsweep.cuh"

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

// words[0], words[1]: the two warps' node flags (never set); words[2]: the abort word.
// waited[0]: clock cycles the second warp waited.
__global__ void k_flag_wait_timeout(long long budget, int *words, int *err, long long *waited)
{
    const int warp = threadIdx.x / 32;
    const long long t0 = clock64();
    (void)h2s::ws_wait_for(words + warp, words + 2, err, warp == 0 ? budget : 50 * budget);
    if (warp == 1 && (threadIdx.x & 31) == 0) waited[0] = clock64() - t0;
}

constexpr int kChains = 8;  // ex2 chains per thread
constexpr int kFmaChains = 4;
constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSm = 4;

// Two forms of FMA chains, 128 FMAs per thread per iteration; each unit's rate is the faster
// of the two (on this part the FP64 pipe reaches its full rate only with the first form, the
// FP32 pipe only with the second):
//   FORM 0: a_j <- b_{(j+u) mod 4} * c_j + a_j on four accumulators whose multiplicands rotate
//           through distinct registers;
//   FORM 1: a_j <- a_j * m + c on eight chains that share m and c.
template <typename T, int FORM>
__global__ void __launch_bounds__(kPeakThreads) k_fma_chains(int iters, const T *__restrict__ in, T *sink)
{
    constexpr int NA = FORM == 0 ? kFmaChains : kChains;
    T a[NA], b[kFmaChains], c[kFmaChains];
#pragma unroll
    for (int j = 0; j < kFmaChains; ++j) {
        b[j] = in[j];
        c[j] = in[kFmaChains + j];
    }
#pragma unroll
    for (int j = 0; j < NA; ++j) a[j] = FORM == 0 ? T(0) : T(threadIdx.x + j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 128 / NA; ++u) {
#pragma unroll
            for (int j = 0; j < NA; ++j) {
                const T x = FORM == 0 ? b[(j + u) & 3] : a[j];
                const T y = FORM == 0 ? c[j] : T(1) - b[0];  // 1 - 1e-3: the chains decay
                const T z = FORM == 0 ? a[j] : c[0];
                if constexpr (sizeof(T) == 8)
                    a[j] = __fma_rn(x, y, z);
                else
                    a[j] = __fmaf_rn(x, y, z);
            }
        }
    }
    T s = T(0);
#pragma unroll
    for (int j = 0; j < NA; ++j) s += a[j];
    if (s == T(-1)) sink[blockIdx.x] = s;  // never true for these inputs; keeps the chains live
}

// a <- 2^(-a) on kChains chains through the special-function unit (one ex2 per step);
// 128 evaluations per thread per iteration.
__global__ void __launch_bounds__(kPeakThreads) k_ex2_chains(int iters, float *sink)
{
    float a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = 0.25f + 0.01f * float((threadIdx.x + j) & 31);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int j = 0; j < kChains; ++j) asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(a[j]) : "f"(-a[j]));
        }
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    if (s == -1.f) sink[blockIdx.x] = s;
}

// One timed launch (ms) of unit's chains with `iters` outer iterations. `in` holds the FMA
// multiplicands: 8 doubles, then 8 floats.
cudaError_t launch_chains(int unit, int form, int grid, int iters, const void *in, void *sink, float *ms)
{
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess) e = cudaEventRecord(a, 0);
    if (e == cudaSuccess) {
        const double *din = static_cast<const double *>(in);
        const float *fin = reinterpret_cast<const float *>(din + 8);
        if (unit == H2_PEAK_DFMA && form == 0)
            k_fma_chains<double, 0><<<grid, kPeakThreads>>>(iters, din, static_cast<double *>(sink));
        else if (unit == H2_PEAK_DFMA)
            k_fma_chains<double, 1><<<grid, kPeakThreads>>>(iters, din, static_cast<double *>(sink));
        else if (unit == H2_PEAK_FFMA && form == 0)
            k_fma_chains<float, 0><<<grid, kPeakThreads>>>(iters, fin, static_cast<float *>(sink));
        else if (unit == H2_PEAK_FFMA)
            k_fma_chains<float, 1><<<grid, kPeakThreads>>>(iters, fin, static_cast<float *>(sink));
        else
            k_ex2_chains<<<grid, kPeakThreads>>>(iters, static_cast<float *>(sink));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(b, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    return e;
}

}  // namespace

extern "C" int h2_selftest_wait_timeout(int64_t budget_cycles)
{
    if (budget_cycles < 1 || budget_cycles > 4000000000LL / 50) return H2_EINVAL;
    // [0] error flag of the barrier wait, [1] error flag of the flag waits, [2 .. 4] flags and
    // abort word, then the second warp's wait in cycles (8-byte aligned)
    int *buf = nullptr;
    if (cudaMalloc(&buf, 8 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return H2_ENOMEM;
    }
    int host[8] = {};
    long long waited = 0;
    long long *dwaited = reinterpret_cast<long long *>(buf + 6);
    cudaError_t e = cudaMemset(buf, 0, 8 * sizeof(int));
    if (e == cudaSuccess) {
        k_wait_timeout<<<1, 32>>>(budget_cycles, buf);
        k_flag_wait_timeout<<<1, 64>>>(budget_cycles, buf + 2, buf + 1, dwaited);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(host, buf, 6 * sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&waited, dwaited, sizeof(waited), cudaMemcpyDeviceToHost);
    cudaFree(buf);
    if (e != cudaSuccess) return H2_ECUDA;
    // both kinds of wait gave up and said so, and the second flag waiter left on the abort
    // word rather than on its own (fifty times longer) budget
    const bool flag_waits = host[1] && host[4] && waited < 10 * budget_cycles;
    return host[0] && flag_waits ? H2_ETIMEOUT : H2_OK;
}

extern "C" int h2_measure_peak(int unit, double target_ms, double *rate, double *ms)
{
    if (unit < H2_PEAK_DFMA || unit > H2_PEAK_EX2 || !rate || !(target_ms >= 1.0 && target_ms <= 1000.0))
        return H2_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        return H2_ECUDA;
    const int grid = sms * kPeakBlocksPerSm;
    void *sink = nullptr, *in = nullptr;
    if (cudaMalloc(&sink, size_t(grid) * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&in, 8 * sizeof(double) + 8 * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        if (sink) cudaFree(sink);
        return H2_ENOMEM;
    }
    // multiplicands of about 1e-3: the accumulators grow by about 1e-6 per step and stay far
    // from overflow and from the subnormal range
    double hin[8];
    float fin[8];
    for (int j = 0; j < 8; ++j) {
        hin[j] = 1e-3 * (1.0 + 0.125 * j);
        fin[j] = float(hin[j]);
    }
    cudaError_t e = cudaMemcpy(in, hin, sizeof(hin), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(static_cast<double *>(in) + 8, fin, sizeof(fin), cudaMemcpyHostToDevice);
    // per form: a short calibration run sets the iteration count that takes about target_ms,
    // then five timed launches; the rate is the best over forms and launches
    double best_rate = 0.0;
    float best_ms = 0.f;
    const int forms = unit == H2_PEAK_EX2 ? 1 : 2;
    for (int form = 0; e == cudaSuccess && form < forms; ++form) {
        int iters = unit == H2_PEAK_DFMA ? 64 : 2048;
        float t = 0.f;
        e = launch_chains(unit, form, grid, iters, in, sink, &t);  // also loads the module
        if (e == cudaSuccess) e = launch_chains(unit, form, grid, iters, in, sink, &t);
        if (e == cudaSuccess && t > 0.f)
            iters = int(std::min(2.0e9, std::max(1.0, double(iters) * target_ms / double(t))));
        const double ops = double(grid) * kPeakThreads * 128.0 * double(iters);
        for (int r = 0; e == cudaSuccess && r < 5; ++r) {
            e = launch_chains(unit, form, grid, iters, in, sink, &t);
            const double rate_r = (unit == H2_PEAK_EX2 ? ops : 2.0 * ops) / (double(t) * 1e-3);
            if (e == cudaSuccess && t > 0.f && rate_r > best_rate) {
                best_rate = rate_r;
                best_ms = t;
            }
        }
    }
    cudaFree(sink);
    cudaFree(in);
    if (e != cudaSuccess || best_rate <= 0.0) return H2_ECUDA;
    *rate = best_rate;
    if (ms) *ms = best_ms;
    return H2_OK;
}
