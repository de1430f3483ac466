// h2_cgk.cuh -- device kernels of conjugate gradients on (A_H2 + sigma2 I) x = b, shared by
// the one-shot solver (h2_cg.cu) and the serving loop (h2_serve.cu), so both take the same
// arithmetic in the same order. Vectors and scalars are FP64. Inner products use a fixed
// two-stage reduction (a fixed number of blocks and a fixed summation order): a solve is
// bitwise repeatable and independent of what else runs on the GPU.
//
// Scalars live in a small device array scal: [0] r.r, [1] p.Ap, [2] r.r after the update,
// [3] b.b, [4] true residual |b - (A + sigma2 I) x|^2. The flagged update kernels skip their
// work once a device flag is set (converged or broken down), so iterations enqueued ahead of
// the host's convergence check leave x unchanged.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/h2.h"

namespace h2cg {
namespace {

constexpr int kDotBlocks = 256;
constexpr int kThreads = 256;

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return H2_OK;
    if (e == cudaErrorMemoryAllocation) return H2_ENOMEM;
    return H2_ECUDA;
}

// partial[b] = sum over block b's contiguous range of a[i] * c[i], in a fixed order.
__global__ void k_dot_partial(const double *__restrict__ a, const double *__restrict__ c, int64_t n,
                              double *__restrict__ partial)
{
    __shared__ double red[kThreads];
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = blockIdx.x * per, hi = lo + per < n ? lo + per : n;
    double s = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) s += a[i] * c[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w /= 2) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_dot_final(const double *__restrict__ partial, int nb, double *__restrict__ out)
{
    __shared__ double red[kThreads];
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += partial[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w /= 2) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

__global__ void k_to_float(const double *__restrict__ a, float *__restrict__ f, int64_t n)
{
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        f[i] = float(a[i]);
}

// Ap = A p + sigma2 p, from the product in float or double.
template <typename T>
__global__ void k_shift(const T *__restrict__ Ap_raw, const double *__restrict__ p, double sigma2,
                        double *__restrict__ Ap, int64_t n)
{
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        Ap[i] = double(Ap_raw[i]) + sigma2 * p[i];
}

// r = b - Ax
__global__ void k_residual(const double *__restrict__ b, const double *__restrict__ Ax, double *__restrict__ r,
                           double *__restrict__ p, int64_t n)
{
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const double v = b[i] - Ax[i];
        r[i] = v;
        if (p) p[i] = v;
    }
}

// alpha = rr / pAp; x += alpha p; r -= alpha Ap
__global__ void k_update_xr(double *__restrict__ x, double *__restrict__ r, const double *__restrict__ p,
                            const double *__restrict__ Ap, const double *__restrict__ scal, int64_t n)
{
    const double alpha = scal[0] / scal[1];
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        x[i] += alpha * p[i];
        r[i] -= alpha * Ap[i];
    }
}

// beta = rr_new / rr; p = r + beta p; then rr = rr_new
__global__ void k_update_p(double *__restrict__ p, const double *__restrict__ r, const double *__restrict__ scal,
                           int64_t n)
{
    const double beta = scal[2] / scal[0];
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        p[i] = r[i] + beta * p[i];
}

__global__ void k_copy_scalar(double *__restrict__ scal, int dst, int src) { scal[dst] = scal[src]; }


// Flagged variants for iterations enqueued ahead of the convergence check.
__global__ void k_update_xr_if(double *__restrict__ x, double *__restrict__ r, const double *__restrict__ p,
                                      const double *__restrict__ Ap, const double *__restrict__ scal,
                                      const int *__restrict__ flag, int64_t n)
{
    if (*flag) return;
    const double alpha = scal[0] / scal[1];
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        x[i] += alpha * p[i];
        r[i] -= alpha * Ap[i];
    }
}

__global__ void k_update_p_if(double *__restrict__ p, const double *__restrict__ r,
                                     const double *__restrict__ scal, const int *__restrict__ flag, int64_t n)
{
    if (*flag) return;
    const double beta = scal[2] / scal[0];
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        p[i] = r[i] + beta * p[i];
}

// One thread: after the update of an active iteration, count it and stop on
// sqrt(r.r / b.b) < tol (flag 1: converged) or a non-finite r.r (flag 2: breakdown) -- the
// same comparison, in the same order, as the host test of the one-shot solver.
__global__ void k_check(const double *__restrict__ scal, int *__restrict__ flag, int *__restrict__ iters, double tol)
{
    if (*flag) return;
    *iters += 1;
    const double rr = scal[2];
    if (!isfinite(rr)) *flag = 2;
    else if (sqrt(rr / scal[3]) < tol) *flag = 1;
}

// One thread: r.r <- the updated value (kept apart from k_update_p_if, whose blocks all read
// the old value).
__global__ void k_roll_if(double *__restrict__ scal, const int *__restrict__ flag)
{
    if (*flag) return;
    scal[0] = scal[2];
}

inline unsigned grid_for(int64_t n) { return unsigned(n / kThreads + 1 < 4096 ? n / kThreads + 1 : 4096); }

inline void dot(const double *a, const double *b, int64_t n, double *partial, double *out, cudaStream_t st)
{
    k_dot_partial<<<kDotBlocks, kThreads, 0, st>>>(a, b, n, partial);
    k_dot_final<<<1, kThreads, 0, st>>>(partial, kDotBlocks, out);
}

}  // namespace
}  // namespace h2cg
