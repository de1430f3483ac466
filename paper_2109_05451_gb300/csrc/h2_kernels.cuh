// h2_kernels.cuh -- generation of the coupling and dense blocks on the device (h2_upload).
//
// The paper populates the matrix-tree entries on each GPU (Sec. 2.2): coupling blocks
// from the kernel at the clusters' Chebyshev points (Sec. 6.3) and dense blocks by
// evaluating the kernel directly (Sec. 6.4). Entries are evaluated in FP64 and rounded
// once to the storage type T. Both block kinds are stored transposed (output index
// contiguous) for the product kernels.
#pragma once

#include <cstdint>

#include <cuda_bf16.h>

#include "../../include/h2.h"
#include "h2_tc.cuh"

namespace h2k {

// ------------------------------------------------------------------ kernel function

struct KernelFn {
    int kind;
    double a, b;
    int deg;
};

__device__ __forceinline__ double kernel_eval(const KernelFn &f, const double *x, const double *y, int dim)
{
    if (f.kind == H2_K_POLY) {
        double v = 1.0;
        for (int d = 0; d < dim; ++d) {
            const double g = 1.0 + x[d] * y[d];
            for (int e = 0; e < f.deg; ++e) v *= g;
        }
        return v;
    }
    double r2 = 0.0;
    for (int d = 0; d < dim; ++d) {
        const double dx = x[d] - y[d];
        r2 += dx * dx;
    }
    if (f.kind == H2_K_EXP) return exp(-sqrt(r2) / f.a);
    if (f.kind == H2_K_GAUSS) return exp(-r2 / f.a);
    return pow(r2 + f.a, -f.b);
}

// ---------------------------------------------------- block generation (h2_upload)

// Coupling blocks S_ts[nu][mu] = kappa(xi^t_nu, xi^s_mu), evaluated in FP64, stored
// transposed in T (entry (nu, mu) at mu*k + nu), block b at b*kkp. One CTA per block
// (grid-stride over blocks).
template <typename T>
__global__ void gen_coupling(T *__restrict__ S, const int32_t *__restrict__ row, const int32_t *__restrict__ col,
                             int64_t nblocks, const double *__restrict__ cheb, int dim, int p, int k, int kx,
                             KernelFn f)
{
    // S_ts stored transposed, [mu][nu] with ld kx (nu fastest, zero for k <= nu < kx)
    const int64_t bs = int64_t(k) * kx;
    for (int64_t b = blockIdx.x; b < nblocks; b += gridDim.x) {
        const int64_t t = row[b], s = col[b];
        for (int64_t e = threadIdx.x; e < bs; e += blockDim.x) {
            const int nu = int(e % kx), mu = int(e / kx);
            double v = 0.0;
            if (nu < k) {
                double xt[3], xs[3];
                int rn = nu, rm = mu;
                for (int d = 0; d < dim; ++d) {
                    xt[d] = cheb[(t * dim + d) * p + rn % p];
                    xs[d] = cheb[(s * dim + d) * p + rm % p];
                    rn /= p;
                    rm /= p;
                }
                v = kernel_eval(f, xt, xs, dim);
            }
            S[b * bs + e] = T(v);
        }
    }
}

// Dense blocks D_ts[i][j] = kappa(x_i, x_j), stored transposed: [j][i] with ld = rows rounded
// up to 4 (i fastest, zero for rows <= i < ld).
template <typename T>
__global__ void gen_dense(T *__restrict__ D, const int64_t *__restrict__ off, const int32_t *__restrict__ row,
                          const int32_t *__restrict__ col, int64_t nblocks, const int32_t *__restrict__ leaf_lo,
                          const double *__restrict__ pts_tree, int dim, KernelFn f)
{
    for (int64_t b = blockIdx.x; b < nblocks; b += gridDim.x) {
        const int t = row[b], s = col[b];
        const int r0 = leaf_lo[t], rt = leaf_lo[t + 1] - r0;
        const int c0 = leaf_lo[s], cs = leaf_lo[s + 1] - c0;
        const int ld = (rt + 3) / 4 * 4;
        const int64_t cnt = int64_t(ld) * cs;
        for (int64_t e = threadIdx.x; e < cnt; e += blockDim.x) {
            const int i = int(e % ld), j = int(e / ld);
            D[off[b] + e] = i < rt ? T(kernel_eval(f, pts_tree + int64_t(r0 + i) * dim, pts_tree + int64_t(c0 + j) * dim, dim))
                                   : T(0);
        }
    }
}


// Split-BF16 tiles for the tensor-core path: block b as a 64 x 64 K-major tile (rows = output
// index, K = input index, zero-padded), hi = bf16(v) at tile + offset, lo = bf16(v - hi) at
// tile + 8192 + offset, 128-byte swizzled. Coupling: row nu, column mu = S_ts[nu][mu].
__device__ __forceinline__ void put_split(unsigned char *tile, int r, int c, double v)
{
    const float f = float(v);
    const __nv_bfloat16 hi = __float2bfloat16_rn(f);
    const __nv_bfloat16 lo = __float2bfloat16_rn(float(v - double(__bfloat162float(hi))));
    const uint32_t o = h2t::sw128_offset(r, c);
    *reinterpret_cast<__nv_bfloat16 *>(tile + o) = hi;
    *reinterpret_cast<__nv_bfloat16 *>(tile + 8192 + o) = lo;
}

__global__ void gen_coupling_tc(unsigned char *__restrict__ tiles, const int32_t *__restrict__ row,
                                const int32_t *__restrict__ col, int64_t nblocks, const double *__restrict__ cheb,
                                int dim, int p, int k, KernelFn f)
{
    for (int64_t b = blockIdx.x; b < nblocks; b += gridDim.x) {
        const int64_t t = row[b], s = col[b];
        unsigned char *tile = tiles + size_t(b) * 16384;
        for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
            const int nu = e / 64, mu = e % 64;
            double v = 0.0;
            if (nu < k && mu < k) {
                double xt[3], xs[3];
                int rn = nu, rm = mu;
                for (int d = 0; d < dim; ++d) {
                    xt[d] = cheb[(t * dim + d) * p + rn % p];
                    xs[d] = cheb[(s * dim + d) * p + rm % p];
                    rn /= p;
                    rm /= p;
                }
                v = kernel_eval(f, xt, xs, dim);
            }
            put_split(tile, nu, mu, v);
        }
    }
}

// Dense: row i (point of leaf t), column j (point of leaf s) = kappa(x_i, x_j), zero-padded.
__global__ void gen_dense_tc(unsigned char *__restrict__ tiles, const int32_t *__restrict__ row,
                             const int32_t *__restrict__ col, int64_t nblocks, const int32_t *__restrict__ leaf_lo,
                             const double *__restrict__ pts_tree, int dim, KernelFn f)
{
    for (int64_t b = blockIdx.x; b < nblocks; b += gridDim.x) {
        const int t = row[b], s = col[b];
        const int r0 = leaf_lo[t], rt = leaf_lo[t + 1] - r0;
        const int c0 = leaf_lo[s], cs = leaf_lo[s + 1] - c0;
        unsigned char *tile = tiles + size_t(b) * 16384;
        for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
            const int i = e / 64, j = e % 64;
            const double v = (i < rt && j < cs)
                                 ? kernel_eval(f, pts_tree + int64_t(r0 + i) * dim, pts_tree + int64_t(c0 + j) * dim, dim)
                                 : 0.0;
            put_split(tile, i, j, v);
        }
    }
}

}  // namespace h2k
