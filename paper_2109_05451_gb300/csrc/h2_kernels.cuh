// h2_kernels.cuh -- device kernels of the H^2 matvec (FP64 / FP32 entries).
//
// The product follows Sec. 3 of the paper: upsweep xhat = V^T x (Sec. 3.1, Alg 1), tree
// multiply yhat^l = S^l xhat^l on every level (Sec. 3.2, Alg 4), downsweep y = U yhat
// (Sec. 3.3, Alg 6), plus the dense block-sparse product A_de x (Sec. 3). The paper
// runs each level as marshaled batched GEMVs; here every phase is one kernel over
// level-ordered CSR arrays built once on the host, so no marshaling runs per product.
//
// Layouts (T = double or float):
//   U   n x k row-major, rows in tree order (leaf t = rows leaf_lo[t] .. leaf_lo[t+1])
//   E   per heap node c >= 2 a k x k row-major block E_c[mu][nu] at c*k*k
//   S   coupling blocks in CSR order, each stored transposed: S_ts[nu][mu] at mu*k + nu
//   D   dense blocks in CSR order at dns_off[b], transposed: D_ts[i][j] at j*rows_t + i
//   xt, yd   n x nv column-major in tree order (permuted input, dense partial result)
//   xh, yh   per heap node k x nv column-major at node*k*nv (coefficient trees)
// Block transposition makes the thread that owns output row nu read consecutive
// addresses with its neighbours, so every block streams from HBM fully coalesced.
#pragma once

#include <cstdint>

#include "../../include/h2.h"

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
// transposed in T. One CTA per block (grid-stride over blocks).
template <typename T>
__global__ void gen_coupling(T *__restrict__ S, const int32_t *__restrict__ row, const int32_t *__restrict__ col,
                             int64_t nblocks, const double *__restrict__ cheb, int dim, int p, int k, KernelFn f)
{
    const int64_t kk = int64_t(k) * k;
    for (int64_t b = blockIdx.x; b < nblocks; b += gridDim.x) {
        const int64_t t = row[b], s = col[b];
        for (int64_t e = threadIdx.x; e < kk; e += blockDim.x) {
            const int nu = int(e % k), mu = int(e / k);
            double xt[3], xs[3];
            int rn = nu, rm = mu;
            for (int d = 0; d < dim; ++d) {
                xt[d] = cheb[(t * dim + d) * p + rn % p];
                xs[d] = cheb[(s * dim + d) * p + rm % p];
                rn /= p;
                rm /= p;
            }
            S[b * kk + e] = T(kernel_eval(f, xt, xs, dim));
        }
    }
}

// Dense blocks D_ts[i][j] = kappa(x_i, x_j), stored transposed (i fastest).
template <typename T>
__global__ void gen_dense(T *__restrict__ D, const int64_t *__restrict__ off, const int32_t *__restrict__ row,
                          const int32_t *__restrict__ col, int64_t nblocks, const int32_t *__restrict__ leaf_lo,
                          const double *__restrict__ pts_tree, int dim, KernelFn f)
{
    for (int64_t b = blockIdx.x; b < nblocks; b += gridDim.x) {
        const int t = row[b], s = col[b];
        const int r0 = leaf_lo[t], rt = leaf_lo[t + 1] - r0;
        const int c0 = leaf_lo[s], cs = leaf_lo[s + 1] - c0;
        const int64_t cnt = int64_t(rt) * cs;
        for (int64_t e = threadIdx.x; e < cnt; e += blockDim.x) {
            const int i = int(e % rt), j = int(e / rt);
            D[off[b] + e] = T(kernel_eval(f, pts_tree + int64_t(r0 + i) * dim, pts_tree + int64_t(c0 + j) * dim, dim));
        }
    }
}

// ------------------------------------------------------------------ matvec kernels

// Step 1 + leaf part of Alg 1: xt = X[perm] (tree order) and xhat^q_t = U_t^T xt_t.
// One CTA per leaf; thread nu owns coefficient nu and reads U rows coalesced.
template <typename T>
__global__ void leaf_project(const T *__restrict__ X, int64_t n, int nv, const int32_t *__restrict__ perm,
                             const int32_t *__restrict__ leaf_lo, const T *__restrict__ U, int k,
                             int64_t first_leaf, T *__restrict__ xt, T *__restrict__ xh)
{
    extern __shared__ unsigned char smem_raw[];
    T *xs = reinterpret_cast<T *>(smem_raw);
    const int leaf = blockIdx.x;
    const int r0 = leaf_lo[leaf], rows = leaf_lo[leaf + 1] - r0;
    T *out = xh + (first_leaf + leaf) * int64_t(k) * nv;
    for (int v = 0; v < nv; ++v) {
        for (int i = threadIdx.x; i < rows; i += blockDim.x) {
            const T x = X[int64_t(v) * n + perm[r0 + i]];
            xs[i] = x;
            xt[int64_t(v) * n + r0 + i] = x;
        }
        __syncthreads();
        for (int nu = threadIdx.x; nu < k; nu += blockDim.x) {
            T acc = 0;
            const T *u = U + int64_t(r0) * k + nu;
            for (int i = 0; i < rows; ++i) acc += u[int64_t(i) * k] * xs[i];
            out[v * k + nu] = acc;
        }
        __syncthreads();
    }
}

// One upsweep level of Alg 1: xhat^{l-1}_p = E_{2p}^T xhat^l_{2p} + E_{2p+1}^T xhat^l_{2p+1}.
template <typename T>
__global__ void upsweep_level(int64_t first_parent, const T *__restrict__ E, T *__restrict__ xh, int k, int nv)
{
    extern __shared__ unsigned char smem_raw[];
    T *xc = reinterpret_cast<T *>(smem_raw);  // 2 children x k x nv
    const int64_t par = first_parent + blockIdx.x;
    const int64_t c0 = 2 * par;
    const int kn = k * nv;
    for (int e = threadIdx.x; e < 2 * kn; e += blockDim.x) xc[e] = xh[c0 * kn + e];
    __syncthreads();
    for (int e = threadIdx.x; e < kn; e += blockDim.x) {
        const int nu = e % k, v = e / k;
        T acc = 0;
        for (int c = 0; c < 2; ++c) {
            const T *Ec = E + (c0 + c) * int64_t(k) * k + nu;
            const T *x = xc + c * kn + v * k;
            for (int mu = 0; mu < k; ++mu) acc += Ec[int64_t(mu) * k] * x[mu];
        }
        xh[par * kn + e] = acc;
    }
}

// Block-row GEMV over a list of transposed blocks: out[v][i] = sum_b sum_j B_b[j][i] x_b[v][j].
// The CTA's threads are split into G column groups of R threads (R = rows rounded up to a
// warp multiple); group g takes columns j = g, g+G, ...; partial sums are reduced in
// shared memory in a fixed order, so the result is deterministic.
template <typename T, typename BlockFn>
__device__ __forceinline__ void block_row_gemv(int rows, int64_t b0, int64_t b1, int nv, BlockFn blk, T *out,
                                               int64_t out_ld, T *red)
{
    const int R = ((rows + 31) / 32) * 32;
    const int G = max(1, int(blockDim.x) / R);
    const int g = threadIdx.x / R, i = threadIdx.x % R;
    for (int v = 0; v < nv; ++v) {
        T acc = 0;
        if (g < G && i < rows) {
            for (int64_t b = b0; b < b1; ++b) {
                const T *B;
                const T *x;
                int cols;
                blk(b, v, B, x, cols);
                for (int j = g; j < cols; j += G) acc += B[int64_t(j) * rows + i] * x[j];
            }
        }
        if (G > 1) {
            if (g < G) red[threadIdx.x] = acc;
            __syncthreads();
            if (g == 0 && i < rows) {
                for (int gg = 1; gg < G; ++gg) acc += red[gg * R + i];
                out[v * out_ld + i] = acc;
            }
            __syncthreads();
        } else if (g == 0 && i < rows) {
            out[v * out_ld + i] = acc;
        }
    }
}

// Alg 4 on every level at once: yhat^l_t = sum_{s in b_t} S^l_ts xhat^l_s. One CTA per
// non-empty block row; rows of different levels are independent.
template <typename T>
__global__ void coupling_rows(const int32_t *__restrict__ rows_list, const int64_t *__restrict__ rowptr,
                              const int32_t *__restrict__ col, const T *__restrict__ S, const T *__restrict__ xh,
                              T *__restrict__ yh, int k, int nv)
{
    extern __shared__ unsigned char smem_raw[];
    T *red = reinterpret_cast<T *>(smem_raw);
    const int64_t t = rows_list[blockIdx.x];
    const int64_t kk = int64_t(k) * k;
    auto blk = [&](int64_t b, int v, const T *&B, const T *&x, int &cols) {
        B = S + b * kk;
        x = xh + (int64_t(col[b]) * nv + v) * k;
        cols = k;
    };
    block_row_gemv<T>(k, rowptr[t], rowptr[t + 1], nv, blk, yh + t * int64_t(k) * nv, k, red);
}

// Dense near field (Sec. 3): yd_t = sum_s D_ts xt_s for each leaf row t.
template <typename T>
__global__ void dense_rows(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                           const int64_t *__restrict__ off, const T *__restrict__ D,
                           const int32_t *__restrict__ leaf_lo, const T *__restrict__ xt, T *__restrict__ yd,
                           int64_t n, int nv)
{
    extern __shared__ unsigned char smem_raw[];
    T *red = reinterpret_cast<T *>(smem_raw);
    const int t = blockIdx.x;
    const int r0 = leaf_lo[t], rows = leaf_lo[t + 1] - r0;
    auto blk = [&](int64_t b, int v, const T *&B, const T *&x, int &cols) {
        const int s = col[b];
        B = D + off[b];
        x = xt + int64_t(v) * n + leaf_lo[s];
        cols = leaf_lo[s + 1] - leaf_lo[s];
    };
    block_row_gemv<T>(rows, rowptr[t], rowptr[t + 1], nv, blk, yd + r0, n, red);
}

// One downsweep level of Alg 6: yhat^l_c = E_c yhat^{l-1}_parent + (S^l xhat^l)_c, written
// in place. A node without coupling blocks contributes zero; the root's value is its own
// coupling row (or zero).
template <typename T>
__global__ void downsweep_level(int64_t first_node, const T *__restrict__ E, T *__restrict__ yh,
                                const int64_t *__restrict__ rowptr, int k, int nv, int parent_is_root)
{
    extern __shared__ unsigned char smem_raw[];
    T *Es = reinterpret_cast<T *>(smem_raw);  // k x (k+1)
    T *yp = Es + k * (k + 1);                 // k x nv
    const int64_t c = first_node + blockIdx.x;
    const int64_t par = c / 2;
    const int kn = k * nv;
    const bool parent_valid = !parent_is_root || rowptr[par + 1] > rowptr[par];
    const bool own_valid = rowptr[c + 1] > rowptr[c];
    const T *Ec = E + c * int64_t(k) * k;
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) Es[(e / k) * (k + 1) + e % k] = Ec[e];
    for (int e = threadIdx.x; e < kn; e += blockDim.x) yp[e] = parent_valid ? yh[par * kn + e] : T(0);
    __syncthreads();
    for (int e = threadIdx.x; e < kn; e += blockDim.x) {
        const int mu = e % k, v = e / k;
        T acc = 0;
        const T *er = Es + mu * (k + 1);
        const T *y = yp + v * k;
        for (int nu = 0; nu < k; ++nu) acc += er[nu] * y[nu];
        if (own_valid) acc += yh[c * kn + e];
        yh[c * kn + e] = acc;
    }
}

// Leaf expansion of Alg 6 plus the dense partial result and the BLAS-style epilogue:
// y_t = U_t yhat^q_t + yd_t; Y[perm] = alpha y + beta Y (Y not read when beta == 0).
template <typename T>
__global__ void leaf_expand(const T *__restrict__ U, const T *__restrict__ yh, const T *__restrict__ yd,
                            const int32_t *__restrict__ perm, const int32_t *__restrict__ leaf_lo,
                            int64_t first_leaf, int k, int nv, int64_t n, bool yh_valid, T alpha, T beta,
                            T *__restrict__ Y)
{
    extern __shared__ unsigned char smem_raw[];
    T *Us = reinterpret_cast<T *>(smem_raw);  // 64 x (k+1)
    T *ys = Us + 64 * (k + 1);                // k x nv
    const int leaf = blockIdx.x;
    const int r0 = leaf_lo[leaf], rows = leaf_lo[leaf + 1] - r0;
    const int kn = k * nv;
    const T *yt = yh + (first_leaf + leaf) * kn;
    for (int e = threadIdx.x; e < kn; e += blockDim.x) ys[e] = yh_valid ? yt[e] : T(0);
    for (int c0 = 0; c0 < rows; c0 += 64) {
        const int cr = min(64, rows - c0);
        __syncthreads();
        for (int e = threadIdx.x; e < cr * k; e += blockDim.x)
            Us[(e / k) * (k + 1) + e % k] = U[int64_t(r0 + c0) * k + e];
        __syncthreads();
        for (int e = threadIdx.x; e < cr * nv; e += blockDim.x) {
            const int i = e % cr, v = e / cr;
            T acc = 0;
            const T *ur = Us + i * (k + 1);
            const T *y = ys + v * k;
            for (int nu = 0; nu < k; ++nu) acc += ur[nu] * y[nu];
            acc += yd[int64_t(v) * n + r0 + c0 + i];
            const int64_t o = int64_t(v) * n + perm[r0 + c0 + i];
            Y[o] = (beta == T(0)) ? alpha * acc : alpha * acc + beta * Y[o];
        }
    }
}

}  // namespace h2k
