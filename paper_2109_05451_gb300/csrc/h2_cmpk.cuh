// h2_cmpk.cuh -- FP64 kernels of the algebraic recompression (Sec. 5).
//
// One CTA of 256 threads per node or per coupling block; every matrix of a step sits in
// shared memory (row-major, leading dimension k + 1). The building blocks:
//   * Householder QR (reflectors below the diagonal, R above) and the explicit Q by backward
//     accumulation of the reflectors (Golub & Van Loan, Alg. 5.1.1 / 5.2.1);
//   * the QR update of an upper-triangular R by a dense k x k block, R <- R-factor of
//     [R; B]: the new-basis downsweep folds the stack of Eq. for B_i^q into R one block at a
//     time, so a stack of any length needs k x k of memory;
//   * the Gram-matrix form of that downsweep (Cholesky factor of the accumulated B^T B);
//   * one-sided (Hestenes) Jacobi SVD with round-robin pair ordering, in two precisions;
//   * small products with triangular or rectangular factors.
// GB300 issues about two FP64 FMAs per clock per SM, so the kernels are laid out to keep
// lanes on useful FP64 work: few threads per reduction, no FP64 shuffle trees where a
// product term per lane will do.
// The rank of every level is decided on the device (atomicMax of the per-node counts), read
// by the next kernel, and never sent to the host until the end.
#pragma once

#include <cstdint>

namespace h2c {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxK = 64;      // rank of the operator being compressed
constexpr int kMaxRows = 128;  // points of a leaf; rows of a sibling pair's stack (2k)
constexpr int kMaxSweeps = 40;
constexpr double kJacobiTol = 1e-14;  // rotate while |a_p . a_q| > tol * |a_p| |a_q|
constexpr double kGramMinTau = 1e-7;  // the downsweep takes the Gram route for tau >= this
constexpr double kJacobiQuad = 1e-9;  // a sweep whose pairs were all this orthogonal ends the FP64 sweeps

// Shared-memory bytes of each kernel (ld = k + 1 doubles per matrix row).
__host__ __device__ constexpr size_t mat_bytes(int rows, int k) { return size_t(rows) * (k + 1) * 8; }
__host__ __device__ constexpr size_t scratch_bytes() { return size_t(4 * kMaxK + 16) * 8; }
__host__ __device__ constexpr size_t smem_leaf_qr(int M, int k) { return 2 * mat_bytes(M, k) + scratch_bytes(); }
__host__ __device__ constexpr size_t smem_transfer_qr(int k) { return 2 * mat_bytes(2 * k, k) + scratch_bytes(); }
__host__ __device__ constexpr size_t smem_sandwich(int k) { return 4 * mat_bytes(k, k) + scratch_bytes(); }
__host__ __device__ constexpr size_t smem_down(int k) { return 4 * mat_bytes(k, k) + scratch_bytes(); }
__host__ __device__ constexpr size_t smem_down_gram(int k) { return 3 * mat_bytes(k, k) + scratch_bytes(); }
// leaf SVD: A (max(M, k): Rh^T rows, then the leaf's Q), B (k: A32 + V32, then the result),
// V64 (k), Vq (k: then W')
__host__ __device__ constexpr size_t smem_leaf_svd(int M, int k)
{
    return mat_bytes(M > k ? M : k, k) + 3 * mat_bytes(k, k) + scratch_bytes();
}
// node SVD: Z (2k: then A32 + V32, then the result), X (2k), Rh / V64 (k), Vq (k)
__host__ __device__ constexpr size_t smem_node_svd(int k) { return 2 * mat_bytes(2 * k, k) + 2 * mat_bytes(k, k) + scratch_bytes(); }

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int level_of(int64_t t) { return 63 - __clzll(t); }

template <int G, typename T>
__device__ __forceinline__ T group_sum(T v)
{
#pragma unroll
    for (int o = G / 2; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}


// Apply the reflector I - tau v v^T (v = e_j + the tail below row j of column j of V) to
// the columns c0 .. c1-1 of A: 4 threads per column (8 columns per warp), each over a
// quarter of the rows, so that nearly every lane of an FP64 instruction does useful work.
__device__ __forceinline__ void reflect_columns(const double *V, int ldv, double *A, int lda, int rows, int j, int c0,
                                                int c1, double tau)
{
    const int grp = threadIdx.x / 4, gl = threadIdx.x % 4;
    for (int cb = c0; cb < c1; cb += kThreads / 4) {
        if (cb + (threadIdx.x / 32) * 8 >= c1) continue;  // the whole warp is past the last column
        const int c = cb + grp;
        const bool act = c < c1;
        double w = 0.0;
        if (act) {
            if (gl == 0) w = A[j * lda + c];
            for (int i = j + 1 + gl; i < rows; i += 4) w += V[i * ldv + j] * A[i * lda + c];
        }
        w = group_sum<4>(w) * tau;
        if (act) {
            if (gl == 0) A[j * lda + c] -= w;
            for (int i = j + 1 + gl; i < rows; i += 4) A[i * lda + c] -= V[i * ldv + j] * w;
        }
    }
}

// Householder QR of the rows x cols matrix A in place: R on and above the diagonal, the
// reflectors' tails below it (leading entry 1 implicit), their scalars in tau.
// red: 2 doubles of scratch. All threads of the CTA take part.
__device__ void house_qr(double *A, int ld, int rows, int cols, double *tau, double *red)
{
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int p = rows < cols ? rows : cols;
    for (int j = 0; j < p; ++j) {
        if (warp == 0) {
            double s = 0.0;
            for (int i = j + 1 + lane; i < rows; i += 32) s += A[i * ld + j] * A[i * ld + j];
            s = warp_sum(s);
            if (lane == 0) {
                const double alpha = A[j * ld + j];
                if (s == 0.0) {
                    tau[j] = 0.0;
                    red[0] = 0.0;
                } else {
                    const double beta = -copysign(sqrt(alpha * alpha + s), alpha);
                    tau[j] = (beta - alpha) / beta;
                    red[0] = 1.0 / (alpha - beta);
                    A[j * ld + j] = beta;
                }
            }
        }
        __syncthreads();
        const double tj = tau[j];
        if (tj != 0.0) {
            const double sc = red[0];
            for (int i = j + 1 + threadIdx.x; i < rows; i += kThreads) A[i * ld + j] *= sc;
            __syncthreads();
            reflect_columns(A, ld, A, ld, rows, j, j + 1, cols, tj);
        }
        __syncthreads();
    }
}

// Explicit Q (rows x cols) of house_qr's factorization: H_0 ... H_{p-1} applied to the first
// p columns of the identity, p = min(rows, cols); columns p..cols-1 are zero.
__device__ void house_form_q(const double *A, int ld, int rows, int cols, const double *tau, double *Q, int ldq)
{
    const int p = rows < cols ? rows : cols;
    for (int idx = threadIdx.x; idx < rows * cols; idx += kThreads) {
        const int i = idx / cols, c = idx % cols;
        Q[i * ldq + c] = (i == c && c < p) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int j = p - 1; j >= 0; --j) {
        const double tj = tau[j];
        if (tj != 0.0) reflect_columns(A, ld, Q, ldq, rows, j, j, p, tj);
        __syncthreads();
    }
}

// R <- R-factor of [R; B] for an upper-triangular k x k R and a dense k x k B (both in shared
// memory; B is destroyed). The reflector of column j touches row j of R and all of B.
__device__ void qr_fold(double *R, double *B, int ld, int k, double *red)
{
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    for (int j = 0; j < k; ++j) {
        if (warp == 0) {
            double s = 0.0;
            for (int i = lane; i < k; i += 32) s += B[i * ld + j] * B[i * ld + j];
            s = warp_sum(s);
            if (lane == 0) {
                const double alpha = R[j * ld + j];
                if (s == 0.0) {
                    red[0] = 0.0;
                } else {
                    const double beta = -copysign(sqrt(alpha * alpha + s), alpha);
                    red[0] = (beta - alpha) / beta;
                    red[1] = 1.0 / (alpha - beta);
                    R[j * ld + j] = beta;
                }
            }
        }
        __syncthreads();
        const double tj = red[0];
        if (tj != 0.0) {
            const double sc = red[1];
            for (int i = threadIdx.x; i < k; i += kThreads) B[i * ld + j] *= sc;
            __syncthreads();
            for (int c = j + 1 + warp; c < k; c += kWarps) {
                double w = lane == 0 ? R[j * ld + c] : 0.0;
                for (int i = lane; i < k; i += 32) w += B[i * ld + j] * B[i * ld + c];
                w = warp_sum(w) * tj;
                if (lane == 0) R[j * ld + c] -= w;
                for (int i = lane; i < k; i += 32) B[i * ld + c] -= B[i * ld + j] * w;
            }
        }
        __syncthreads();
    }
}

// One-sided (Hestenes) Jacobi on the columns of A (rows x cols, shared memory, leading
// dimension lda): sweeps of round-robin pairs, G threads per pair, until every pair is
// orthogonal to tol (|a_p . a_q| <= tol |a_p| |a_q|), or until a sweep's largest relative
// |a_p . a_q| was under quad (convergence is quadratic from there: the next sweep would find
// every pair below tol), or max_sweeps. Columns whose squared norm is under null2 are left
// alone (the numerical null space of a rank-deficient A would otherwise keep rotating). With V
// (cols x cols, leading dimension ldv) the rotations are accumulated, V <- V J. Returns the
// sweeps taken. flag: two ints of shared memory.
template <int G, typename T>
__device__ int jacobi_columns(T *A, int lda, int rows, int cols, T *V, int ldv, T tol, T quad, T null2, int max_sweeps,
                              int *flag)
{
    const int n2 = cols + (cols & 1);  // an odd column count plays against an absent column
    const int npairs = n2 / 2;
    const int g = threadIdx.x / G, gl = threadIdx.x % G;
    const bool warp_busy = (threadIdx.x / 32) * (32 / G) < npairs;  // uniform over the warp
    const T tol2 = tol * tol, huge = sizeof(T) == 8 ? T(1e150) : T(1e18);
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) flag[0] = flag[1] = 0;
        __syncthreads();
        for (int r = 0; r < n2 - 1; ++r) {
            if (warp_busy) {
                int p, q;
                if (g == 0) {
                    p = r;
                    q = n2 - 1;
                } else {
                    p = (r + g) % (n2 - 1);
                    q = (r - g + n2 - 1) % (n2 - 1);
                }
                if (p > q) {
                    const int tmp = p;
                    p = q;
                    q = tmp;
                }
                // every lane of the warp takes part in the group reductions
                const bool active = g < npairs && q < cols;
                T al = 0, be = 0, ga = 0;
                if (active)
                    for (int i = gl; i < rows; i += G) {
                        const T x = A[i * lda + p], y = A[i * lda + q];
                        al += x * x;
                        be += y * y;
                        ga += x * y;
                    }
                al = group_sum<G>(al);
                be = group_sum<G>(be);
                ga = group_sum<G>(ga);
                if (active && al > null2 && be > null2) {
                    const T off2 = ga * ga, ab = al * be;
                    if (gl == 0 && off2 > quad * quad * ab) atomicOr(flag + 1, 1);
                    if (off2 > tol2 * ab) {
                        const T zeta = (be - al) / (T(2) * ga);
                        const T az = fabs(zeta);  // zeta^2 would overflow
                        const T t = az > huge ? T(0.5) / zeta : copysign(T(1), zeta) / (az + sqrt(T(1) + zeta * zeta));
                        const T c = rsqrt(T(1) + t * t), s = c * t;
                        for (int i = gl; i < rows; i += G) {
                            const T x = A[i * lda + p], y = A[i * lda + q];
                            A[i * lda + p] = c * x - s * y;
                            A[i * lda + q] = s * x + c * y;
                        }
                        if (V)
                            for (int i = gl; i < cols; i += G) {
                                const T x = V[i * ldv + p], y = V[i * ldv + q];
                                V[i * ldv + p] = c * x - s * y;
                                V[i * ldv + q] = s * x + c * y;
                            }
                        if (gl == 0) flag[0] = 1;
                    }
                }
            }
            __syncthreads();
        }
        const int any = flag[0], large = flag[1];
        __syncthreads();
        if (!any || !large) break;
    }
    return sweep + 1;
}

// Relative size under which a singular vector is taken as numerical null space: far below
// any cut tau * sigma_1 the truncation can make (and the rounding level for tau = 0).
__device__ __forceinline__ double null_floor(double tau) { return tau > 0.0 ? fmin(1e-10, 1e-2 * tau) : 1e-13; }

// SVD of A (rows x cols, FP64, shared memory) by one-sided Jacobi in two precisions: sweeps
// on an FP32 copy (scaled to unit largest entry) accumulate the rotations in V32; V32, made
// orthogonal again in FP64 by a Householder QR, is applied to A (into B, rows x cols, which
// becomes the result); FP64 sweeps from there need one to three passes instead of about ten,
// and every FP64 rotation costs 64x an FP32 one on this part. A32 and V32 share the region
// f32 (rows + cols) * ld floats; V64 and Vq are cols x ld doubles. Columns under
// floor_rel * |A|_F are the numerical null space: the FP64 sweeps leave them alone. Returns
// the FP64 sweeps; the result's columns are in B, scr[kMaxK + 1] holds |A|_F^2, and with
// keep_v Vq holds every rotation (A Vq = B).
__device__ int svd_columns_mixed(const double *A, double *B, int ld, int rows, int cols, float *f32, double *V64,
                                 double *Vq, double *scr, double floor_rel, int *flag, bool keep_v = false)
{
    float *A32 = f32, *V32 = f32 + size_t(rows) * ld;
    double *tau = scr, *red = scr + kMaxK;
    // scale: the largest magnitude (rotations do not depend on it); the squared Frobenius
    // norm sets the null-column threshold
    if (threadIdx.x == 0) red[0] = red[1] = 0.0;
    __syncthreads();
    {
        double m = 0.0, f = 0.0;
        for (int idx = threadIdx.x; idx < rows * cols; idx += kThreads) {
            const double v = A[(idx / cols) * ld + idx % cols];
            m = fmax(m, fabs(v));
            f += v * v;
        }
        for (int o = 16; o; o >>= 1) {
            m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
            f += __shfl_xor_sync(0xffffffffu, f, o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMax(reinterpret_cast<unsigned long long *>(red), __double_as_longlong(m));
            atomicAdd(red + 1, f);
        }
    }
    __syncthreads();
    const double mx = red[0], fro2 = red[1], inv = mx > 0.0 ? 1.0 / mx : 0.0;
    for (int idx = threadIdx.x; idx < rows * cols; idx += kThreads) {
        const int i = idx / cols, j = idx % cols;
        A32[i * ld + j] = float(A[i * ld + j] * inv);
    }
    for (int idx = threadIdx.x; idx < cols * cols; idx += kThreads) {
        const int i = idx / cols, j = idx % cols;
        V32[i * ld + j] = i == j ? 1.0f : 0.0f;
    }
    __syncthreads();
    jacobi_columns<8, float>(A32, ld, rows, cols, V32, ld, 1e-5f, 0.0f, float(1e-12 * fro2 * inv * inv), 20, flag);
    for (int idx = threadIdx.x; idx < cols * cols; idx += kThreads) {
        const int i = idx / cols, j = idx % cols;
        V64[i * ld + j] = double(V32[i * ld + j]);
    }
    __syncthreads();
    house_qr(V64, ld, cols, cols, tau, red + 2);  // (red[1] = |A|_F^2 stays for the caller)
    house_form_q(V64, ld, cols, cols, tau, Vq, ld);
    for (int idx = threadIdx.x; idx < rows * cols; idx += kThreads) {  // B = A Vq
        const int i = idx / cols, j = idx % cols;
        double v = 0.0;
        for (int m = 0; m < cols; ++m) v += A[i * ld + m] * Vq[m * ld + j];
        B[i * ld + j] = v;
    }
    __syncthreads();
    // threads per pair: few (fewer rotation parameters per pair) while the columns are short
    const double null2 = floor_rel * floor_rel * fro2;
    double *V = keep_v ? Vq : nullptr;  // Vq J: all the rotations, when the caller needs them
    if (rows <= 40)
        return jacobi_columns<2, double>(B, ld, rows, cols, V, ld, kJacobiTol, kJacobiQuad, null2, kMaxSweeps, flag);
    if (rows <= 80)
        return jacobi_columns<4, double>(B, ld, rows, cols, V, ld, kJacobiTol, kJacobiQuad, null2, kMaxSweeps, flag);
    return jacobi_columns<8, double>(B, ld, rows, cols, V, ld, kJacobiTol, kJacobiQuad, null2, kMaxSweeps, flag);
}

// After jacobi_columns: the singular values (column norms) in descending order into sig[],
// the normalized columns in that order into W (rows x cols, global, leading dimension ldw),
// and the count of singular values above tau times the largest. Columns under floor_abs
// (the numerical null space, left out of the Jacobi sweeps) are neither normalized nor
// counted, and at most min(rows, cols) are. sv, pos: cols doubles / ints of scratch.
// With Vsrc (cols x cols, leading dimension ld) the columns of Vsrc are written instead (the
// right singular vectors; wrows = cols), unnormalized.
__device__ int sort_columns(const double *A, int ld, int rows, int cols, double *sv, int *pos, double *W, int ldw,
                            int wrows, double *sig, double tau, double floor_abs, const double *Vsrc = nullptr)
{
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    for (int j = warp; j < cols; j += kWarps) {
        double s = 0.0;
        for (int i = lane; i < rows; i += 32) s += A[i * ld + j] * A[i * ld + j];
        s = warp_sum(s);
        if (lane == 0) sv[j] = sqrt(s);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < cols; j += kThreads) {
        int r = 0;
        for (int i = 0; i < cols; ++i) r += (sv[i] > sv[j]) || (sv[i] == sv[j] && i < j);
        pos[j] = r;
    }
    __syncthreads();
    double smax = 0.0;
    for (int j = 0; j < cols; ++j) smax = fmax(smax, sv[j]);
    const double floor_ = fmax(floor_abs, 1e-13 * smax);
    for (int idx = threadIdx.x; idx < wrows * cols; idx += kThreads) {
        const int i = idx / cols, j = idx % cols;
        const double s = sv[j];
        if (Vsrc)
            W[int64_t(i) * ldw + pos[j]] = (i < cols && s > floor_) ? Vsrc[i * ld + j] : 0.0;
        else
            W[int64_t(i) * ldw + pos[j]] = (i < rows && s > floor_) ? A[i * ld + j] / s : 0.0;
    }
    for (int j = threadIdx.x; j < cols; j += kThreads) sig[pos[j]] = sv[j];
    int count = 0;
    if (smax > 0.0)
        for (int j = 0; j < cols; ++j) count += sv[j] > fmax(tau * smax, floor_);
    count = min(count, min(rows, cols));
    __syncthreads();
    return count;
}

// Carve helpers: matrices of `rows` rows at leading dimension k + 1.
struct Carve {
    double *p;
    __device__ double *take(int rows, int k)
    {
        double *r = p;
        p += size_t(rows) * (k + 1);
        return r;
    }
};

// ---------------------------------------------------------------- 1. orthogonalization

// Leaf bases: U_t = Q_t R_t. U: n x k in tree order; Q: per leaf an M x k slab.
__global__ void __launch_bounds__(kThreads) k_leaf_qr(const double *__restrict__ U, const int32_t *__restrict__ leaf_lo,
                                                      int64_t nleaves, int k, int M, double *__restrict__ Q,
                                                      double *__restrict__ R, int64_t first)
{
    extern __shared__ double sm[];
    const int ld = k + 1;
    Carve cv{sm};
    double *A = cv.take(M, k), *Qs = cv.take(M, k), *tau = cv.p, *red = tau + kMaxK;
    for (int64_t t = blockIdx.x; t < nleaves; t += gridDim.x) {
        const int lo = leaf_lo[t], rows = leaf_lo[t + 1] - lo;
        for (int idx = threadIdx.x; idx < rows * k; idx += kThreads) A[(idx / k) * ld + idx % k] = U[int64_t(lo) * k + idx];
        __syncthreads();
        house_qr(A, ld, rows, k, tau, red);
        house_form_q(A, ld, rows, k, tau, Qs, ld);
        double *Rt = R + (first + t) * k * k;
        for (int idx = threadIdx.x; idx < k * k; idx += kThreads) {
            const int i = idx / k, j = idx % k;
            Rt[idx] = (i < rows && j >= i) ? A[i * ld + j] : 0.0;
        }
        double *Qt = Q + t * int64_t(M) * k;
        for (int idx = threadIdx.x; idx < M * k; idx += kThreads) {
            const int i = idx / k, j = idx % k;
            Qt[idx] = i < rows ? Qs[i * ld + j] : 0.0;
        }
        __syncthreads();
    }
}

// Parents at level lp: [R_c1 E_c1; R_c2 E_c2] = Q R_t; the row blocks of Q are the
// orthogonal transfers E1 of the two children.
__global__ void __launch_bounds__(kThreads) k_transfer_qr(int lp, int k, const double *__restrict__ E0,
                                                          double *__restrict__ E1, double *__restrict__ R)
{
    extern __shared__ double sm[];
    const int ld = k + 1;
    Carve cv{sm};
    double *Z = cv.take(2 * k, k), *X = cv.take(2 * k, k), *tau = cv.p, *red = tau + kMaxK;
    double *Rc = X, *Ec = X + size_t(k) * ld;  // staging, then the explicit Q
    const int64_t p0 = int64_t(1) << lp;
    for (int64_t t = p0 + blockIdx.x; t < 2 * p0; t += gridDim.x) {
        for (int h = 0; h < 2; ++h) {
            const int64_t c = 2 * t + h;
            for (int idx = threadIdx.x; idx < k * k; idx += kThreads) {
                Rc[(idx / k) * ld + idx % k] = R[c * k * k + idx];
                Ec[(idx / k) * ld + idx % k] = E0[c * k * k + idx];
            }
            __syncthreads();
            for (int idx = threadIdx.x; idx < k * k; idx += kThreads) {
                const int i = idx / k, j = idx % k;
                double s = 0.0;
                for (int m = i; m < k; ++m) s += Rc[i * ld + m] * Ec[m * ld + j];
                Z[(h * k + i) * ld + j] = s;
            }
            __syncthreads();
        }
        house_qr(Z, ld, 2 * k, k, tau, red);
        house_form_q(Z, ld, 2 * k, k, tau, X, ld);
        double *Eo = E1 + (2 * t) * k * k;  // E1[2t] and E1[2t+1] are adjacent
        for (int idx = threadIdx.x; idx < 2 * k * k; idx += kThreads) Eo[idx] = X[(idx / k) * ld + idx % k];
        double *Rt = R + t * k * k;
        for (int idx = threadIdx.x; idx < k * k; idx += kThreads) {
            const int i = idx / k, j = idx % k;
            Rt[idx] = j >= i ? Z[i * ld + j] : 0.0;
        }
        __syncthreads();
    }
}

// Every coupling block re-expressed in the orthogonal bases: S <- R_t S R_s^T (in place;
// R upper triangular).
__global__ void __launch_bounds__(kThreads) k_orth_blocks(double *__restrict__ S, const int32_t *__restrict__ brow,
                                                          const int32_t *__restrict__ bcol, int64_t nb,
                                                          const double *__restrict__ R, int k)
{
    extern __shared__ double sm[];
    const int ld = k + 1;
    Carve cv{sm};
    double *Ss = cv.take(k, k), *Rt = cv.take(k, k), *Rs = cv.take(k, k), *Tm = cv.take(k, k);
    for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
        const int64_t t = brow[b], s = bcol[b];
        for (int idx = threadIdx.x; idx < k * k; idx += kThreads) {
            const int o = (idx / k) * ld + idx % k;
            Ss[o] = S[b * k * k + idx];
            Rt[o] = R[t * k * k + idx];
            Rs[o] = R[s * k * k + idx];
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < k * k; idx += kThreads) {  // Tm = S R_s^T
            const int j = idx / k, i = idx % k;  // lanes along i: one trip count per warp
            double v = 0.0;
            for (int m = j; m < k; ++m) v += Ss[i * ld + m] * Rs[j * ld + m];
            Tm[i * ld + j] = v;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < k * k; idx += kThreads) {  // R_t Tm
            const int i = idx / k, j = idx % k;
            double v = 0.0;
            for (int m = i; m < k; ++m) v += Rt[i * ld + m] * Tm[m * ld + j];
            S[b * k * k + idx] = v;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- 2. new-basis downsweep

// Nodes of level l: Rh_i = R-factor of [Rh_{i+} E1_i^T; S_{i j1}^T; ...], folded one block
// at a time (the parent's term first, then the block row in CSR order).
__global__ void __launch_bounds__(kThreads) k_down_qr(int l, int k, const int64_t *__restrict__ rowptr,
                                                      const double *__restrict__ S, const double *__restrict__ E1,
                                                      double *__restrict__ Rh)
{
    extern __shared__ double sm[];
    const int ld = k + 1;
    Carve cv{sm};
    double *Rm = cv.take(k, k), *B = cv.take(k, k), *P = cv.take(k, k), *X = cv.take(k, k), *red = cv.p;
    const int64_t n0 = int64_t(1) << l;
    for (int64_t i = n0 + blockIdx.x; i < 2 * n0; i += gridDim.x) {
        for (int idx = threadIdx.x; idx < k * k; idx += kThreads) Rm[(idx / k) * ld + idx % k] = 0.0;
        if (i > 1) {
            for (int idx = threadIdx.x; idx < k * k; idx += kThreads) {
                P[(idx / k) * ld + idx % k] = Rh[(i / 2) * k * k + idx];
                X[(idx / k) * ld + idx % k] = E1[i * k * k + idx];
            }
            __syncthreads();
            for (int idx = threadIdx.x; idx < k * k; idx += kThreads) {  // B = Rh_p E1_i^T
                const int a = idx / k, c = idx % k;
                double v = 0.0;
                for (int m = a; m < k; ++m) v += P[a * ld + m] * X[c * ld + m];
                B[a * ld + c] = v;
            }
            __syncthreads();
            qr_fold(Rm, B, ld, k, red);
        }
        for (int64_t b = rowptr[i]; b < rowptr[i + 1]; ++b) {
            for (int idx = threadIdx.x; idx < k * k; idx += kThreads) {
                const int a = idx / k, c = idx % k;
                B[c * ld + a] = S[b * k * k + idx];  // S_ij^T
            }
            __syncthreads();
            qr_fold(Rm, B, ld, k, red);
        }
        double *Ro = Rh + i * k * k;
        for (int idx = threadIdx.x; idx < k * k; idx += kThreads) {
            const int a = idx / k, c = idx % k;
            Ro[idx] = c >= a ? Rm[a * ld + c] : 0.0;
        }
        __syncthreads();
    }
}

// The same factors through their Gram matrices: only Rh_i^T Rh_i = B_i^T B_i enters the
// truncation (the left singular vectors and values of U_i Rh_i^T), and
//   G_i = B_i^T B_i = E1_i G_{i+} E1_i^T + sum_j S_ij S_ij^T
// accumulates with every lane on a product term, where the QR update spends most of its
// FP64 instructions on reductions. Rh_i is then the transposed Cholesky factor of G_i
// (columns whose pivot falls under k * eps * max diag are set to zero: G_i is semidefinite).
// Squaring the data limits what is resolved to singular values above ~1e-8 of a node's
// largest. Nodes of level l; Gout keeps G_i for the next level.
constexpr int kMaxOut = (kMaxK * (kMaxK + 1) / 2 + kThreads - 1) / kThreads;  // lower-triangle outputs per thread

__device__ __forceinline__ void tri_index(int idx, int &a, int &b)
{
    a = int((sqrtf(8.0f * float(idx) + 1.0f) - 1.0f) * 0.5f);
    while ((a + 1) * (a + 2) / 2 <= idx) ++a;
    while (a * (a + 1) / 2 > idx) --a;
    b = idx - a * (a + 1) / 2;
}

__global__ void __launch_bounds__(kThreads) k_down_gram(int l, int k, const int64_t *__restrict__ rowptr,
                                                        const double *__restrict__ S, const double *__restrict__ E1,
                                                        double *__restrict__ Gout, double *__restrict__ Rh)
{
    extern __shared__ double sm[];
    const int ld = k + 1;
    Carve cv{sm};
    double *B0 = cv.take(k, k), *B1 = cv.take(k, k), *X = cv.take(k, k), *red = cv.p;
    const int np = k * (k + 1) / 2;
    int oa[kMaxOut], ob[kMaxOut];
#pragma unroll
    for (int u = 0; u < kMaxOut; ++u) {
        const int idx = threadIdx.x + u * kThreads;
        if (idx < np) tri_index(idx, oa[u], ob[u]);
        else oa[u] = ob[u] = 0;
    }
    const int64_t n0 = int64_t(1) << l;
    for (int64_t i = n0 + blockIdx.x; i < 2 * n0; i += gridDim.x) {
        double acc[kMaxOut];
#pragma unroll
        for (int u = 0; u < kMaxOut; ++u) acc[u] = 0.0;
        if (i > 1) {  // E1_i G_p E1_i^T
            for (int idx = threadIdx.x; idx < k * k; idx += kThreads) {
                B0[(idx / k) * ld + idx % k] = Gout[(i / 2) * k * k + idx];
                B1[(idx / k) * ld + idx % k] = E1[i * k * k + idx];
            }
            __syncthreads();
            for (int idx = threadIdx.x; idx < k * k; idx += kThreads) {  // X = E1_i G_p
                const int a = idx / k, c = idx % k;
                double v = 0.0;
                for (int m = 0; m < k; ++m) v += B1[a * ld + m] * B0[m * ld + c];
                X[a * ld + c] = v;
            }
            __syncthreads();
#pragma unroll
            for (int u = 0; u < kMaxOut; ++u)
                if (threadIdx.x + u * kThreads < np) {
                    const double *xa = X + oa[u] * ld, *eb = B1 + ob[u] * ld;
                    double v = 0.0;
                    for (int m = 0; m < k; ++m) v += xa[m] * eb[m];
                    acc[u] = v;
                }
            __syncthreads();
        }
        for (int64_t b = rowptr[i]; b < rowptr[i + 1]; ++b) {  // + S_ij S_ij^T
            for (int idx = threadIdx.x; idx < k * k; idx += kThreads) B0[(idx / k) * ld + idx % k] = S[b * k * k + idx];
            __syncthreads();
#pragma unroll
            for (int u = 0; u < kMaxOut; ++u)
                if (threadIdx.x + u * kThreads < np) {
                    const double *sa = B0 + oa[u] * ld, *sb = B0 + ob[u] * ld;
                    double v = 0.0;
                    for (int m = 0; m < k; ++m) v += sa[m] * sb[m];
                    acc[u] += v;
                }
            __syncthreads();
        }
        // G_i (full, symmetric) to global and shared memory
#pragma unroll
        for (int u = 0; u < kMaxOut; ++u)
            if (threadIdx.x + u * kThreads < np) {
                const int a = oa[u], c = ob[u];
                Gout[i * k * k + a * k + c] = acc[u];
                Gout[i * k * k + c * k + a] = acc[u];
                X[a * ld + c] = acc[u];
                X[c * ld + a] = acc[u];
            }
        __syncthreads();
        // Cholesky G = L L^T in place (lower triangle of X), columns in order
        if (threadIdx.x == 0) {
            double dmax = 0.0;
            for (int j = 0; j < k; ++j) dmax = fmax(dmax, X[j * ld + j]);
            red[0] = double(k) * 2.220446049250313e-16 * dmax;
        }
        __syncthreads();
        const double delta = red[0];
        for (int j = 0; j < k; ++j) {
            const double d = X[j * ld + j];
            const double piv = d > delta ? sqrt(d) : 0.0;
            const double inv = piv > 0.0 ? 1.0 / piv : 0.0;
            __syncthreads();
            for (int r = j + threadIdx.x; r < k; r += kThreads) X[r * ld + j] = r == j ? piv : X[r * ld + j] * inv;
            __syncthreads();
            for (int idx = threadIdx.x; idx < (k - j - 1) * (k - j - 1); idx += kThreads) {
                const int r = j + 1 + idx / (k - j - 1), c = j + 1 + idx % (k - j - 1);
                if (c <= r) X[r * ld + c] -= X[r * ld + j] * X[c * ld + j];
            }
            __syncthreads();
        }
        double *Ro = Rh + i * k * k;  // Rh = L^T
        for (int idx = threadIdx.x; idx < k * k; idx += kThreads) {
            const int a = idx / k, c = idx % k;
            Ro[idx] = c >= a ? X[c * ld + a] : 0.0;
        }
        __syncthreads();
    }
}

// ||A_lr||_F^2 = sum over leaves of trace(G_t) = ||Rh_t||_F^2 (A_lr the low-rank part), summed
// in a fixed order by one CTA into norm[0] (a check of the downsweep).
// gram: G holds the Gram matrices (sum of the diagonals), else the R factors (sum of squares).
__global__ void __launch_bounds__(kThreads) k_norm(const double *__restrict__ G, int64_t first, int64_t nleaves, int k,
                                                   bool gram, double *__restrict__ norm)
{
    __shared__ double part[kThreads];
    double s = 0.0;
    const double *base = G + first * k * k;
    if (gram) {
        for (int64_t i = threadIdx.x; i < nleaves * k; i += kThreads) s += base[(i / k) * k * k + (i % k) * (k + 1)];
    } else {
        for (int64_t i = threadIdx.x; i < nleaves * k * k; i += kThreads) s += base[i] * base[i];
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = kThreads / 2; w; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) norm[0] = sqrt(part[0]);
}

// ---------------------------------------------------------------- 3. truncation upsweep

// Leaves: SVD of the reweighted basis Q_t Rh_t^T (rows x k). Q_t has orthonormal columns
// (then zero columns from p = min(rows, k) on), so its left singular vectors are Q_t W' with
// W' those of the p x k matrix Rh_t^T[0:p, :], which the Jacobi sweeps take instead (k rows
// instead of the leaf's points). W: per leaf an M x k slab of left singular vectors by
// descending singular value; sig: k per leaf; the count above tau times the largest raises
// rank[q].
__global__ void __launch_bounds__(kThreads) k_leaf_svd(const double *__restrict__ Q, const int32_t *__restrict__ leaf_lo,
                                                       int64_t nleaves, int k, int M, const double *__restrict__ Rh,
                                                       int64_t first, double tau,
                                                       double *__restrict__ W, double *__restrict__ sig,
                                                       int *__restrict__ rank, int q, unsigned long long *sweeps)
{
    extern __shared__ double sm[];
    const int ld = k + 1;
    Carve cv{sm};
    double *A = cv.take(M > k ? M : k, k), *B = cv.take(k, k), *Rs = cv.take(k, k), *Vq = cv.take(k, k);
    double *sv = cv.p, *qscr = sv + 2 * kMaxK;
    int *pos = reinterpret_cast<int *>(sv + kMaxK), *flag = pos + kMaxK;
    const double floor_rel = null_floor(tau);
    for (int64_t t = blockIdx.x; t < nleaves; t += gridDim.x) {
        const int rows = leaf_lo[t + 1] - leaf_lo[t], p = rows < k ? rows : k;
        for (int idx = threadIdx.x; idx < p * k; idx += kThreads) {  // A = Rh^T[0:p, :]
            const int i = idx / k, j = idx % k;
            A[i * ld + j] = Rh[(first + t) * k * k + j * k + i];
        }
        __syncthreads();
        const int sw = svd_columns_mixed(A, B, ld, p, k, reinterpret_cast<float *>(B), Rs, Vq, qscr, floor_rel, flag);
        const int count = sort_columns(B, ld, p, k, sv, pos, Vq, ld, p, sig + t * k, tau,
                                       floor_rel * sqrt(qscr[kMaxK + 1]));
        const double *Qt = Q + t * int64_t(M) * k;  // W = Q[:, 0:p] W'
        for (int idx = threadIdx.x; idx < rows * k; idx += kThreads) A[(idx / k) * ld + idx % k] = Qt[idx];
        __syncthreads();
        double *Wt = W + t * int64_t(M) * k;
        for (int idx = threadIdx.x; idx < M * k; idx += kThreads) {
            const int i = idx / k, j = idx % k;
            double v = 0.0;
            if (i < rows)
                for (int m = 0; m < p; ++m) v += A[i * ld + m] * Vq[m * ld + j];
            Wt[idx] = v;
        }
        if (threadIdx.x == 0) {
            atomicMax(rank + q, count);
            atomicAdd(sweeps, (unsigned long long)sw);
        }
        __syncthreads();
    }
}

// Leaves, once rank[q] is known: T_t = U'_t^T Q_t (r x k), U'_t the first r columns of W;
// the squares of the singular values not kept are added to dropped[0].
__global__ void __launch_bounds__(kThreads) k_leaf_t(const double *__restrict__ Q, const double *__restrict__ W,
                                                     const int32_t *__restrict__ leaf_lo, int64_t nleaves, int k, int M,
                                                     const int *__restrict__ rank, int q, int64_t first,
                                                     double *__restrict__ T, const double *__restrict__ sig,
                                                     double *__restrict__ dropped)
{
    const int r = rank[q];
    for (int64_t t = blockIdx.x; t < nleaves; t += gridDim.x) {
        if (threadIdx.x == 0) {
            double d = 0.0;
            for (int j = r; j < k; ++j) d += sig[(first + t) * k + j] * sig[(first + t) * k + j];
            atomicAdd(dropped, d);
        }
        const int rows = leaf_lo[t + 1] - leaf_lo[t];
        const double *Qt = Q + t * int64_t(M) * k, *Wt = W + t * int64_t(M) * k;
        double *Tt = T + (first + t) * k * k;
        for (int idx = threadIdx.x; idx < k * k; idx += kThreads) {
            const int a = idx / k, j = idx % k;
            double v = 0.0;
            if (a < r)
                for (int i = 0; i < rows; ++i) v += Wt[int64_t(i) * k + a] * Qt[int64_t(i) * k + j];
            Tt[idx] = v;
        }
    }
}

// Parents at level lp (children at lp + 1 with rank r = rank[lp+1]): Z = [T_c1 E1_c1;
// T_c2 E1_c2] (2r x k), SVD of Z Rh_t^T; Z and the sorted left singular vectors are kept
// for k_node_t; the count above the cut raises rank[lp].
__global__ void __launch_bounds__(kThreads) k_node_svd(int lp, int k, const double *__restrict__ T,
                                                       const double *__restrict__ E1, const double *__restrict__ Rh,
                                                       double tau, double *__restrict__ Zb,
                                                       double *__restrict__ Wb, double *__restrict__ sig,
                                                       int *__restrict__ rank, unsigned long long *sweeps)
{
    extern __shared__ double sm[];
    const int ld = k + 1;
    Carve cv{sm};
    double *Z = cv.take(2 * k, k), *X = cv.take(2 * k, k), *Rs = cv.take(k, k), *Vq = cv.take(k, k);
    double *sv = cv.p, *qscr = sv + 2 * kMaxK;
    int *pos = reinterpret_cast<int *>(sv + kMaxK), *flag = pos + kMaxK;
    double *Tc = X, *Ec = X + size_t(k) * ld;  // staging; then X holds Z Rh^T
    const int r = rank[lp + 1];
    const double floor_rel = null_floor(tau);
    const int64_t p0 = int64_t(1) << lp;
    for (int64_t t = p0 + blockIdx.x; t < 2 * p0; t += gridDim.x) {
        const int64_t slot = t - p0;
        for (int h = 0; h < 2; ++h) {
            const int64_t c = 2 * t + h;
            for (int idx = threadIdx.x; idx < k * k; idx += kThreads) {
                Tc[(idx / k) * ld + idx % k] = T[c * k * k + idx];
                Ec[(idx / k) * ld + idx % k] = E1[c * k * k + idx];
            }
            __syncthreads();
            for (int idx = threadIdx.x; idx < r * k; idx += kThreads) {
                const int i = idx / k, j = idx % k;
                double v = 0.0;
                for (int m = 0; m < k; ++m) v += Tc[i * ld + m] * Ec[m * ld + j];
                Z[(h * r + i) * ld + j] = v;
            }
            __syncthreads();
        }
        for (int idx = threadIdx.x; idx < k * k; idx += kThreads)
            Rs[(idx / k) * ld + idx % k] = Rh[t * k * k + idx];
        double *Zo = Zb + slot * 2 * k * k;
        for (int idx = threadIdx.x; idx < 2 * r * k; idx += kThreads) Zo[idx] = Z[(idx / k) * ld + idx % k];
        __syncthreads();
        // X = Z Rh^T (2r x k). With 2r < k the Jacobi sweeps take X^T (k x 2r: 2r columns of
        // full rank, where X's k columns would carry k - 2r null ones) and the left singular
        // vectors of X are the accumulated rotations.
        const int n = 2 * r;
        const bool wide = n < k;
        for (int idx = threadIdx.x; idx < n * k; idx += kThreads) {
            const int j = idx / n, i = idx % n;  // lanes along i: one trip count per warp
            double v = 0.0;
            for (int m = j; m < k; ++m) v += Z[i * ld + m] * Rs[j * ld + m];
            if (wide) X[j * ld + i] = v;
            else X[i * ld + j] = v;
        }
        __syncthreads();
        int count = 0;
        if (r > 0) {
            const int rows = wide ? k : n, cols = wide ? n : k;
            const int sw = svd_columns_mixed(X, Z, ld, rows, cols, reinterpret_cast<float *>(Z), Rs, Vq, qscr, floor_rel,
                                             flag, wide);
            for (int j = threadIdx.x; j < k; j += kThreads) sig[t * k + j] = 0.0;
            __syncthreads();
            count = sort_columns(Z, ld, rows, cols, sv, pos, Wb + slot * 2 * k * k, k, n, sig + t * k, tau,
                                 floor_rel * sqrt(qscr[kMaxK + 1]), wide ? Vq : nullptr);
            if (threadIdx.x == 0) atomicAdd(sweeps, (unsigned long long)sw);
        } else {
            for (int j = threadIdx.x; j < k; j += kThreads) sig[t * k + j] = 0.0;
        }
        if (threadIdx.x == 0) atomicMax(rank + lp, count);
        __syncthreads();
    }
}

// Parents at level lp, once rank[lp] = rp is known: E'_c1, E'_c2 = the two row blocks of the
// first rp singular vectors; T_t = W^T Z (rp x k); dropped energy as in k_leaf_t.
__global__ void __launch_bounds__(kThreads) k_node_t(int lp, int k, const double *__restrict__ Zb,
                                                     const double *__restrict__ Wb, const int *__restrict__ rank,
                                                     double *__restrict__ E2, double *__restrict__ T,
                                                     const double *__restrict__ sig, double *__restrict__ dropped)
{
    const int r = rank[lp + 1], rp = rank[lp];
    const int64_t p0 = int64_t(1) << lp;
    for (int64_t t = p0 + blockIdx.x; t < 2 * p0; t += gridDim.x) {
        if (threadIdx.x == 0) {
            double d = 0.0;
            for (int j = rp; j < k; ++j) d += sig[t * k + j] * sig[t * k + j];
            atomicAdd(dropped, d);
        }
        const int64_t slot = t - p0;
        const double *Zo = Zb + slot * 2 * k * k, *Wo = Wb + slot * 2 * k * k;
        for (int h = 0; h < 2; ++h) {
            double *Ec = E2 + (2 * t + h) * k * k;
            for (int idx = threadIdx.x; idx < k * k; idx += kThreads) {
                const int i = idx / k, j = idx % k;
                Ec[idx] = (i < r && j < rp) ? Wo[int64_t(h * r + i) * k + j] : 0.0;
            }
        }
        double *Tt = T + t * k * k;
        for (int idx = threadIdx.x; idx < k * k; idx += kThreads) {
            const int a = idx / k, j = idx % k;
            double v = 0.0;
            if (a < rp)
                for (int i = 0; i < 2 * r; ++i) v += Wo[int64_t(i) * k + a] * Zo[int64_t(i) * k + j];
            Tt[idx] = v;
        }
    }
}

// ---------------------------------------------------------------- 4. projection

// S'_ts = T_t S_ts T_s^T (r x r at the block's level, zero elsewhere in the k x k slab).
__global__ void __launch_bounds__(kThreads) k_project(double *__restrict__ S, const int32_t *__restrict__ brow,
                                                      const int32_t *__restrict__ bcol, int64_t nb,
                                                      const double *__restrict__ T, const int *__restrict__ rank, int k)
{
    extern __shared__ double sm[];
    const int ld = k + 1;
    Carve cv{sm};
    double *Ss = cv.take(k, k), *Tt = cv.take(k, k), *Ts = cv.take(k, k), *Tm = cv.take(k, k);
    for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
        const int64_t t = brow[b], s = bcol[b];
        const int r = rank[level_of(t)];
        for (int idx = threadIdx.x; idx < k * k; idx += kThreads) {
            const int o = (idx / k) * ld + idx % k;
            Ss[o] = S[b * k * k + idx];
            Tt[o] = T[t * k * k + idx];
            Ts[o] = T[s * k * k + idx];
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < k * r; idx += kThreads) {  // Tm = S T_s^T (k x r)
            const int i = idx / r, j = idx % r;
            double v = 0.0;
            for (int m = 0; m < k; ++m) v += Ss[i * ld + m] * Ts[j * ld + m];
            Tm[i * ld + j] = v;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < k * k; idx += kThreads) {  // T_t Tm
            const int i = idx / k, j = idx % k;
            double v = 0.0;
            if (i < r && j < r)
                for (int m = 0; m < k; ++m) v += Tt[i * ld + m] * Tm[m * ld + j];
            S[b * k * k + idx] = v;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- compaction to rank kc

__global__ void k_compact_u(const double *__restrict__ W, const int32_t *__restrict__ leaf_lo, int64_t nleaves, int k,
                            int M, const int *__restrict__ rank, int q, int kc, double *__restrict__ U)
{
    const int r = rank[q];
    for (int64_t t = blockIdx.x; t < nleaves; t += gridDim.x) {
        const int lo = leaf_lo[t], rows = leaf_lo[t + 1] - lo;
        for (int idx = threadIdx.x; idx < rows * kc; idx += blockDim.x) {
            const int i = idx / kc, j = idx % kc;
            U[(int64_t(lo) + i) * kc + j] = j < r ? W[(t * int64_t(M) + i) * k + j] : 0.0;
        }
    }
}

// k x k slabs -> kc x kc (top-left), for the transfers and the coupling blocks.
__global__ void k_compact_slabs(const double *__restrict__ src, int64_t count, int k, int kc, double *__restrict__ dst)
{
    const int64_t n = count * kc * kc;
    for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < n; idx += int64_t(gridDim.x) * blockDim.x) {
        const int64_t b = idx / (int64_t(kc) * kc);
        const int i = int((idx / kc) % kc), j = int(idx % kc);
        dst[idx] = (i < k && j < k) ? src[(b * k + i) * k + j] : 0.0;
    }
}

}  // namespace h2c
