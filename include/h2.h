/*
 * h2.h -- C ABI of libh2, an H^2-matrix library for one GB300 GPU (sm_103a).
 *
 * The operator is the H^2 representation of Zampini et al., "H2Opus: a distributed-
 * memory multi-GPU software package for non-local operators" (arXiv 2109.05451):
 *
 *     A_H2 = A_de + <U, S, V^T>                                      (Sec. 2.1)
 *
 * with dense m x m blocks A_de at the finest level, k x k coupling blocks S^l_ts on
 * every level, leaf bases U = V (m x k) and k x k interlevel transfers E = F. The
 * product y = A_H2 x runs the three phases of Sec. 3: upsweep xhat = V^T x (Sec. 3.1,
 * Alg 1), tree multiply yhat^l = S^l xhat^l on every level (Sec. 3.2, Alg 4), downsweep
 * y = U yhat (Sec. 3.3, Alg 6), plus the dense block-sparse product A_de x (Sec. 3).
 *
 * Construction (Sec. 2.2, Sec. 6.1, Sec. 6.3-6.4): a k-d tree with leaf size m, the
 * geometric admissibility condition eta |C_t - C_s| >= (D_t + D_s)/2 on cluster
 * bounding boxes, tensor Chebyshev interpolation (p points per dimension, rank
 * k = p^dim) for bases, transfers and couplings, and direct kernel evaluation for the
 * dense blocks. The tie and rounding rules that the paper leaves open are fixed as:
 *   - depth q = smallest q >= 0 with n <= m 2^q; all leaves are on level q;
 *   - split dimension = largest bounding-box extent (lowest dimension on ties); points
 *     ordered by (coordinate, original index); left child = first floor(size/2);
 *   - admissibility evaluated in FP64 as eta*sqrt(sum_d (c_t,d-c_s,d)^2) >= 0.5*(D_t+D_s)
 *     with c = (lo+hi)/2, D = |hi-lo|; equality is admissible; same-level pairs only;
 *   - first-kind Chebyshev points, box extents clamped below at 1e-12 x root diagonal;
 *     multi-index nu = j_0 + p j_1 + p^2 j_2.
 *
 * Conventions for every call:
 *   - Every function returns an h2_status (0 = H2_OK); no exception crosses the ABI.
 *   - Device calls are asynchronous on the given CUDA stream (a cudaStream_t passed as
 *     void*, NULL = the legacy default stream). Launch errors are returned at once; a
 *     fault during execution surfaces at a later call or synchronisation as H2_ECUDA.
 *   - Multivectors are n x nv, column-major, leading dimension n, in the caller's point
 *     order. Element type: double for H2_FP64, float for H2_FP32, H2_BF16X2 and H2_FP32_MF.
 *   - Inputs are copied at h2_build; device X, Y, b, x stay owned by the caller; the
 *     handle owns its host operator and its device copy until h2_destroy.
 *   - Products on one handle may be issued concurrently from several host threads and on
 *     several streams: h2_matvec keeps one workspace per stream (products on one stream are
 *     ordered by it), h2_matvec_ws runs on the workspace it is given (distinct workspaces
 *     for products that may overlap), and every product borrows its own fork/join context
 *     (side stream and events) while its launches are enqueued. h2_upload, h2_destroy,
 *     h2_set_timing and h2_get_timing must not overlap other calls on the same handle.
 *   - Device calls run on the current CUDA device, which must be the one the operator was
 *     uploaded to (H2_EINVAL otherwise).
 */
#ifndef H2_H
#define H2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct h2_op *h2_handle; /* opaque, owned by libh2 */

typedef enum {
    H2_OK = 0,
    H2_EINVAL = -1,   /* bad argument (null pointer, size out of range, wrong state) */
    H2_ENOMEM = -2,   /* host or device allocation failed */
    H2_ECUDA = -3,    /* a CUDA runtime call or kernel launch failed */
    H2_ETIMEOUT = -4, /* a bounded device-side wait ran out */
    H2_ESTATE = -5,   /* call not valid in the handle's state (e.g. no device copy) */
    H2_ECANCELED = -6, /* a served request was cancelled before it finished */
    H2_ENOTCONV = 1   /* iterative solve stopped at maxit without reaching tol */
} h2_status;

typedef enum {
    H2_K_EXP = 0,   /* exp(-r / a) */
    H2_K_GAUSS = 1, /* exp(-r^2 / a) */
    H2_K_IMQ = 2,   /* (r^2 + a)^(-b) */
    H2_K_POLY = 3   /* prod_d (1 + x_d y_d)^deg (reproduced exactly when deg < p) */
} h2_kernel_kind;

typedef struct {
    h2_kernel_kind kind;
    double a, b;
    int deg;
} h2_kernel;

typedef enum {
    H2_FP64 = 0,  /* entries and arithmetic in double */
    H2_FP32 = 1,  /* entries and arithmetic in float */
    H2_BF16X2 = 2, /* entries as bf16 hi + bf16 lo pairs, FP32 accumulation */
    H2_FP32_MF = 3 /* matrix-free FP32: bases and transfers stored, coupling and dense entries
                      evaluated in float inside every product (no blocks stored) */
} h2_prec;

#define H2_MAX_LEVELS 32

typedef struct {
    int64_t n;                  /* number of points */
    int dim;                    /* 1..3 */
    int depth;                  /* leaf level q (root = level 0) */
    int rank;                   /* k = cheb_order^dim */
    int leaf_size;              /* m */
    int cheb_order;             /* p */
    double eta;
    int64_t n_nodes;            /* 2^(q+1) - 1 clusters, heap numbered 1..n_nodes */
    int64_t n_leaves;           /* 2^q */
    int64_t n_coupling;         /* coupling blocks over all levels */
    int64_t n_dense;            /* dense blocks (leaf level) */
    int64_t coupling_per_level[H2_MAX_LEVELS];
    int32_t max_coupling_per_row; /* sparsity constant C_sp over all levels */
    int32_t max_dense_per_row;
    int64_t coupling_entries;   /* n_coupling * k * k */
    int64_t dense_entries;      /* sum over dense blocks of |t| * |s| */
    int64_t basis_entries;      /* n * k (leaf bases) */
    int64_t transfer_entries;   /* (n_nodes - 1) * k * k */
    int uploaded_prec;          /* h2_prec of the device copy, or -1 */
    size_t device_bytes;        /* bytes held on the device by the handle */
} h2_info;

/* Build the H^2 operator on the host in FP64 (Sec. 2.2, 6.1, 6.3): k-d tree, admissible
 * partition, Chebyshev leaf bases and transfers. Coupling and dense entries are defined
 * by (kernel, cluster Chebyshev points, points) and are materialised on the device by
 * h2_upload, as each GPU populates its own blocks in Sec. 2.2.
 *   points: host, n x dim row-major, copied. n >= 1, 1 <= dim <= 3, leaf_size >= 2,
 *   1 <= cheb_order with cheb_order^dim <= 64, eta >= 0, n < 2^31.
 *   out: receives the handle. Errors: H2_EINVAL, H2_ENOMEM. Host only: no CUDA call. */
int h2_build(const double *points, int64_t n, int dim, h2_kernel kernel, int leaf_size,
             int cheb_order, double eta, h2_handle *out);

/* Copy the operator to the current CUDA device in precision prec, generating every
 * coupling block S_ts[nu][mu] = kappa(xi^t_nu, xi^s_mu) and dense block kappa(x_i, x_j)
 * in FP64 on the device and rounding once to prec. Replaces an earlier device copy.
 * Synchronises the stream before returning. Errors: H2_EINVAL, H2_ENOMEM, H2_ECUDA. */
int h2_upload(h2_handle h, h2_prec prec, void *cuda_stream);

/* Bytes of device workspace one product with nv vectors needs (tree vectors xhat, yhat,
 * the permuted input and the dense partial result). 0 if h is NULL or not uploaded. */
size_t h2_workspace_bytes(h2_handle h, int nv);

/* Y = alpha * A_H2 * X + beta * Y (Sec. 3: upsweep, tree multiply, downsweep, dense).
 *   X, Y: device, n x nv column-major, ld = n, caller's point order; element type double
 *   for H2_FP64, float otherwise. X and Y must not overlap. When beta == 0, Y is not
 *   read (NaN in Y is ignored). nv >= 1. Uses a workspace that the handle keeps for this
 *   stream (by its cudaStream_t value), allocated on the stream's first product and grown
 *   when nv grows (a growth waits for that workspace's last product and frees it); each
 *   product on it is ordered after the previous one, also when a destroyed stream's handle
 *   value is reused. Errors: H2_EINVAL (also: another device is current), H2_ESTATE (no
 *   device copy), H2_ENOMEM, H2_ECUDA. */
int h2_matvec(h2_handle h, const void *X, void *Y, int nv, double alpha, double beta,
              void *cuda_stream);

/* As h2_matvec, with a caller-owned device workspace of ws_bytes >= h2_workspace_bytes
 * (h, nv), 256-byte aligned, on the operator's device. Products on one handle with distinct
 * workspaces may run concurrently on different streams, issued from any host threads.
 * Allocates no device memory. */
int h2_matvec_ws(h2_handle h, const void *X, void *Y, int nv, double alpha, double beta,
                 void *workspace, size_t ws_bytes, void *cuda_stream);

/* Product for callers that must not allocate device memory (no counterpart in the paper).
 * Some callers cannot call cudaMalloc where they need a product: code running inside a
 * fixed memory-pool budget, code called from an allocator or an out-of-memory handler
 * (where allocating could recurse or deadlock), and real-time loops that may not block
 * on an allocation's device-wide synchronisation. h2_matvec_noalloc computes exactly what
 * h2_matvec computes (Y = alpha * A_H2 * X + beta * Y, same arguments and layouts), but
 * takes its workspace from one fixed scratch area of H2_NOALLOC_SCRATCH_BYTES that every
 * GPU loading this library reserves for the life of the process. It allocates nothing.
 *   - Limit: h2_workspace_bytes(h, nv) must not exceed H2_NOALLOC_SCRATCH_BYTES (64 MiB:
 *     about 2^20 points at rank 64 in FP64 with nv = 1, or in FP32 with nv <= 2);
 *     larger operators are rejected with H2_EINVAL before anything is launched.
 *   - The first call on a device looks up the scratch area's device address for that
 *     device (cudaGetSymbolAddress, with the device current); make that first call before
 *     any stream capture on the device. With CUDA's lazy module loading that first lookup
 *     is also when the device reserves the scratch area, so it can fail with H2_ENOMEM.
 *   - The current device must be the one holding the operator's device copy (H2_EINVAL
 *     otherwise, before anything is launched).
 *   - All calls on one device share the one scratch area, whichever handle they use, and
 *     it keeps the previous call's contents (each product resets what it needs). Calls
 *     whose execution overlaps on the GPU (different streams, no ordering between them)
 *     race on it: order them on one stream or with events.
 * Errors: H2_EINVAL (bad argument, operator too large, another device current), H2_ESTATE
 * (no device copy), H2_ENOMEM (first call only, see above), H2_ECUDA. */
#define H2_NOALLOC_SCRATCH_BYTES (64u << 20)
int h2_matvec_noalloc(h2_handle h, const void *X, void *Y, int nv, double alpha, double beta,
                      void *cuda_stream);

/* Multi-vector FP32 products on the tensor cores (Sec. 3.2, Alg 4: with nv vectors the
 * per-level products are small GEMMs). For an H2_FP32 device copy with rank and leaf size
 * of at most 64, passes of more than 8 vectors stream the stored FP32 blocks through
 * tcgen05 MMAs in 3xTF32 form: each block value a and each vector value x is split into
 * hi = tf32(a) and lo = tf32(a - hi), and the four products hi*hi, hi*lo, lo*hi, lo*lo
 * accumulate in FP32 in tensor memory (22 of FP32's 24 significant bits per operand; the
 * result meets the FP32 accuracy of the CUDA-core path). enable = 0 sends those passes to
 * the CUDA-core FMA path instead; enable = 1 (the default after h2_upload) restores the
 * tensor cores. No effect on other precisions, shapes or vector counts. Host only; must
 * not overlap a product on the same handle. Errors: H2_EINVAL (h NULL), H2_ESTATE (no
 * device copy). */
int h2_set_fp32_tensor(h2_handle h, int enable);

/* Unpreconditioned conjugate gradients for (A_H2 + sigma2 I) x = b (the Krylov solve of
 * Sec. 6.4, without its multigrid preconditioner). The products run in the uploaded
 * precision; Krylov vectors, dot products and updates are FP64 on the device.
 *   b: device, n doubles; x: device, n doubles, holds x0 on entry and the solution on
 *   return. Stops when the recursive residual |r|/|b| < tol or after maxit iterations.
 *   iters (host, may be NULL): iterations done. true_relres (host, may be NULL):
 *   |b - (A + sigma2 I) x| / |b| recomputed with one more product. Synchronises the
 *   stream. Returns H2_OK, H2_ENOTCONV (maxit reached) or an error. */
int h2_cg_solve(h2_handle h, double sigma2, const double *b, double *x, double tol, int maxit,
                int *iters, double *true_relres, void *cuda_stream);

/* Sizes and counts of the operator. Host only. */
int h2_get_info(h2_handle h, h2_info *info);

/* Tree-order position -> caller index permutation (host array of n int64). */
int h2_get_perm(h2_handle h, int64_t *perm);

/* Coupling partition as block-row CSR over heap-numbered clusters (rows 1..n_nodes,
 * level-ordered): rowptr (host, n_nodes + 2 int64, row t spans [rowptr[t], rowptr[t+1]))
 * and col (host, n_coupling int32 heap indices, ascending within a row). */
int h2_get_coupling_csr(h2_handle h, int64_t *rowptr, int32_t *col);

/* Dense partition as CSR over leaves (0-based leaf index = heap index - 2^q): rowptr
 * (n_leaves + 1 int64) and col (n_dense int32 leaf indices, ascending within a row). */
int h2_get_dense_csr(h2_handle h, int64_t *rowptr, int32_t *col);

/* FP64 host copies of the leaf bases (n x k row-major, rows in tree order) and the
 * transfers ((n_nodes + 1) x k x k; E_c[mu][nu] at c*k*k + mu*k + nu, rows 0 and 1
 * unused). Either pointer may be NULL. */
int h2_get_bases(h2_handle h, double *U, double *E);

/* Instrumentation (no counterpart in the paper). With timing on, every product records
 * a CUDA event pair around each of its phases on the stream that runs the phase.
 * h2_get_timing waits for those events and returns, per phase, the summed milliseconds
 * and the number of kernel launches since the previous read, then resets the sums.
 * Phases: 0 gather + upsweep of the lowest levels (Alg 1), 1 streaming product of the
 * coupling rows of those levels (Alg 4) and of the dense rows (the dominant kernel),
 * 2 the top levels on the side stream (upsweep, coupling rows, downsweep), 3 downsweep of
 * the lowest levels + leaf expansion + epilogue (Alg 6). phase_ms and phase_launches: host arrays of H2_NPHASES entries (either
 * may be NULL); products (may be NULL): products timed. Counting launches is always on;
 * timing adds event records to the stream and is off by default. */
#define H2_NPHASES 4
int h2_set_timing(h2_handle h, int enable);
int h2_get_timing(h2_handle h, double *phase_ms, int64_t *phase_launches, int64_t *products);

/* Checkpoint of the host operator (no paper counterpart): h2_save writes the construction
 * (parameters, points, tree, partition, bases and transfers; not the device copy) to a binary
 * file; h2_load reads such a file into a new handle, ready for h2_upload, without rebuilding.
 * H2_EINVAL if the file cannot be written or read, or is not a consistent operator file. */
int h2_save(h2_handle h, const char *path);
int h2_load(const char *path, h2_handle *out);

/* ---------------------------------------------------------------- algebraic recompression
 * Sec. 5 on the current CUDA device, in FP64 (the paper's precision):
 *   1. orthogonalization of the basis tree: an upsweep of QR factorizations of the leaf bases
 *      and of each sibling pair's stacked, reweighted transfers; every coupling block is
 *      re-expressed in the orthogonal bases (S <- R_t S R_s^T);
 *   2. the new-basis downsweep: for every node the R factor of the stack of Eq. for B_i^q
 *      (the parent's factor times the transposed transfer, then the transposed blocks of the
 *      node's block row). For tau >= 1e-7 it is the Cholesky factor of the stack's Gram
 *      matrix, accumulated block by block (FP64-lean; resolves a node's singular values down
 *      to ~1e-8 of its largest, so results carry relative errors of order 1e-16 / tau); for
 *      smaller tau each block is folded in by a QR update, as the paper writes it;
 *   3. the truncation upsweep: SVDs of the reweighted leaf bases and of the stacked
 *      projected transfers; of each node, the singular values above tau times its largest
 *      are kept (every block row keeps relative accuracy tau); each level keeps the largest
 *      count over its nodes (one rank per level);
 *   4. projection of every coupling block on the new bases (S' = T_t S T_s^T).
 * Dense blocks are unchanged. The result is a new handle holding the compressed operator on
 * the host in FP64 (bases, transfers and coupling blocks stored at one rank, the largest level
 * rank, smaller levels zero-padded), ready for h2_upload at H2_FP64 or H2_FP32 (not H2_BF16X2 or
 * H2_FP32_MF) and for h2_save, or for another h2_compress. The input handle is unchanged and
 * need not be uploaded. Requires rank <= 64 and leaves of at most 128 points.
 *   tau: relative tolerance, >= 0 (0 keeps every nonzero singular value).
 *   out: receives the new handle. info (host, may be NULL): see h2_compress_info.
 * Synchronises the stream. Errors: H2_EINVAL, H2_ENOMEM, H2_ECUDA. */
typedef struct {
    double tau;
    double norm_lowrank;           /* ||A_lr||_F, A_lr the low-rank part: its square is the sum
                                      over leaves of ||R_t||_F^2 */
    double dropped_energy;         /* sum of the squares of the singular values not kept:
                                      ||A_lr - A'_lr||_F <= 2 sqrt(dropped_energy) */
    int depth;
    int rank_in;                   /* rank of the input */
    int rank_out;                  /* stored rank of the result: max of level_rank, >= 1 */
    int level_rank[H2_MAX_LEVELS]; /* rank of each level after truncation */
    double ms[4];                  /* device time of steps 1-4 (CUDA events) */
    double flops[4];               /* FP64 operations of steps 1-4 as the kernels perform them */
    int64_t jacobi_sweeps;         /* FP64 one-sided Jacobi sweeps over all SVDs of step 3 (after
                                      each SVD's FP32 sweeps, which are not counted) */
    size_t lowrank_bytes_in;       /* FP64 bytes of bases, transfers and coupling blocks */
    size_t lowrank_bytes_out;      /* the same at the level ranks of the result */
} h2_compress_info;
int h2_compress(h2_handle h, double tau, void *cuda_stream, h2_handle *out, h2_compress_info *info);

/* Rank of each level (host array of depth + 1 ints): the build's uniform rank, or the
 * level ranks of a compressed operator. */
int h2_get_level_ranks(h2_handle h, int *ranks);

/* Free the host operator, its device copy and its workspace. NULL is accepted. */
int h2_destroy(h2_handle h);

/* ---------------------------------------------------------------- batched products
 * Many products of uneven operators as one unit (no paper counterpart as an interface: the
 * batched, level-by-level marshaling of Sec. 3 runs inside one operator there). For each
 * member i: Y_i = alpha A_i X_i + beta Y_i with nv[i] vectors (device, column-major, ld = n_i,
 * element type of the uploads). The members' coupling and dense block rows of every level
 * form one work list that a persistent launch streams (one launch per width class of nv:
 * 1, 2-4, 5-8, 9-16, 17-32 and tile-size class); the members' upsweeps and downsweeps run
 * as merged launches too, one per sweep step and width class over a table of the members'
 * subtrees (Sec. 3.1 and 3.3 per member), so a replay takes a few dozen launches whatever
 * the member count. The whole product is captured once as a CUDA graph and replayed by
 * h2_batch_run, always with the X, Y, alpha and beta given here (update the contents of X
 * and Y between runs, not the pointers). All members share one precision, FP64 or FP32 (not
 * H2_BF16X2), and take one pass each (nv <= 4, or nv <= 32 when k <= 64 and leaves hold <= 64
 * points); members must stay uploaded and alive while the batch exists.
 * flags: H2_BATCH_AUTOTUNE times candidate launch configurations of each merged stream (CTAs
 * per SM, pipeline stages, scheduling chunk size) and appends the best to the autotuning
 * cache (the file named by the environment variable H2_TUNE_CACHE, else h2_autotune.txt next
 * to the library); without it a cached choice is used when present, else a default.
 * H2_BATCH_MEMBER_SWEEPS runs each member's sweeps as its own launches instead of the merged
 * ones (the earlier schedule, kept for comparison). */
typedef struct h2_batch *h2_batch_t;
#define H2_BATCH_AUTOTUNE 1
#define H2_BATCH_MEMBER_SWEEPS 2
int h2_batch_create(const h2_handle *ops, int count, const void *const *X, void *const *Y, const int *nv, double alpha,
                    double beta, int flags, h2_batch_t *out);
/* Replay the batched product on the stream (asynchronous). */
int h2_batch_run(h2_batch_t b, void *cuda_stream);
/* After a synchronize: H2_ETIMEOUT if a bounded wait of any kernel of the batch ran out. */
int h2_batch_check(h2_batch_t b);
/* One-line description of the groups and their launch configurations (NUL-terminated). */
int h2_batch_describe(h2_batch_t b, char *buf, size_t len);
int h2_batch_destroy(h2_batch_t b);

/* ---------------------------------------------------------------- CG serving loop
 * No paper counterpart as an interface (the paper's application calls its Krylov solver,
 * Sec. 6.4, inline): a request loop that runs CG solves of (A_H2 + sigma2 I) x = b on
 * resident operators as requests arrive. Requests wait in FIFO order and are admitted as
 * soon as a solve slot and enough slot memory are free (admission by device-memory
 * footprint, h2_server_request_bytes); admitted solves advance concurrently, each on its
 * own CUDA stream with its own workspace, so a solve admitted while others run overlaps
 * them on the device (continuous batching). Each solve is unpreconditioned CG from x0 = 0
 * with FP64 Krylov state and products in the operator's uploaded precision, with the
 * arithmetic of h2_cg_solve in the same order: a served x equals h2_cg_solve's bitwise and
 * does not depend on the other requests in flight. One scheduler thread per server; the
 * calls below may come from any host thread. Operators used by a server must stay uploaded
 * and alive until their requests complete, and must not have timing enabled. */
typedef struct h2_server *h2_server_t;

typedef struct {
    int64_t request_id;
    int status;          /* H2_OK converged, H2_ENOTCONV maxit reached or breakdown, < 0 error */
    int iters;           /* CG iterations applied */
    double true_relres;  /* |b - (A + sigma2 I) x| / |b| from one more product (0 when b = 0) */
    double t_submit, t_admit, t_done;  /* seconds since h2_server_create, steady clock */
} h2_request_result;

/* slot_memory_bytes: device memory reserved once for the Krylov state and product workspace
 * of admitted solves; max_slots >= 1: most solves in flight; max_points: largest n of any
 * request (sizes each slot's pinned host staging). Binds to the current CUDA device and
 * starts the scheduler thread. */
int h2_server_create(size_t slot_memory_bytes, int max_slots, int64_t max_points, h2_server_t *out);
/* Device bytes one request on this uploaded operator occupies inside a server (0 if h is
 * NULL or not uploaded). */
size_t h2_server_request_bytes(h2_handle h);
/* Queue a solve with relative tolerance tol and at most maxit iterations. b and x: host
 * arrays of n doubles owned by the caller; b is read when the request is admitted and x
 * written when it completes, so both must stay valid until its result has been polled.
 * *request_id identifies the result. Errors: H2_EINVAL (arguments, n > max_points),
 * H2_ESTATE (operator not uploaded), H2_ENOMEM (the request can never fit the slot memory). */
int h2_server_submit(h2_server_t s, h2_handle op, double sigma2, const double *b, double *x, double tol, int maxit,
                     int64_t *request_id);
/* A solve by mixed-precision iterative refinement: products in op's precision (FP32 or
 * split-BF16) inside, FP64 residuals outside. op64 is an FP64 device copy of the same
 * operator (another handle of the same build, e.g. h2_load of its h2_save, uploaded in
 * H2_FP64). From x = 0: an inner CG on (A_op + sigma2 I) d = r to the relative tolerance
 * inner_tol (0 < inner_tol < 1), then x += d and r = b - (A_op64 + sigma2 I) x in FP64, until
 * |r| / |b| < tol or maxit inner iterations in all. An FP32 product's error (about 1e-7 of
 * |A| |x|) bounds what plain CG on op can reach; the refinement's bound is op64's. Result:
 * iters = inner iterations in all, true_relres = the last FP64 residual, status H2_OK when it
 * is below tol. Errors as h2_server_submit; H2_ESTATE if op64 is not uploaded in FP64. */
int h2_server_submit_refined(h2_server_t s, h2_handle op, h2_handle op64, double sigma2, const double *b, double *x,
                             double tol, double inner_tol, int maxit, int64_t *request_id);
/* Device bytes one refined request occupies (0 unless op is uploaded and op64 is an FP64
 * copy with the same n). */
size_t h2_server_request_bytes_refined(h2_handle op, h2_handle op64);
/* Move up to max_results completed requests into results (host array) and set *n_results;
 * never blocks. */
int h2_server_poll(h2_server_t s, h2_request_result *results, int max_results, int *n_results);
/* Block until no request is queued or in flight; H2_ETIMEOUT after timeout_s seconds. */
int h2_server_wait(h2_server_t s, double timeout_s);
/* Cancel a request: a queued one completes at once with status H2_ECANCELED (x untouched);
 * one in flight stops after the iterations already enqueued, and completes with status
 * H2_ECANCELED, its current iterate in x and that iterate's true residual. H2_EINVAL if the
 * id is unknown or its result is already available. */
int h2_server_cancel(h2_server_t s, int64_t request_id);
/* Drop queued requests, let the ones in flight finish, stop the scheduler, free all. */
int h2_server_destroy(h2_server_t s);

/* Self-test of the bounded device waits (no paper counterpart): launches one thread that
 * waits on a shared-memory barrier nothing arrives on, with a budget of budget_cycles clock
 * cycles, and two warps that wait on node flags in global memory nothing sets (the waits of
 * the small-rank warp sweeps), the first with budget_cycles, the second with fifty times that.
 * The barrier wait and the first flag wait give up and record the failure in device flags;
 * the first also raises the launch's abort word, on which the second must leave. The call
 * returns H2_ETIMEOUT when all of this happened (H2_OK otherwise), and the CUDA context stays
 * usable. H2_EINVAL unless 1 <= budget_cycles <= 8e7. The kernels' own waits use the same
 * mechanisms with a budget of about one second. */
int h2_selftest_wait_timeout(int64_t budget_cycles);

/* Measured arithmetic peak of the current device (no paper counterpart; it supplies the
 * denominators of the rooflines: the FP64 product is bound by the FP64 fused multiply-add
 * rate, the FP32 multi-vector product on the CUDA cores by the FP32 one, the matrix-free
 * product by the special-function unit). Runs register-resident chains of one instruction
 * kind on every SM (32 warps per SM; per thread either four FMA accumulators whose
 * multiplicands rotate through distinct registers or eight FMA chains sharing their
 * multiplicands, whichever is faster; eight chains for ex2) for about target_ms milliseconds
 * per launch, after a calibration launch, and keeps the fastest of five timed launches per
 * form (CUDA events on the legacy default stream; synchronises the device).
 *   unit: H2_PEAK_DFMA (FP64 FMA, 2 flops each), H2_PEAK_FFMA (FP32 FMA, 2 flops each) or
 *   H2_PEAK_EX2 (special-function 2^x, 1 evaluation each). target_ms in [1, 1000].
 *   rate (host): flop/s, or evaluations/s for H2_PEAK_EX2. ms (host, may be NULL): the
 *   fastest launch's duration. Changes no clock or power setting: the rate is the one at the
 *   clocks the device runs at while measuring. Errors: H2_EINVAL, H2_ENOMEM, H2_ECUDA. */
#define H2_PEAK_DFMA 0
#define H2_PEAK_FFMA 1
#define H2_PEAK_EX2 2
int h2_measure_peak(int unit, double target_ms, double *rate, double *ms);

/* Static description of a status code. */
const char *h2_status_str(int status);

#ifdef __cplusplus
}
#endif

#endif /* H2_H */
