// h2_device.cu -- device copy of the H^2 operator, the product and the C ABI entry points.
//
// h2_upload materialises the operator in HBM: leaf bases and transfers are copied from
// the host build; coupling blocks S_ts = kappa(xi_t, xi_s) and dense blocks are generated
// on the device in FP64 and rounded once to the requested precision (each GPU populates
// its own blocks, Sec. 2.2). h2_matvec runs Sec. 3 as: leaf projection -> upsweep levels
// (Alg 1) -> all-level coupling product (Alg 4) -> downsweep levels (Alg 6) -> leaf
// expansion fused with the dense near field result and the alpha/beta epilogue.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "h2_internal.h"
#include "h2_kernels.cuh"

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x, size_t a = kAlign) { return (x + a - 1) / a * a; }

}  // namespace

struct h2_device {
    int device = -1;
    h2_prec prec = H2_FP64;
    size_t esize = 8;
    void *arena = nullptr;  // one allocation for the whole operator
    size_t arena_bytes = 0;
    // views into the arena
    int32_t *perm = nullptr;       // n
    int32_t *leaf_lo = nullptr;    // nleaves + 1
    void *U = nullptr;             // n * k
    void *E = nullptr;             // (nnodes + 1) * k * k
    int64_t *cpl_rowptr = nullptr; // nnodes + 2
    int32_t *cpl_col = nullptr;    // ncpl
    int32_t *cpl_rows = nullptr;   // non-empty block rows (heap indices)
    int64_t n_cpl_rows = 0;
    void *S = nullptr;             // ncpl * k * k
    int64_t *dns_rowptr = nullptr; // nleaves + 1
    int32_t *dns_col = nullptr;    // ndns
    int64_t *dns_off = nullptr;    // ndns + 1
    void *D = nullptr;
    int max_leaf_rows = 0;
    // handle-owned workspace for h2_matvec
    void *ws = nullptr;
    size_t ws_bytes = 0;
    // instrumentation (not synchronised between host threads)
    bool timing = false;
    struct PhaseRec {
        int phase;
        cudaEvent_t a, b;
    };
    std::vector<cudaEvent_t> event_pool;
    std::vector<PhaseRec> pending;
    double phase_ms[H2_NPHASES] = {};
    int64_t phase_launches[H2_NPHASES] = {};
    int64_t products = 0;

    cudaEvent_t event()
    {
        cudaEvent_t e = nullptr;
        if (!event_pool.empty()) {
            e = event_pool.back();
            event_pool.pop_back();
        } else {
            cudaEventCreate(&e);
        }
        return e;
    }
    // Opens a phase on stream st; returns the start event (null when timing is off).
    cudaEvent_t begin(cudaStream_t st)
    {
        if (!timing) return nullptr;
        cudaEvent_t a = event();
        cudaEventRecord(a, st);
        return a;
    }
    void end(int phase, cudaEvent_t a, cudaStream_t st, int launches)
    {
        phase_launches[phase] += launches;
        if (!a) return;
        cudaEvent_t b = event();
        cudaEventRecord(b, st);
        pending.push_back({phase, a, b});
    }
    void drain()
    {
        for (auto &r : pending) {
            float ms = 0.f;
            cudaEventSynchronize(r.b);
            cudaEventElapsedTime(&ms, r.a, r.b);
            phase_ms[r.phase] += ms;
            event_pool.push_back(r.a);
            event_pool.push_back(r.b);
        }
        pending.clear();
    }
    ~h2_device()
    {
        drain();
        for (auto e : event_pool) cudaEventDestroy(e);
    }
};

namespace {

struct Workspace {
    void *xt, *yd, *xh, *yh;
};

size_t ws_layout(const h2_op &op, size_t esize, int nv, Workspace *w, void *base)
{
    nv = std::min(nv, 32);  // products run in chunks of at most 32 vectors
    const size_t vec = align_up(size_t(op.n) * nv * esize);
    const size_t tree = align_up(size_t(op.nnodes + 1) * op.k * nv * esize);
    if (w) {
        char *p = static_cast<char *>(base);
        w->xt = p;
        w->yd = p + vec;
        w->xh = p + 2 * vec;
        w->yh = p + 2 * vec + tree;
    }
    return 2 * vec + 2 * tree;
}

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return H2_OK;
    if (e == cudaErrorMemoryAllocation) return H2_ENOMEM;
    return H2_ECUDA;
}

// Vectors are processed in chunks of at most kMaxChunk columns per pass.
constexpr int kMaxChunk = 32;

template <typename T>
void raise_smem_limits()
{
    static bool done = false;  // attributes are per device function; set once per process
    if (done) return;
    const int lim = 160 * 1024;
    cudaFuncSetAttribute(h2k::downsweep_level<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(h2k::leaf_expand<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(h2k::upsweep_level<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(h2k::leaf_project<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    done = true;
}

template <typename T>
int launch_matvec(const h2_op &op, h2_device &dv, const T *X, T *Y, int nv, double alpha, double beta,
                  const Workspace &w, cudaStream_t st)
{
    using namespace h2k;
    raise_smem_limits<T>();
    const int k = op.k;
    const int64_t n = op.n, first_leaf = op.first_leaf(), nleaves = op.nleaves();
    const T *U = static_cast<const T *>(dv.U);
    const T *E = static_cast<const T *>(dv.E);
    T *xt = static_cast<T *>(w.xt), *yd = static_cast<T *>(w.yd);
    T *xh = static_cast<T *>(w.xh), *yh = static_cast<T *>(w.yh);

    // upsweep (Alg 1)
    cudaEvent_t ev = dv.begin(st);
    leaf_project<T><<<unsigned(nleaves), 64, op.m * sizeof(T), st>>>(X, n, nv, dv.perm, dv.leaf_lo, U, k, first_leaf,
                                                                      xt, xh);
    for (int l = op.q; l >= 1; --l) {
        const int64_t parents = int64_t(1) << (l - 1);
        upsweep_level<T><<<unsigned(parents), 64, 2 * k * nv * sizeof(T), st>>>(parents, E, xh, k, nv);
    }
    dv.end(0, ev, st, 1 + op.q);
    // tree multiply on all levels (Alg 4)
    ev = dv.begin(st);
    if (dv.n_cpl_rows > 0)
        coupling_rows<T><<<unsigned(dv.n_cpl_rows), 128, 128 * sizeof(T), st>>>(
            dv.cpl_rows, dv.cpl_rowptr, dv.cpl_col, static_cast<const T *>(dv.S), xh, yh, k, nv);
    dv.end(1, ev, st, dv.n_cpl_rows > 0 ? 1 : 0);
    // dense near field
    ev = dv.begin(st);
    {
        const int threads = std::max(128, (dv.max_leaf_rows + 31) / 32 * 32);
        dense_rows<T><<<unsigned(nleaves), threads, threads * sizeof(T), st>>>(
            dv.dns_rowptr, dv.dns_col, dv.dns_off, static_cast<const T *>(dv.D), dv.leaf_lo, xt, yd, n, nv);
    }
    dv.end(2, ev, st, 1);
    // downsweep (Alg 6)
    ev = dv.begin(st);
    for (int l = 1; l <= op.q; ++l) {
        const int64_t nodes = int64_t(1) << l;
        const size_t sm = (size_t(k) * (k + 1) + size_t(k) * nv) * sizeof(T);
        downsweep_level<T><<<unsigned(nodes), 64, sm, st>>>(nodes, E, yh, dv.cpl_rowptr, k, nv, l == 1);
    }
    // leaf expansion + dense + epilogue
    {
        const bool yh_valid = op.q > 0 || op.cpl_rowptr[2] > op.cpl_rowptr[1];
        const size_t sm = (64 * size_t(k + 1) + size_t(k) * nv) * sizeof(T);
        leaf_expand<T><<<unsigned(nleaves), 128, sm, st>>>(U, yh, yd, dv.perm, dv.leaf_lo, first_leaf, k, nv, n,
                                                           yh_valid, T(alpha), T(beta), Y);
    }
    dv.end(3, ev, st, op.q + 1);
    return cuda_status(cudaGetLastError());
}

template <typename T>
int generate_blocks(const h2_op &op, h2_device &dv, const int32_t *d_cpl_row, const int32_t *d_dns_row,
                    const double *d_cheb, const double *d_pts_tree, cudaStream_t st)
{
    h2k::KernelFn f{int(op.ker.kind), op.ker.a, op.ker.b, op.ker.deg};
    const int64_t ncpl = int64_t(op.cpl_col.size()), ndns = int64_t(op.dns_col.size());
    if (ncpl > 0)
        h2k::gen_coupling<T><<<unsigned(std::min<int64_t>(ncpl, 1 << 20)), 256, 0, st>>>(
            static_cast<T *>(dv.S), d_cpl_row, dv.cpl_col, ncpl, d_cheb, op.dim, op.p, op.k, f);
    if (ndns > 0)
        h2k::gen_dense<T><<<unsigned(std::min<int64_t>(ndns, 1 << 20)), 256, 0, st>>>(
            static_cast<T *>(dv.D), dv.dns_off, d_dns_row, dv.dns_col, ndns, dv.leaf_lo, d_pts_tree, op.dim, f);
    return cuda_status(cudaGetLastError());
}

}  // namespace

void h2_device_free(h2_op *op)
{
    if (!op || !op->dev) return;
    int prev = -1;
    cudaGetDevice(&prev);
    if (op->dev->device >= 0) cudaSetDevice(op->dev->device);
    if (op->dev->arena) cudaFree(op->dev->arena);
    if (op->dev->ws) cudaFree(op->dev->ws);
    if (prev >= 0) cudaSetDevice(prev);
    delete op->dev;
    op->dev = nullptr;
}

extern "C" {

int h2_upload(h2_handle h, h2_prec prec, void *cuda_stream)
{
    if (!h) return H2_EINVAL;
    if (prec != H2_FP64 && prec != H2_FP32) return H2_EINVAL;  // split-BF16: multi-RHS module
    h2_op &op = *h;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    h2_device_free(&op);
    h2_device *dv = new (std::nothrow) h2_device;
    if (!dv) return H2_ENOMEM;
    op.dev = dv;
    cudaGetDevice(&dv->device);
    dv->prec = prec;
    dv->esize = prec == H2_FP64 ? 8 : 4;
    const size_t es = dv->esize;
    const int k = op.k;
    const int64_t nleaves = op.nleaves(), ncpl = int64_t(op.cpl_col.size()), ndns = int64_t(op.dns_col.size());

    // host-side index arrays
    std::vector<int32_t> perm32(op.n), leaf_lo(nleaves + 1), cpl_rows, cpl_row(ncpl), dns_row(ndns);
    std::vector<int64_t> dns_off(ndns + 1);
    for (int64_t i = 0; i < op.n; ++i) perm32[i] = int32_t(op.perm[i]);
    for (int64_t t = 0; t < nleaves; ++t) leaf_lo[t] = int32_t(op.lo[op.first_leaf() + t]);
    leaf_lo[nleaves] = int32_t(op.n);
    dv->max_leaf_rows = 0;
    for (int64_t t = 0; t < nleaves; ++t) dv->max_leaf_rows = std::max(dv->max_leaf_rows, leaf_lo[t + 1] - leaf_lo[t]);
    for (int64_t t = 1; t <= op.nnodes; ++t) {
        if (op.cpl_rowptr[t + 1] > op.cpl_rowptr[t]) cpl_rows.push_back(int32_t(t));
        for (int64_t b = op.cpl_rowptr[t]; b < op.cpl_rowptr[t + 1]; ++b) cpl_row[b] = int32_t(t);
    }
    dv->n_cpl_rows = int64_t(cpl_rows.size());
    const int64_t blk_align = 32;  // each dense block starts on a 128-byte boundary (FP32)
    dns_off[0] = 0;
    for (int64_t t = 0; t < nleaves; ++t)
        for (int64_t b = op.dns_rowptr[t]; b < op.dns_rowptr[t + 1]; ++b) {
            dns_row[b] = int32_t(t);
            const int64_t s = op.dns_col[b];
            const int64_t cnt = int64_t(leaf_lo[t + 1] - leaf_lo[t]) * (leaf_lo[s + 1] - leaf_lo[s]);
            dns_off[b + 1] = dns_off[b] + (cnt + blk_align - 1) / blk_align * blk_align;
        }
    std::vector<double> pts_tree(op.n * op.dim);
    for (int64_t i = 0; i < op.n; ++i)
        for (int d = 0; d < op.dim; ++d) pts_tree[i * op.dim + d] = op.pts[op.perm[i] * op.dim + d];

    // arena layout: persistent part
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += align_up(std::max<size_t>(bytes, 1));
        return o;
    };
    const size_t o_perm = take(op.n * 4), o_leaf = take((nleaves + 1) * 4);
    const size_t o_U = take(size_t(op.n) * k * es), o_E = take(size_t(op.nnodes + 1) * k * k * es);
    const size_t o_cptr = take((op.nnodes + 2) * 8), o_ccol = take(ncpl * 4), o_crows = take(cpl_rows.size() * 4);
    const size_t o_S = take(size_t(ncpl) * k * k * es);
    const size_t o_dptr = take((nleaves + 1) * 8), o_dcol = take(ndns * 4), o_doff = take((ndns + 1) * 8);
    const size_t o_D = take(size_t(dns_off[ndns]) * es);
    const size_t persistent = off;
    // temporaries for generation (freed after upload)
    const size_t t_cheb = op.cheb.size() * 8, t_pts = pts_tree.size() * 8, t_crow = ncpl * 4, t_drow = ndns * 4;
    const size_t tmp_bytes = align_up(t_cheb) + align_up(t_pts) + align_up(t_crow) + align_up(t_drow) + 4 * kAlign;

    char *arena = nullptr;
    if (cudaMalloc(&arena, persistent) != cudaSuccess) {
        cudaGetLastError();
        h2_device_free(&op);
        return H2_ENOMEM;
    }
    dv->arena = arena;
    dv->arena_bytes = persistent;
    char *tmp = nullptr;
    if (cudaMalloc(&tmp, tmp_bytes) != cudaSuccess) {
        cudaGetLastError();
        h2_device_free(&op);
        return H2_ENOMEM;
    }
    dv->perm = reinterpret_cast<int32_t *>(arena + o_perm);
    dv->leaf_lo = reinterpret_cast<int32_t *>(arena + o_leaf);
    dv->U = arena + o_U;
    dv->E = arena + o_E;
    dv->cpl_rowptr = reinterpret_cast<int64_t *>(arena + o_cptr);
    dv->cpl_col = reinterpret_cast<int32_t *>(arena + o_ccol);
    dv->cpl_rows = reinterpret_cast<int32_t *>(arena + o_crows);
    dv->S = arena + o_S;
    dv->dns_rowptr = reinterpret_cast<int64_t *>(arena + o_dptr);
    dv->dns_col = reinterpret_cast<int32_t *>(arena + o_dcol);
    dv->dns_off = reinterpret_cast<int64_t *>(arena + o_doff);
    dv->D = arena + o_D;
    double *d_cheb = reinterpret_cast<double *>(tmp);
    double *d_pts = reinterpret_cast<double *>(tmp + align_up(t_cheb));
    int32_t *d_crow = reinterpret_cast<int32_t *>(tmp + align_up(t_cheb) + align_up(t_pts));
    int32_t *d_drow = reinterpret_cast<int32_t *>(tmp + align_up(t_cheb) + align_up(t_pts) + align_up(t_crow));

    // bases in the target precision
    std::vector<unsigned char> Ubuf(size_t(op.n) * k * es), Ebuf(size_t(op.nnodes + 1) * k * k * es);
    if (es == 8) {
        std::memcpy(Ubuf.data(), op.U.data(), Ubuf.size());
        std::memcpy(Ebuf.data(), op.E.data(), Ebuf.size());
    } else {
        float *u = reinterpret_cast<float *>(Ubuf.data()), *e = reinterpret_cast<float *>(Ebuf.data());
        for (size_t i = 0; i < op.U.size(); ++i) u[i] = float(op.U[i]);
        for (size_t i = 0; i < op.E.size(); ++i) e[i] = float(op.E[i]);
    }
    int rc = H2_OK;
    auto cp = [&](void *dst, const void *src, size_t bytes) {
        if (rc == H2_OK && bytes) rc = cuda_status(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st));
    };
    cp(dv->perm, perm32.data(), op.n * 4);
    cp(dv->leaf_lo, leaf_lo.data(), (nleaves + 1) * 4);
    cp(dv->U, Ubuf.data(), Ubuf.size());
    cp(dv->E, Ebuf.data(), Ebuf.size());
    cp(dv->cpl_rowptr, op.cpl_rowptr.data(), (op.nnodes + 2) * 8);
    cp(dv->cpl_col, op.cpl_col.data(), ncpl * 4);
    cp(dv->cpl_rows, cpl_rows.data(), cpl_rows.size() * 4);
    cp(dv->dns_rowptr, op.dns_rowptr.data(), (nleaves + 1) * 8);
    cp(dv->dns_col, op.dns_col.data(), ndns * 4);
    cp(dv->dns_off, dns_off.data(), (ndns + 1) * 8);
    cp(d_cheb, op.cheb.data(), t_cheb);
    cp(d_pts, pts_tree.data(), t_pts);
    cp(d_crow, cpl_row.data(), t_crow);
    cp(d_drow, dns_row.data(), t_drow);
    if (rc == H2_OK)
        rc = es == 8 ? generate_blocks<double>(op, *dv, d_crow, d_drow, d_cheb, d_pts, st)
                     : generate_blocks<float>(op, *dv, d_crow, d_drow, d_cheb, d_pts, st);
    if (rc == H2_OK) rc = cuda_status(cudaStreamSynchronize(st));
    cudaFree(tmp);
    if (rc != H2_OK) h2_device_free(&op);
    return rc;
}

size_t h2_workspace_bytes(h2_handle h, int nv)
{
    if (!h || !h->dev || nv < 1) return 0;
    return ws_layout(*h, h->dev->esize, nv, nullptr, nullptr);
}

int h2_matvec_ws(h2_handle h, const void *X, void *Y, int nv, double alpha, double beta, void *workspace,
                 size_t ws_bytes, void *cuda_stream)
{
    if (!h || !X || !Y || nv < 1 || !workspace) return H2_EINVAL;
    if (!h->dev) return H2_ESTATE;
    const h2_device &dv = *h->dev;
    if (ws_bytes < ws_layout(*h, dv.esize, nv, nullptr, nullptr)) return H2_EINVAL;
    if (reinterpret_cast<uintptr_t>(workspace) % kAlign) return H2_EINVAL;
    Workspace w;
    ws_layout(*h, dv.esize, nv, &w, workspace);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    h2_device &dvm = *h->dev;
    dvm.products += 1;
    for (int v0 = 0; v0 < nv; v0 += kMaxChunk) {
        const int c = std::min(kMaxChunk, nv - v0);
        const size_t o = size_t(v0) * h->n;
        const int rc = dv.esize == 8
                           ? launch_matvec<double>(*h, dvm, static_cast<const double *>(X) + o,
                                                   static_cast<double *>(Y) + o, c, alpha, beta, w, st)
                           : launch_matvec<float>(*h, dvm, static_cast<const float *>(X) + o,
                                                  static_cast<float *>(Y) + o, c, alpha, beta, w, st);
        if (rc != H2_OK) return rc;
    }
    return H2_OK;
}

int h2_matvec(h2_handle h, const void *X, void *Y, int nv, double alpha, double beta, void *cuda_stream)
{
    if (!h || !X || !Y || nv < 1) return H2_EINVAL;
    if (!h->dev) return H2_ESTATE;
    h2_device &dv = *h->dev;
    const size_t need = ws_layout(*h, dv.esize, nv, nullptr, nullptr);
    if (dv.ws_bytes < need) {
        if (dv.ws) {
            cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream));
            cudaFree(dv.ws);
            dv.ws = nullptr;
            dv.ws_bytes = 0;
        }
        if (cudaMalloc(&dv.ws, need) != cudaSuccess) {
            cudaGetLastError();
            dv.ws = nullptr;
            return H2_ENOMEM;
        }
        dv.ws_bytes = need;
    }
    return h2_matvec_ws(h, X, Y, nv, alpha, beta, dv.ws, dv.ws_bytes, cuda_stream);
}

int h2_set_timing(h2_handle h, int enable)
{
    if (!h) return H2_EINVAL;
    if (!h->dev) return H2_ESTATE;
    h->dev->timing = enable != 0;
    return H2_OK;
}

int h2_get_timing(h2_handle h, double *phase_ms, int64_t *phase_launches, int64_t *products)
{
    if (!h) return H2_EINVAL;
    if (!h->dev) return H2_ESTATE;
    h2_device &dv = *h->dev;
    dv.drain();
    for (int i = 0; i < H2_NPHASES; ++i) {
        if (phase_ms) phase_ms[i] = dv.phase_ms[i];
        if (phase_launches) phase_launches[i] = dv.phase_launches[i];
        dv.phase_ms[i] = 0;
        dv.phase_launches[i] = 0;
    }
    if (products) *products = dv.products;
    dv.products = 0;
    return cuda_status(cudaGetLastError());
}

int h2_destroy(h2_handle h)
{
    if (!h) return H2_OK;
    h2_device_free(h);
    delete h;
    return H2_OK;
}

int h2_build(const double *points, int64_t n, int dim, h2_kernel kernel, int leaf_size, int cheb_order, double eta,
             h2_handle *out)
{
    if (!out) return H2_EINVAL;
    *out = nullptr;
    h2_op *op = new (std::nothrow) h2_op;
    if (!op) return H2_ENOMEM;
    const int rc = h2_host_build(op, points, n, dim, kernel, leaf_size, cheb_order, eta);
    if (rc != H2_OK) {
        delete op;
        return rc;
    }
    *out = op;
    return H2_OK;
}

int h2_get_info(h2_handle h, h2_info *info)
{
    if (!h || !info) return H2_EINVAL;
    const h2_op &op = *h;
    std::memset(info, 0, sizeof(*info));
    info->n = op.n;
    info->dim = op.dim;
    info->depth = op.q;
    info->rank = op.k;
    info->leaf_size = op.m;
    info->cheb_order = op.p;
    info->eta = op.eta;
    info->n_nodes = op.nnodes;
    info->n_leaves = op.nleaves();
    info->n_coupling = int64_t(op.cpl_col.size());
    info->n_dense = int64_t(op.dns_col.size());
    int32_t cmax = 0, dmax = 0;
    for (int64_t t = 1; t <= op.nnodes; ++t) {
        const int64_t c = op.cpl_rowptr[t + 1] - op.cpl_rowptr[t];
        int l = 0;
        for (int64_t x = t; x > 1; x >>= 1) ++l;
        info->coupling_per_level[l] += c;
        cmax = std::max<int32_t>(cmax, int32_t(c));
    }
    int64_t dense_entries = 0;
    for (int64_t t = 0; t < op.nleaves(); ++t) {
        dmax = std::max<int32_t>(dmax, int32_t(op.dns_rowptr[t + 1] - op.dns_rowptr[t]));
        const int64_t rt = op.hi[op.first_leaf() + t] - op.lo[op.first_leaf() + t];
        for (int64_t b = op.dns_rowptr[t]; b < op.dns_rowptr[t + 1]; ++b) {
            const int64_t s = op.first_leaf() + op.dns_col[b];
            dense_entries += rt * (op.hi[s] - op.lo[s]);
        }
    }
    info->max_coupling_per_row = cmax;
    info->max_dense_per_row = dmax;
    info->coupling_entries = info->n_coupling * op.k * op.k;
    info->dense_entries = dense_entries;
    info->basis_entries = op.n * op.k;
    info->transfer_entries = (op.nnodes - 1) * op.k * op.k;
    info->uploaded_prec = op.dev ? int(op.dev->prec) : -1;
    info->device_bytes = op.dev ? op.dev->arena_bytes + op.dev->ws_bytes : 0;
    return H2_OK;
}

int h2_get_perm(h2_handle h, int64_t *perm)
{
    if (!h || !perm) return H2_EINVAL;
    std::memcpy(perm, h->perm.data(), h->n * sizeof(int64_t));
    return H2_OK;
}

int h2_get_coupling_csr(h2_handle h, int64_t *rowptr, int32_t *col)
{
    if (!h || !rowptr || (!col && !h->cpl_col.empty())) return H2_EINVAL;
    std::memcpy(rowptr, h->cpl_rowptr.data(), h->cpl_rowptr.size() * sizeof(int64_t));
    if (!h->cpl_col.empty()) std::memcpy(col, h->cpl_col.data(), h->cpl_col.size() * sizeof(int32_t));
    return H2_OK;
}

int h2_get_dense_csr(h2_handle h, int64_t *rowptr, int32_t *col)
{
    if (!h || !rowptr || (!col && !h->dns_col.empty())) return H2_EINVAL;
    std::memcpy(rowptr, h->dns_rowptr.data(), h->dns_rowptr.size() * sizeof(int64_t));
    if (!h->dns_col.empty()) std::memcpy(col, h->dns_col.data(), h->dns_col.size() * sizeof(int32_t));
    return H2_OK;
}

int h2_get_bases(h2_handle h, double *U, double *E)
{
    if (!h) return H2_EINVAL;
    if (U) std::memcpy(U, h->U.data(), h->U.size() * sizeof(double));
    if (E) std::memcpy(E, h->E.data(), h->E.size() * sizeof(double));
    return H2_OK;
}

const char *h2_status_str(int status)
{
    switch (status) {
    case H2_OK: return "ok";
    case H2_EINVAL: return "invalid argument";
    case H2_ENOMEM: return "out of memory";
    case H2_ECUDA: return "CUDA error";
    case H2_ETIMEOUT: return "device wait timed out";
    case H2_ESTATE: return "invalid handle state";
    case H2_ENOTCONV: return "not converged";
    default: return "unknown status";
    }
}

int h2_cg_solve(h2_handle h, double sigma2, const double *b, double *x, double tol, int maxit, int *iters,
                double *true_relres, void *cuda_stream)
{
    (void)sigma2; (void)b; (void)x; (void)tol; (void)maxit; (void)iters; (void)true_relres; (void)cuda_stream;
    if (!h) return H2_EINVAL;
    return H2_ESTATE;  // provided by the solver module
}

}  // extern "C"
