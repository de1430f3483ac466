// h2_device.cu -- device copy of the H^2 operator, the product and the C ABI entry points.
//
// h2_upload materialises the operator in HBM: leaf bases and transfers come from the host
// build (plus transposed copies for the downsweep), coupling blocks S_ts = kappa(xi_t, xi_s)
// and dense blocks are generated on the device in FP64 and rounded once to the requested
// precision (each GPU populates its own blocks, Sec. 2.2). It also builds the flat list of
// tile descriptors that the streaming kernel walks, split over persistent CTAs by bytes.
//
// h2_matvec runs the three phases of Sec. 3 plus the dense product on two streams:
//   stream A: gather -> bottom upsweep (leaves + lowest L levels, Alg 1) -> streaming
//             product of every coupling row of the lower levels and every dense row
//             (Alg 4 + A_de x) -> [join] -> bottom downsweep + leaf expansion + epilogue (Alg 6)
//   stream B: [after the bottom upsweep] top upsweep levels -> coupling rows of the top
//             levels -> top downsweep levels -> [join]
// Stream B's latency-bound small levels run underneath stream A's bandwidth-bound stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "h2_internal.h"
#include "h2_kernels.cuh"
#include "h2_stream.cuh"
#include "h2_tcstream.cuh"
#include "h2_tf32stream.cuh"
#include "h2_batch.cuh"
#include "h2_mf.cuh"
#include "h2_warpsweep.cuh"
#include "h2_nvtx.h"

#include <dlfcn.h>

#include <chrono>
#include <cstdlib>
#include <fstream>
#include <memory>
#include <mutex>
#include <sstream>
#include <string>

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x, size_t a = kAlign) { return (x + a - 1) / a * a; }
inline int round4(int x) { return (x + 3) / 4 * 4; }

// Column chunk of one product pass (the streaming kernels keep nv <= 4 accumulators).
constexpr int kChunk = 4;
constexpr int kMaxLeaf = 128;

}  // namespace

struct h2_device {
    int device = -1;
    int num_sms = 0;
    h2_prec prec = H2_FP64;
    size_t esize = 8;
    void *arena = nullptr;  // one allocation for the whole operator
    size_t arena_bytes = 0;
    // layout
    int kx = 0, mp = 0, L = 0, Lb = 0;
    int64_t kkp = 0;
    int max_leaf_rows = 0;
    bool root_row = false;  // the root has coupling blocks
    bool tc = false;        // split-BF16 blocks for the tensor-core stream (H2_BF16X2)
    // FP32 operators with ranks and leaves of at most 64: passes of more than 8 vectors run on
    // the tensor cores (3xTF32, k_stream_tf32) unless switched off by h2_set_fp32_tensor
    bool tf32_ok = false, tf32_on = true;
    // ranks of at most 32: single-vector products run the warp-granular kernels of
    // h2_warpsweep.cuh (bottom subtrees one CTA each, upper levels one warp per node,
    // coupling rows one warp per chunk) instead of the staged subtree kernels and streams
    bool warp_sweeps = false;
    // FP32 ranks 33 .. 64: single-vector products run the bottom subtrees' downsweep with one
    // CTA each, two warps per node (k_down_cta2)
    bool cta64 = false;
    // views into the arena
    int32_t *perm = nullptr, *leaf_lo = nullptr;
    int64_t *cpl_rowptr = nullptr;
    void *U = nullptr, *Ut = nullptr, *E = nullptr, *Et = nullptr;
    unsigned char *vals = nullptr;  // coupling blocks, then dense blocks
    h2s::StreamDesc *desc_bottom = nullptr, *desc_top = nullptr;
    int64_t *chunks_bottom = nullptr, *chunks_top = nullptr;  // (first << 16) | count
    // when dense tiles are at least twice the coupling tiles (small ranks, e.g. after
    // recompression), the bottom list's dense rows get a stream of their own: each stream's
    // stages are sized for its own tiles, so small coupling tiles get a deep pipeline.
    // chunks_bottom then covers the coupling rows, chunks_dense the dense rows (descriptor
    // indices into the same desc_bottom array); otherwise n_chunks_dense = 0
    int64_t *chunks_dense = nullptr;
    int64_t n_chunks_dense = 0;
    int grid_dense = 0;
    uint32_t tile_cpl = 0, tile_dns = 0;  // bytes of the largest coupling / dense tile
    int grid_bottom = 0, grid_top = 0;
    int64_t n_chunks_bottom = 0, n_chunks_top = 0;
    int64_t n_desc_bottom = 0, n_desc_top = 0;
    int *err = nullptr;  // device error flag (a bounded wait ran out)
    // matrix-free FP32 (H2_FP32_MF): coordinates instead of blocks
    bool mf = false;
    h2s::MfArgs mfa{};
    // fork/join contexts (side stream + events) of products in flight on the host: a product
    // takes an idle one for its launch sequence and gives it back (calls from several host
    // threads never share one); the first is created at upload
    std::mutex exec_mutex;
    std::vector<h2_exec> exec_idle, exec_all;
    // h2_matvec's workspaces, one per CUDA stream it has been called with; `done` is recorded
    // after each product, and the next product on that workspace waits for it
    struct StreamWs {
        void *stream = nullptr;
        void *ws = nullptr;
        size_t bytes = 0;
        cudaEvent_t done = nullptr;
        std::mutex m;  // held while a product is enqueued on this workspace
    };
    std::mutex ws_mutex;
    std::vector<std::unique_ptr<StreamWs>> stream_ws;
    size_t ws_total = 0;  // bytes of all stream workspaces
    // instrumentation: the launch and product counters are atomic; the event records of the
    // phase timing are guarded by timing_mutex
    bool timing = false;
    std::mutex timing_mutex;
    struct PhaseRec {
        int phase;
        cudaEvent_t a, b;
    };
    std::vector<cudaEvent_t> event_pool;
    std::vector<PhaseRec> pending;
    double phase_ms[H2_NPHASES] = {};
    std::atomic<int64_t> phase_launches[H2_NPHASES] = {};
    std::atomic<int64_t> products{0};

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
    cudaEvent_t begin(cudaStream_t st)
    {
        if (!timing) return nullptr;
        std::lock_guard<std::mutex> lock(timing_mutex);
        cudaEvent_t a = event();
        cudaEventRecord(a, st);
        return a;
    }
    void end(int phase, cudaEvent_t a, cudaStream_t st, int launches)
    {
        phase_launches[phase] += launches;
        if (!a) return;
        std::lock_guard<std::mutex> lock(timing_mutex);
        cudaEvent_t b = event();
        cudaEventRecord(b, st);
        pending.push_back({phase, a, b});
    }
    void drain()
    {
        std::lock_guard<std::mutex> lock(timing_mutex);
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
        for (auto &x : exec_all) h2_exec_destroy(&x);
        for (auto &w : stream_ws) {
            if (w->ws) cudaFree(w->ws);
            if (w->done) cudaEventDestroy(w->done);
        }
    }
};

namespace {

struct Workspace {
    void *xt, *yd, *xh, *yh;
    int *tickets;
    int *flags = nullptr;  // warp sweeps: 2 (nnodes + 1) node flags, upsweep then downsweep
    // tensor-core path (H2_BF16X2): split-BF16 vector tiles of the coefficient tree and of
    // the permuted input
    unsigned char *xb = nullptr, *xtb = nullptr;
    // wide passes: row-major copy of X, later of the result rows (n x round4(pass vectors))
    void *rows = nullptr;
};

constexpr int kTcSmemBudget = 224 * 1024;  // dynamic shared memory of the tensor-core stream
constexpr int kTfSmemBudget = 227 * 1024;  // of the 3xTF32 stream: the most one CTA may have
constexpr int kWidePass = 32;  // vectors per pass of the wide kernels and of the tensor-core stream

inline int pad16(int x) { return (x + 15) / 16 * 16; }

// The wide accumulator holds tiles of at most 64 outputs.
inline bool wide_ok(const h2_device &dv) { return dv.kx <= 64 && dv.mp <= 64; }

// FP32 passes of this many vectors run on the tensor cores (3xTF32).
inline bool tf32_pass(const h2_device &dv, int vp) { return dv.tf32_ok && dv.tf32_on && vp > 8; }

// Vectors per pass: up to kWidePass on the tensor-core path and, for more than kChunk
// vectors, on the wide kernels; otherwise kChunk.
inline int pass_vectors(const h2_device &dv, int nv)
{
    if (dv.mf) return std::min(nv, kChunk);
    if (dv.tc || (nv > kChunk && wide_ok(dv))) return std::min(nv, kWidePass);
    return std::min(nv, kChunk);
}

// Workspace for one pass of vp vectors: permuted input and dense result ([leaf][v][mp]),
// coefficient trees xhat and yhat ([node][v][kx]), the split-BF16 vector tiles of the
// tensor-core path, the row-major staging buffer of wide passes, and the scheduling tickets.
size_t ws_layout(const h2_op &op, const h2_device &dv, int nv, Workspace *w, void *base)
{
    const int vp = pass_vectors(dv, nv), np = pad16(vp);
    const bool wide = vp > kChunk || dv.tc;
    const bool tiles = dv.tc;
    const size_t tile_bytes = h2s::vec_tile_bytes(np);
    const size_t es = dv.esize;
    const size_t vec = align_up(size_t(op.nleaves()) * vp * dv.mp * es);
    const size_t tree = align_up(size_t(op.nnodes + 1) * vp * dv.kx * es);
    const size_t xb = tiles ? align_up(size_t(op.nnodes + 1) * tile_bytes) : 0;
    const size_t xtb = tiles ? align_up(size_t(op.nleaves()) * tile_bytes) : 0;
    const size_t rows = wide ? align_up(size_t(op.n) * round4(vp) * es) : 0;
    const size_t flags = dv.warp_sweeps ? align_up(size_t(2) * (op.nnodes + 1) * sizeof(int)) : 0;
    static_assert(h2s::kTickets * sizeof(int) <= kAlign, "scheduling words fit the ticket slot");
    if (w) {
        char *p = static_cast<char *>(base);
        w->xt = p;
        w->yd = p + vec;
        w->xh = p + 2 * vec;
        w->yh = p + 2 * vec + tree;
        w->xb = tiles ? reinterpret_cast<unsigned char *>(p + 2 * vec + 2 * tree) : nullptr;
        w->xtb = tiles ? w->xb + xb : nullptr;
        w->rows = wide ? p + 2 * vec + 2 * tree + xb + xtb : nullptr;
        w->tickets = reinterpret_cast<int *>(p + 2 * vec + 2 * tree + xb + xtb + rows);
        w->flags = dv.warp_sweeps ? reinterpret_cast<int *>(p + 2 * vec + 2 * tree + xb + xtb + rows + kAlign) : nullptr;
    }
    return 2 * vec + 2 * tree + xb + xtb + rows + kAlign + flags;
}

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return H2_OK;
    if (e == cudaErrorMemoryAllocation) return H2_ENOMEM;
    return H2_ECUDA;
}

template <typename T>
h2s::Op<T> make_op(const h2_op &op, const h2_device &dv)
{
    h2s::Op<T> o;
    o.n = op.n;
    o.nleaves = op.nleaves();
    o.first_leaf = op.first_leaf();
    o.k = op.k;
    o.kx = dv.kx;
    o.mp = dv.mp;
    o.q = op.q;
    o.perm = dv.perm;
    o.leaf_lo = dv.leaf_lo;
    o.U = static_cast<const T *>(dv.U);
    o.Ut = static_cast<const T *>(dv.Ut);
    o.E = static_cast<const T *>(dv.E);
    o.Et = static_cast<const T *>(dv.Et);
    o.vals = dv.vals;
    return o;
}

// Stage sizing for a kernel: as many stages as fit in `budget` bytes of shared memory.
template <typename T, int NVMAX>
h2s::Pipe make_pipe(uint32_t tile_bytes, uint32_t x_bytes, int sub_nodes, int kx, bool chunks, size_t budget,
                    int max_ns)
{
    h2s::Pipe p{1, tile_bytes, x_bytes};
    for (int ns = max_ns; ns >= 1; --ns) {
        p.ns = ns;
        if (h2s::smem_bytes<T, NVMAX>(p, sub_nodes, kx, chunks) <= budget) break;
    }
    return p;
}

// The FP64 single-vector block stream runs 256 consumer threads (the FP64 pipe bounds it, and
// eight consumer warps per SM keep it busier than four).
template <typename T, int NVMAX>
constexpr int stream_consumers()
{
    return (sizeof(T) == 8 && NVMAX == 1) ? 2 * h2s::kConsumers : h2s::kConsumers;
}

template <typename T, int NVMAX>
void set_kernel_attributes()
{
    static bool done = false;  // per template instance
    if (done) return;
    for (const void *f : {(const void *)h2s::k_up_sub<T, NVMAX>, (const void *)h2s::k_down_sub<T, NVMAX>,
                          (const void *)h2s::k_stream<T, NVMAX>,
                          (const void *)h2s::k_stream<T, NVMAX, stream_consumers<T, NVMAX>()>}) {
        cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        // the largest shared-memory carveout lets the side stream's kernels become
        // resident next to the persistent streaming kernel
        cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    }
    done = true;
}

// Matrix-free stream launch for the operator's kernel kind and dimension (FP32 only).
template <int KIND, int DIM, int NVMAX>
void launch_mf_kind(const h2s::Op<float> &o, const h2s::Vec<float> &v, const h2s::MfArgs &ma, const h2s::Pipe &p,
                    size_t smem, unsigned grid, const h2s::StreamDesc *desc, const int64_t *chunks, int64_t nchunks,
                    int ticket, cudaStream_t st)
{
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(h2s::k_stream_mf<KIND, DIM, NVMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024);
        cudaFuncSetAttribute(h2s::k_stream_mf<KIND, DIM, NVMAX>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        attr = true;
    }
    h2s::k_stream_mf<KIND, DIM, NVMAX><<<grid, h2s::kThreads, smem, st>>>(o, v, ma, p, desc, chunks, nchunks, ticket);
}

template <int DIM, int NVMAX>
void launch_mf_dim(int kind, const h2s::Op<float> &o, const h2s::Vec<float> &v, const h2s::MfArgs &ma,
                   const h2s::Pipe &p, size_t smem, unsigned grid, const h2s::StreamDesc *desc, const int64_t *chunks,
                   int64_t nchunks, int ticket, cudaStream_t st)
{
    switch (kind) {
    case H2_K_EXP:
        return launch_mf_kind<H2_K_EXP, DIM, NVMAX>(o, v, ma, p, smem, grid, desc, chunks, nchunks, ticket, st);
    case H2_K_GAUSS:
        return launch_mf_kind<H2_K_GAUSS, DIM, NVMAX>(o, v, ma, p, smem, grid, desc, chunks, nchunks, ticket, st);
    case H2_K_IMQ:
        return launch_mf_kind<H2_K_IMQ, DIM, NVMAX>(o, v, ma, p, smem, grid, desc, chunks, nchunks, ticket, st);
    default:
        return launch_mf_kind<H2_K_POLY, DIM, NVMAX>(o, v, ma, p, smem, grid, desc, chunks, nchunks, ticket, st);
    }
}

template <int NVMAX>
void launch_mf(const h2_op &op, const h2s::Op<float> &o, const h2s::Vec<float> &v, const h2s::MfArgs &ma,
               const h2s::Pipe &p, size_t smem, unsigned grid, const h2s::StreamDesc *desc, const int64_t *chunks,
               int64_t nchunks, int ticket, cudaStream_t st)
{
    if (op.dim == 3)
        launch_mf_dim<3, NVMAX>(op.ker.kind, o, v, ma, p, smem, grid, desc, chunks, nchunks, ticket, st);
    else
        launch_mf_dim<2, NVMAX>(op.ker.kind, o, v, ma, p, smem, grid, desc, chunks, nchunks, ticket, st);
}

template <typename T, int KM>
void launch_warp_sweep_km(bool up, const h2_op &op, const h2s::Op<T> &o, const h2s::Vec<T> &v, const h2_device &dv,
                          const Workspace &w, int lo, int hi, int ticket, cudaStream_t st)
{
    using namespace h2s;
    static int occ = 0;  // resident CTAs per SM (per element type and partial width)
    if (!occ) {
        int a = 0, b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_up_warp<T, KM>, kWsThreads, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_down_warp<T, KM>, kWsThreads, 0);
        occ = std::max(1, std::min(a, b));
    }
    // item levels lo .. last: the upsweep's last level is hi - 1, the downsweep's hi
    const int last = up ? hi - 1 : hi;
    if (last < lo) return;
    const int64_t items = (int64_t(2) << last) - (int64_t(1) << lo);
    const int64_t warps = (items + kWsChunk - 1) / kWsChunk;
    const int64_t ctas = std::min<int64_t>((warps + kWsWarps - 1) / kWsWarps, int64_t(dv.num_sms) * occ);
    const WarpSweep ws{w.tickets + ticket, w.tickets + 8, w.flags + (up ? 0 : op.nnodes + 1), lo, hi};
    if (up)
        k_up_warp<T, KM><<<unsigned(ctas), kWsThreads, 0, st>>>(o, v, ws);
    else
        k_down_warp<T, KM><<<unsigned(ctas), kWsThreads, 0, st>>>(o, v, ws);
}

// Bottom subtrees of small ranks, one vector: one CTA per subtree of depth L rooted at level
// Lr (k_up_cta / k_down_cta).
template <typename T, int KM>
void launch_cta_sweep_km(bool up, const h2s::Op<T> &o, const h2s::Vec<T> &v, int Lr, int L, cudaStream_t st)
{
    using namespace h2s;
    const size_t smem = cta_smem_bytes<T, KM>(L);
    const unsigned grid = unsigned(int64_t(1) << Lr);
    if (up)
        k_up_cta<T, KM><<<grid, kCtaThreads, smem, st>>>(o, v, Lr, L);
    else
        k_down_cta<T, KM><<<grid, kCtaThreads, smem, st>>>(o, v, Lr, L);
}

template <typename T>
void launch_cta_sweep(bool up, const h2_op &op, const h2s::Op<T> &o, const h2s::Vec<T> &v, int Lr, int L,
                      cudaStream_t st)
{
    if (op.k <= 16)
        launch_cta_sweep_km<T, 16>(up, o, v, Lr, L, st);
    else
        launch_cta_sweep_km<T, 32>(up, o, v, Lr, L, st);
}

// Bottom downsweep of ranks 33 .. 64, FP32, one vector: one CTA per subtree, two warps per
// node (k_down_cta2).
template <typename T>
void launch_cta2_down(const h2s::Op<T> &o, const h2s::Vec<T> &v, int Lr, int L, cudaStream_t st)
{
    if constexpr (sizeof(T) == 4) {
        using namespace h2s;
        k_down_cta2<T><<<unsigned(int64_t(1) << Lr), kCtaThreads, cta_smem_bytes<float, 64>(L), st>>>(o, v, Lr, L);
    }
}

// Coupling rows of small ranks, one vector: one warp per chunk of rows (k_rows_warp) on the
// scheduling word `ticket`, at most the CTAs resident on the device.
template <typename T, int KM>
void launch_rows_warp_km(const h2s::Op<T> &o, const h2s::Vec<T> &v, const h2_device &dv,
                         const h2s::StreamDesc *desc, const int64_t *chunks, int64_t nchunks, int ticket,
                         bool side, cudaStream_t st)
{
    using namespace h2s;
    static int occ = 0;
    if (!occ) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_rows_warp<T, KM>, kWsThreads, 0);
        occ = std::max(1, occ);
    }
    // a persistent launch that fills every register file would keep the side stream's
    // kernels (the upper levels) from starting until it ends: `side` leaves them one slot
    const int per_sm = side ? std::max(1, occ - 1) : occ;
    const int64_t ctas = std::min<int64_t>((nchunks + kWsWarps - 1) / kWsWarps, int64_t(dv.num_sms) * per_sm);
    k_rows_warp<T, KM><<<unsigned(std::max<int64_t>(1, ctas)), kWsThreads, 0, st>>>(o, v, desc, chunks, nchunks,
                                                                                   ticket);
}

template <typename T>
void launch_rows_warp(const h2_op &op, const h2s::Op<T> &o, const h2s::Vec<T> &v, const h2_device &dv,
                      const h2s::StreamDesc *desc, const int64_t *chunks, int64_t nchunks, int ticket, bool side,
                      cudaStream_t st)
{
    if (op.k <= 16)
        launch_rows_warp_km<T, 16>(o, v, dv, desc, chunks, nchunks, ticket, side, st);
    else
        launch_rows_warp_km<T, 32>(o, v, dv, desc, chunks, nchunks, ticket, side, st);
}

// One launch of a flag-ordered warp sweep of the upper levels (ranks <= 32, one vector;
// h2_warpsweep.cuh): enough warps for the launch's tickets, at most the CTAs resident on the
// device. Upsweep: levels hi-1 .. lo from level hi; downsweep: levels lo .. hi. `ticket` is
// the launch's scheduling word.
template <typename T>
void launch_warp_sweep(bool up, const h2_op &op, const h2s::Op<T> &o, const h2s::Vec<T> &v, const h2_device &dv,
                       const Workspace &w, int lo, int hi, int ticket, cudaStream_t st)
{
    if (op.k <= 16)
        launch_warp_sweep_km<T, 16>(up, op, o, v, dv, w, lo, hi, ticket, st);
    else
        launch_warp_sweep_km<T, 32>(up, op, o, v, dv, w, lo, hi, ticket, st);
}

template <typename T, int NVMAX>
int launch_chunk(const h2_op &op, h2_device &dv, const T *X, T *Y, int nv, double alpha, double beta,
                 const Workspace &w, cudaStream_t st, const h2_exec &ex)
{
    cudaStream_t side = static_cast<cudaStream_t>(ex.side);
    cudaEvent_t ev_up = static_cast<cudaEvent_t>(ex.ev_up), ev_top = static_cast<cudaEvent_t>(ex.ev_top);
    using namespace h2s;
    const uint32_t es = sizeof(T);
    const int k = op.k, kx = dv.kx, mp = dv.mp;
    Op<T> o = make_op<T>(op, dv);
    Vec<T> v{X, Y, nv, nv, T(alpha), T(beta), static_cast<T *>(w.xt), static_cast<T *>(w.yd), static_cast<T *>(w.xh),
             static_cast<T *>(w.yh), w.tickets, dv.err};
    const int Lbot = dv.L, Lb = dv.Lb;
    const int64_t nsub = int64_t(1) << Lb;
    // ranks of at most 32, one vector: the warp-granular kernels, one launch per part of the
    // tree (bottom subtrees, upper levels) and per row list
    const bool wsw = NVMAX == 1 && dv.warp_sweeps && w.flags;
    const bool c64 = NVMAX == 1 && sizeof(T) == 4 && dv.cta64;  // ranks 33 .. 64, FP32
    if (wsw) {
        v.flags = w.flags;
        v.nflags = 2 * (op.nnodes + 1);
    }
    // levels per launch above the bottom subtrees: as many as keep the subtree's vectors
    // within 16 KB of shared memory (at most 5)
    int Ltop = 1;
    while (Ltop < 5 && (size_t(4) << Ltop) * kx * NVMAX * es <= 16 * 1024) ++Ltop;

    // shared-memory plans: the bottom subtree kernels run two CTAs per SM; the streaming
    // kernel one CTA per SM, leaving room for one side-stream CTA next to it
    const uint32_t tile_sub = uint32_t(std::max({size_t(mp) * kx, size_t(k) * kx, size_t(k) * mp}) * es);
    const uint32_t x_sub = uint32_t(2 * std::max(mp, kx) * NVMAX * es);  // two vector segments per stage
    const Pipe p_bsub = make_pipe<T, NVMAX>(tile_sub, x_sub, 2 << Lbot, kx, false, 100 * 1024, 8);
    const Pipe p_tsub = make_pipe<T, NVMAX>(tile_sub, x_sub, 2 << Ltop, kx, false, 64 * 1024, 4);
    const size_t sm_bsub = smem_bytes<T, NVMAX>(p_bsub, 2 << Lbot, kx, false);
    const size_t sm_tsub = smem_bytes<T, NVMAX>(p_tsub, 2 << Ltop, kx, false);
    const uint32_t tile_str = uint32_t(((std::max<size_t>(size_t(k) * kx, size_t(mp) * dv.max_leaf_rows) * es) + 15) /
                                       16 * 16);
    const uint32_t x_str = uint32_t(std::max(mp, kx) * NVMAX * es);
    // matrix-free: no tiles; per stage the input segment and two coordinate lists; the
    // evaluation is bound by instruction issue and latency, so four small CTAs per SM
    // (16 consumer warps) share each SM, leaving room for the side stream's kernels
    const bool mf = dv.mf && sizeof(T) == 4;
    const uint32_t x_mf = mf_seg_bytes(kx, mp, NVMAX) + 2 * mf_coord_bytes(k, mp);
    // With a separate dense stream each stream's stages fit its own tiles. A stream CTA's
    // single producer thread starts about one block per 700 clocks, which is HBM speed for
    // 16 KB tiles but not for small ones: small coupling tiles run 2 or 4 CTAs per SM (each
    // with its own producer) within the same 160 KB.
    const bool dsplit = dv.n_chunks_dense > 0;
    const int cpl_per_sm = !dsplit ? 1 : dv.tile_cpl <= 4096 ? 4 : dv.tile_cpl <= 8192 ? 2 : 1;
    const Pipe p_bot = mf       ? make_pipe<T, NVMAX>(0, x_mf, 0, kx, true, 36 * 1024, 12)
                       : dsplit ? make_pipe<T, NVMAX>(dv.tile_cpl, uint32_t(kx * NVMAX * es), 0, kx, true,
                                                      160 * 1024 / size_t(cpl_per_sm), 32)
                                : make_pipe<T, NVMAX>(tile_str, x_str, 0, kx, true, 160 * 1024, 12);
    const Pipe p_dns = make_pipe<T, NVMAX>(dv.tile_dns, uint32_t(mp * NVMAX * es), 0, kx, true, 160 * 1024, 32);
    const size_t sm_dns = smem_bytes<T, NVMAX>(p_dns, 0, kx, true);
    // (the upper levels' coupling blocks are stored for the matrix-free precision too). The
    // upper rows hold coupling blocks only: stages sized for them keep this kernel small
    // enough to become resident next to the bottom streams.
    const Pipe p_top = make_pipe<T, NVMAX>(dv.tile_cpl, uint32_t(kx * NVMAX * es), 0, kx, true, 64 * 1024, 8);
    const size_t sm_bot = smem_bytes<T, NVMAX>(p_bot, 0, kx, true), sm_top = smem_bytes<T, NVMAX>(p_top, 0, kx, true);
    const unsigned grid_bot =
        mf ? unsigned(std::max<int64_t>(1, std::min<int64_t>(4 * int64_t(dv.num_sms), dv.n_chunks_bottom)))
           : unsigned(std::max<int64_t>(1, std::min<int64_t>(int64_t(cpl_per_sm) * dv.num_sms, dv.n_chunks_bottom)));
    set_kernel_attributes<T, NVMAX>();
    const int grid_bsub = int(std::min<int64_t>(nsub, int64_t(dv.num_sms) * 2));

    // ---- stream A: gather + bottom upsweep (leaf projections and the lowest Lbot levels)
    cudaEvent_t ev = dv.begin(st);
    {
        h2n::Range r("upsweep: leaf subtrees");
        k_gather<T><<<unsigned(std::min<int64_t>(op.nleaves(), 65535)), 128, 0, st>>>(o, v);
        if (wsw)
            launch_cta_sweep<T>(true, op, o, v, Lb, Lbot, st);
        else
            k_up_sub<T, NVMAX><<<grid_bsub, kThreads, sm_bsub, st>>>(o, v, p_bsub, Lb, Lbot, nsub, 1);
    }
    dv.end(0, ev, st, 2);
    const bool top = Lb >= 1;
    cudaEvent_t ev_topup = static_cast<cudaEvent_t>(ex.ev_topup);
    if (top) {
        cudaEventRecord(ev_up, st);
        cudaStreamWaitEvent(side, ev_up, 0);
    }
    cudaEvent_t eb = nullptr;
    int top_launches = 0;
    // ---- stream B, part 1: upsweep of the levels above the bottom subtrees
    auto top_up = [&]() {
        h2n::Range r("upsweep: upper levels");
        eb = dv.begin(side);
        if (wsw) {
            launch_warp_sweep<T>(true, op, o, v, dv, w, 0, Lb, 5, side);
            ++top_launches;
            return;
        }
        for (int lin = Lb; lin > 0;) {
            const int L = std::min(Ltop, lin), lr = lin - L;
            const int64_t ns = int64_t(1) << lr;
            k_up_sub<T, NVMAX><<<unsigned(std::min<int64_t>(ns, dv.num_sms)), kThreads, sm_tsub, side>>>(
                o, v, p_tsub, lr, L, ns, 0);
            ++top_launches;
            lin = lr;
        }
    };
    // The matrix-free stream keeps the SMs' issue slots busy, which slows latency-bound
    // kernels next to it several times: it starts only after the upper upsweep, which then
    // runs alone; the upper rows and downsweep overlap it.
    if (top && mf) {
        top_up();
        cudaEventRecord(ev_topup, side);
        cudaStreamWaitEvent(st, ev_topup, 0);
    }
    // ---- stream A: coupling rows of the lower levels + dense rows
    ev = dv.begin(st);
    if (dv.n_chunks_bottom > 0) {
        h2n::Range r("tree multiply + dense: lower levels");
        if (wsw && dsplit && !mf) {  // the bottom list holds coupling rows only
            launch_rows_warp<T>(op, o, v, dv, dv.desc_bottom, dv.chunks_bottom, dv.n_chunks_bottom, 0, top, st);
        } else if constexpr (sizeof(T) == 4 && NVMAX <= kChunk) {
            if (mf) {
                launch_mf<NVMAX>(op, o, v, dv.mfa, p_bot, sm_bot, grid_bot, dv.desc_bottom, dv.chunks_bottom,
                                 dv.n_chunks_bottom, 0, st);
            } else {
                k_stream<T, NVMAX><<<grid_bot, kThreads, sm_bot, st>>>(o, v, p_bot, dv.desc_bottom, dv.chunks_bottom,
                                                                       dv.n_chunks_bottom, 0);
            }
        } else {
            constexpr int C = stream_consumers<T, NVMAX>();
            k_stream<T, NVMAX, C><<<grid_bot, C + 32, sm_bot, st>>>(o, v, p_bot, dv.desc_bottom, dv.chunks_bottom,
                                                                    dv.n_chunks_bottom, 0);
        }
    }
    if (dsplit) {  // the dense rows, after the coupling rows on the same stream
        h2n::Range r("dense product");
        constexpr int C = (sizeof(T) == 4 && NVMAX <= kChunk) ? kConsumers : stream_consumers<T, NVMAX>();
        k_stream<T, NVMAX, C><<<dv.grid_dense, C + 32, sm_dns, st>>>(o, v, p_dns, dv.desc_bottom, dv.chunks_dense,
                                                                     dv.n_chunks_dense, 2);
    }
    dv.end(1, ev, st, (dv.n_chunks_bottom > 0 ? 1 : 0) + (dsplit ? 1 : 0));
    // ---- stream B, part 2: coupling rows of the upper levels, their downsweep
    if (top) {
        cudaStream_t sb = side;
        if (!mf) top_up();
        h2n::Range r("tree multiply + downsweep: upper levels");
        if (dv.n_chunks_top > 0) {
            if (wsw)
                launch_rows_warp<T>(op, o, v, dv, dv.desc_top, dv.chunks_top, dv.n_chunks_top, 1, false, sb);
            else
                k_stream<T, NVMAX><<<dv.grid_top, kThreads, sm_top, sb>>>(o, v, p_top, dv.desc_top, dv.chunks_top,
                                                                          dv.n_chunks_top, 1);
            ++top_launches;
        }
        if (wsw) {
            launch_warp_sweep<T>(false, op, o, v, dv, w, 0, Lb - 1, 6, sb);
            ++top_launches;
        } else {
            for (int lr = 0; lr <= Lb - 1;) {
                const int L = std::min(Ltop, Lb - 1 - lr);
                const int64_t ns = int64_t(1) << lr;
                k_down_sub<T, NVMAX><<<unsigned(std::min<int64_t>(ns, dv.num_sms)), kThreads, sm_tsub, sb>>>(
                    o, v, p_tsub, lr, L, ns, 0);
                ++top_launches;
                lr += L + 1;
            }
        }
        dv.end(2, eb, sb, top_launches);
        cudaEventRecord(ev_top, sb);
        cudaStreamWaitEvent(st, ev_top, 0);
    }
    // ---- stream A: bottom downsweep + leaf expansion + epilogue
    ev = dv.begin(st);
    {
        h2n::Range r("downsweep: leaf subtrees");
        if (wsw)
            launch_cta_sweep<T>(false, op, o, v, Lb, Lbot, st);
        else if (c64)
            launch_cta2_down<T>(o, v, Lb, Lbot, st);
        else
            k_down_sub<T, NVMAX><<<grid_bsub, kThreads, sm_bsub, st>>>(o, v, p_bsub, Lb, Lbot, nsub, 1);
    }
    dv.end(3, ev, st, 1);
    return cuda_status(cudaGetLastError());
}

// ---------------------------------------------------------------- passes of many vectors

// Shared-memory plan of the subtree kernels for one pass width: leaf subtrees of depth Lw
// (as deep as two CTAs per SM with at least two stages allow, else one CTA per SM), then
// launches of at most Ltop levels up to the root.
template <typename T, int NVMAX>
struct SweepPlan {
    int Lw = 0, Ltop = 1;
    h2s::Pipe bsub, tsub;
    size_t sm_bsub = 0, sm_tsub = 0;
    int64_t nsub = 1;
    unsigned grid_bsub = 1;
};

template <typename T, int NVMAX>
SweepPlan<T, NVMAX> make_sweep_plan(const h2_op &op, const h2_device &dv)
{
    using namespace h2s;
    SweepPlan<T, NVMAX> sp;
    const size_t es = sizeof(T);
    const int k = op.k, kx = dv.kx, mp = dv.mp;
    while (sp.Ltop < 5 && (size_t(4) << sp.Ltop) * kx * NVMAX * es <= 16 * 1024) ++sp.Ltop;
    const uint32_t tile = uint32_t(std::max({size_t(mp) * kx, size_t(k) * kx, size_t(k) * mp}) * es);
    const uint32_t xseg = uint32_t(2 * std::max(mp, kx) * NVMAX * es);
    size_t budget = 0;
    for (size_t b : {size_t(100) * 1024, size_t(200) * 1024}) {
        for (sp.Lw = dv.L; sp.Lw >= 0; --sp.Lw) {
            const Pipe p = make_pipe<T, NVMAX>(tile, xseg, 2 << sp.Lw, kx, false, b, 8);
            if (p.ns >= 2 && smem_bytes<T, NVMAX>(p, 2 << sp.Lw, kx, false) <= b) break;
        }
        budget = b;
        if (sp.Lw >= 0) break;
    }
    if (sp.Lw < 0) sp.Lw = 0;
    sp.bsub = make_pipe<T, NVMAX>(tile, xseg, 2 << sp.Lw, kx, false, budget, 8);
    sp.tsub = make_pipe<T, NVMAX>(tile, xseg, 2 << sp.Ltop, kx, false, 100 * 1024, 8);
    sp.sm_bsub = smem_bytes<T, NVMAX>(sp.bsub, 2 << sp.Lw, kx, false);
    sp.sm_tsub = smem_bytes<T, NVMAX>(sp.tsub, 2 << sp.Ltop, kx, false);
    sp.nsub = int64_t(1) << (op.q - sp.Lw);
    const int per_sm = sp.sm_bsub <= 100 * 1024 ? 2 : 1;
    sp.grid_bsub = unsigned(std::min<int64_t>(sp.nsub, int64_t(dv.num_sms) * per_sm));
    return sp;
}

template <typename T, int NVMAX>
unsigned top_grid(const SweepPlan<T, NVMAX> &sp, const h2_device &dv, int64_t ns)
{
    const int per_sm = sp.sm_tsub <= 100 * 1024 ? 2 : 1;
    return unsigned(std::min<int64_t>(ns, int64_t(dv.num_sms) * per_sm));
}

// Gather + the whole upsweep on one stream: leaf subtrees, then Ltop levels per launch.
template <typename T, int NVMAX>
int up_all(const h2_op &op, const h2_device &dv, const h2s::Op<T> &o, const h2s::Vec<T> &v,
           const SweepPlan<T, NVMAX> &sp, cudaStream_t st)
{
    using namespace h2s;
    int launches = 2;
    if (v.xr) {
        k_rows_in<T><<<dim3(unsigned((op.n + 31) / 32), unsigned((v.nv + 31) / 32)), dim3(32, 8), 0, st>>>(
            v.X, op.n, v.nv, v.xr, v.ldr);
        ++launches;
    }
    if (v.xr)
        k_gather_rows<T><<<unsigned(std::min<int64_t>(op.nleaves(), 65535)), 128, 0, st>>>(o, v);
    else
        k_gather<T><<<unsigned(std::min<int64_t>(op.nleaves(), 65535)), 128, 0, st>>>(o, v);
    k_up_sub<T, NVMAX><<<sp.grid_bsub, kThreads, sp.sm_bsub, st>>>(o, v, sp.bsub, op.q - sp.Lw, sp.Lw, sp.nsub, 1);
    for (int lin = op.q - sp.Lw; lin > 0;) {
        const int L = std::min(sp.Ltop, lin), lr = lin - L;
        const int64_t ns = int64_t(1) << lr;
        k_up_sub<T, NVMAX><<<top_grid(sp, dv, ns), kThreads, sp.sm_tsub, st>>>(o, v, sp.tsub, lr, L, ns, 0);
        ++launches;
        lin = lr;
    }
    return launches;
}

// The whole downsweep on one stream, ending in the leaf expansion and the epilogue.
template <typename T, int NVMAX>
int down_all(const h2_op &op, const h2_device &dv, const h2s::Op<T> &o, const h2s::Vec<T> &v,
             const SweepPlan<T, NVMAX> &sp, cudaStream_t st)
{
    using namespace h2s;
    int launches = 0;
    const int Lr0 = op.q - sp.Lw;
    for (int lr = 0; lr <= Lr0 - 1;) {
        const int L = std::min(sp.Ltop, Lr0 - 1 - lr);
        const int64_t ns = int64_t(1) << lr;
        k_down_sub<T, NVMAX><<<top_grid(sp, dv, ns), kThreads, sp.sm_tsub, st>>>(o, v, sp.tsub, lr, L, ns, 0);
        ++launches;
        lr += L + 1;
    }
    k_down_sub<T, NVMAX><<<sp.grid_bsub, kThreads, sp.sm_bsub, st>>>(o, v, sp.bsub, Lr0, sp.Lw, sp.nsub, 1);
    if (v.yr) {
        k_rows_out<T><<<dim3(unsigned((op.n + 31) / 32), unsigned((v.nv + 31) / 32)), dim3(32, 8), 0, st>>>(
            v.yr, v.ldr, v.Y, op.n, v.nv, v.alpha, v.beta);
        ++launches;
    }
    return launches + 1;
}

// One pass of 8 < nv <= NVMAX vectors on the wide kernels, all on one stream: upsweep,
// coupling and dense rows of every level (bottom, then top descriptor list), downsweep.
template <typename T, int NVMAX>
int launch_wide(const h2_op &op, h2_device &dv, const T *X, T *Y, int nv, double alpha, double beta,
                const Workspace &w, cudaStream_t st)
{
    using namespace h2s;
    const uint32_t es = sizeof(T);
    const int k = op.k, kx = dv.kx, mp = dv.mp;
    const Op<T> o = make_op<T>(op, dv);
    Vec<T> v{X, Y, nv, nv, T(alpha), T(beta), static_cast<T *>(w.xt), static_cast<T *>(w.yd),
             static_cast<T *>(w.xh), static_cast<T *>(w.yh), w.tickets, dv.err};
    v.xr = v.yr = static_cast<T *>(w.rows);
    v.ldr = round4(nv);
    const SweepPlan<T, NVMAX> sp = make_sweep_plan<T, NVMAX>(op, dv);
    const uint32_t tile_str = uint32_t(((std::max<size_t>(size_t(k) * kx, size_t(mp) * dv.max_leaf_rows) * es) + 15) /
                                       16 * 16);
    const uint32_t x_str = uint32_t(std::max(mp, kx) * NVMAX * es);
    // FP32: three CTAs per SM where two stages fit in a third of the shared memory (twelve
    // consumer warps hide the shared-memory latency of the register-blocked products); else
    // two CTAs per SM where three stages fit in half; else one CTA per SM
    Pipe p_str = make_pipe<T, NVMAX>(tile_str, x_str, 0, kx, true, 72 * 1024, 12);
    int per_sm = 3;
    if (sizeof(T) != 4 || p_str.ns < 2) {
        p_str = make_pipe<T, NVMAX>(tile_str, x_str, 0, kx, true, 110 * 1024, 12);
        per_sm = 2;
    }
    if (p_str.ns < 3 && per_sm == 2) {
        p_str = make_pipe<T, NVMAX>(tile_str, x_str, 0, kx, true, 200 * 1024, 12);
        per_sm = 1;
    }
    const size_t sm_str = smem_bytes<T, NVMAX>(p_str, 0, kx, true);
    const unsigned g_bot = unsigned(std::max<int64_t>(1, std::min<int64_t>(int64_t(dv.num_sms) * per_sm, dv.n_chunks_bottom)));
    const unsigned g_top = unsigned(std::max<int64_t>(1, std::min<int64_t>(int64_t(dv.num_sms) * per_sm, dv.n_chunks_top)));
    set_kernel_attributes<T, NVMAX>();

    cudaEvent_t ev = dv.begin(st);
    const int lu = up_all(op, dv, o, v, sp, st);
    dv.end(0, ev, st, lu);
    ev = dv.begin(st);
    int ls = 0;
    if (dv.n_chunks_bottom > 0) {
        k_stream<T, NVMAX><<<g_bot, kThreads, sm_str, st>>>(o, v, p_str, dv.desc_bottom, dv.chunks_bottom,
                                                            dv.n_chunks_bottom, 0);
        ++ls;
    }
    if (dv.n_chunks_dense > 0) {  // dense rows in a list of their own (small coupling tiles)
        const unsigned g_dns =
            unsigned(std::max<int64_t>(1, std::min<int64_t>(int64_t(dv.num_sms) * per_sm, dv.n_chunks_dense)));
        k_stream<T, NVMAX><<<g_dns, kThreads, sm_str, st>>>(o, v, p_str, dv.desc_bottom, dv.chunks_dense,
                                                            dv.n_chunks_dense, 2);
        ++ls;
    }
    if (dv.n_chunks_top > 0) {
        k_stream<T, NVMAX><<<g_top, kThreads, sm_str, st>>>(o, v, p_str, dv.desc_top, dv.chunks_top,
                                                         dv.n_chunks_top, 1);
        ++ls;
    }
    dv.end(1, ev, st, ls);
    ev = dv.begin(st);
    const int ld = down_all(op, dv, o, v, sp, st);
    dv.end(3, ev, st, ld);
    return cuda_status(cudaGetLastError());
}

// Tensor-core stream of one pass (H2_BF16X2): the coupling and dense rows of every level,
// reading the split-BF16 vector tiles that the gather and the upsweep wrote; NP = vectors
// padded to a multiple of 16.
template <int NP>
int launch_tc_stream(const h2_op &op, h2_device &dv, const Workspace &w, int npass, cudaStream_t st)
{
    using namespace h2s;
    static bool attr_done = false;
    if (!attr_done) {
        cudaFuncSetAttribute(k_stream_tc<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemBudget);
        cudaFuncSetAttribute(k_stream_tc<NP>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        attr_done = true;
    }
    int ns = 8;
    while (ns > 2 && tc_smem_bytes(NP, ns) > kTcSmemBudget) --ns;
    TcArgs a;
    a.vals = dv.vals;
    a.desc = dv.desc_bottom;
    a.chunks = dv.chunks_bottom;
    a.nchunks = dv.n_chunks_bottom;
    a.xb = w.xb;
    a.xtb = w.xtb;
    a.yh = static_cast<float *>(w.yh);
    a.yd = static_cast<float *>(w.yd);
    a.nv = npass;
    a.kx = dv.kx;
    a.mp = dv.mp;
    a.ticket = w.tickets + 2;
    a.err = dv.err;
    a.ns = ns;
    if (dv.n_chunks_bottom > 0)
        k_stream_tc<NP><<<dv.grid_bottom, kTcThreads, tc_smem_bytes(NP, ns), st>>>(a);
    return cuda_status(cudaGetLastError());
}

// Tensor-core product (H2_BF16X2), per pass of up to kWidePass vectors: FP32 upsweep on the
// wide subtree kernels (which also write the split-BF16 vector tiles, NVMAX = the padded
// pass width), the coupling and dense rows of every level on the tensor-core stream, FP32
// downsweep with the leaf expansion and the epilogue.
template <int NVMAX>
int launch_tc_pass(const h2_op &op, h2_device &dv, const float *X, float *Y, int npass, double alpha, double beta,
                   const Workspace &w, cudaStream_t st)
{
    using namespace h2s;
    using T = float;
    static_assert(NVMAX % 16 == 0, "tensor-core passes are padded to 16 vectors");
    const Op<T> o = make_op<T>(op, dv);
    Vec<T> v{X, Y, npass, npass, T(alpha), T(beta), static_cast<T *>(w.xt), static_cast<T *>(w.yd),
             static_cast<T *>(w.xh), static_cast<T *>(w.yh), w.tickets, dv.err};
    v.xb = w.xb;
    v.xtb = w.xtb;
    v.np = NVMAX;
    v.xr = v.yr = static_cast<T *>(w.rows);
    v.ldr = round4(npass);
    const SweepPlan<T, NVMAX> sp = make_sweep_plan<T, NVMAX>(op, dv);
    set_kernel_attributes<T, NVMAX>();
    cudaEvent_t ev = dv.begin(st);
    const int lu = up_all(op, dv, o, v, sp, st);
    dv.end(0, ev, st, lu);
    ev = dv.begin(st);
    const int rc = launch_tc_stream<NVMAX>(op, dv, w, npass, st);
    dv.end(1, ev, st, 1);
    if (rc != H2_OK) return rc;
    ev = dv.begin(st);
    const int ld = down_all(op, dv, o, v, sp, st);
    dv.end(3, ev, st, ld);
    return cuda_status(cudaGetLastError());
}

int launch_tc(const h2_op &op, h2_device &dv, const float *X, float *Y, int nv, double alpha, double beta,
              const Workspace &w, cudaStream_t st)
{
    for (int v0 = 0; v0 < nv; v0 += kWidePass) {
        const int c = std::min(kWidePass, nv - v0);
        const size_t o = size_t(v0) * op.n;
        const int rc = c <= 16 ? launch_tc_pass<16>(op, dv, X + o, Y + o, c, alpha, beta, w, st)
                               : launch_tc_pass<32>(op, dv, X + o, Y + o, c, alpha, beta, w, st);
        if (rc != H2_OK) return rc;
    }
    return H2_OK;
}

// Tensor-core stream over one descriptor list of the FP32 operator (3xTF32): NP = vectors
// padded to 16 or 32.
template <int NP>
int launch_tf32_stream(h2_device &dv, const Workspace &w, int npass, const h2s::StreamDesc *desc,
                       const int64_t *chunks, int64_t nchunks, int *ticket, cudaStream_t st)
{
    using namespace h2s;
    static bool attr_done = false;
    if (!attr_done) {
        cudaFuncSetAttribute(k_stream_tf32<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTfSmemBudget);
        cudaFuncSetAttribute(k_stream_tf32<NP>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        attr_done = true;
    }
    if (nchunks <= 0) return H2_OK;
    int ns = 16;
    while (ns > 2 && tf_smem_bytes(NP, ns) > kTfSmemBudget) --ns;
    TfArgs a;
    a.vals = dv.vals;
    a.desc = desc;
    a.chunks = chunks;
    a.nchunks = nchunks;
    a.xh = static_cast<const float *>(w.xh);
    a.xt = static_cast<const float *>(w.xt);
    a.yh = static_cast<float *>(w.yh);
    a.yd = static_cast<float *>(w.yd);
    a.nv = npass;
    a.kx = dv.kx;
    a.mp = dv.mp;
    a.ticket = ticket;
    a.err = dv.err;
    a.ns = ns;
    const unsigned grid = unsigned(std::max<int64_t>(1, std::min<int64_t>(dv.num_sms, nchunks)));
    k_stream_tf32<NP><<<grid, kTfThreads, tf_smem_bytes(NP, ns), st>>>(a);
    return cuda_status(cudaGetLastError());
}

// FP32 pass of 8 < nv <= NVMAX vectors with the block rows on the tensor cores (3xTF32): FP32
// upsweep on the wide subtree kernels, the coupling and dense rows of every level (bottom,
// then top descriptor list) on k_stream_tf32 (which splits blocks and vectors on chip), FP32
// downsweep with the leaf expansion and the epilogue; one stream.
template <int NVMAX>
int launch_tf32_pass(const h2_op &op, h2_device &dv, const float *X, float *Y, int npass, double alpha, double beta,
                     const Workspace &w, cudaStream_t st)
{
    using namespace h2s;
    using T = float;
    static_assert(NVMAX % 16 == 0, "tensor-core passes are padded to 16 vectors");
    const Op<T> o = make_op<T>(op, dv);
    Vec<T> v{X, Y, npass, npass, T(alpha), T(beta), static_cast<T *>(w.xt), static_cast<T *>(w.yd),
             static_cast<T *>(w.xh), static_cast<T *>(w.yh), w.tickets, dv.err};
    v.xr = v.yr = static_cast<T *>(w.rows);
    v.ldr = round4(npass);
    const SweepPlan<T, NVMAX> sp = make_sweep_plan<T, NVMAX>(op, dv);
    set_kernel_attributes<T, NVMAX>();
    cudaEvent_t ev = dv.begin(st);
    const int lu = up_all(op, dv, o, v, sp, st);
    dv.end(0, ev, st, lu);
    ev = dv.begin(st);
    int rc = launch_tf32_stream<NVMAX>(dv, w, npass, dv.desc_bottom, dv.chunks_bottom, dv.n_chunks_bottom,
                                       w.tickets + 0, st);
    if (rc == H2_OK && dv.n_chunks_dense > 0)
        rc = launch_tf32_stream<NVMAX>(dv, w, npass, dv.desc_bottom, dv.chunks_dense, dv.n_chunks_dense,
                                       w.tickets + 2, st);
    if (rc == H2_OK)
        rc = launch_tf32_stream<NVMAX>(dv, w, npass, dv.desc_top, dv.chunks_top, dv.n_chunks_top, w.tickets + 1, st);
    dv.end(1, ev, st, int(dv.n_chunks_bottom > 0) + int(dv.n_chunks_top > 0) + int(dv.n_chunks_dense > 0));
    if (rc != H2_OK) return rc;
    ev = dv.begin(st);
    const int ld = down_all(op, dv, o, v, sp, st);
    dv.end(3, ev, st, ld);
    return cuda_status(cudaGetLastError());
}

template <typename T>
int launch_product(const h2_op &op, h2_device &dv, const T *X, T *Y, int nv, double alpha, double beta,
                   const Workspace &w, cudaStream_t st, const h2_exec &ex)
{
    const int vp = pass_vectors(dv, nv);
    for (int v0 = 0; v0 < nv; v0 += vp) {
        const int c = std::min(vp, nv - v0);
        const size_t o = size_t(v0) * op.n;
        if constexpr (sizeof(T) == 4) {
            if (tf32_pass(dv, c)) {
                const int rc = c <= 16 ? launch_tf32_pass<16>(op, dv, X + o, Y + o, c, alpha, beta, w, st)
                                       : launch_tf32_pass<32>(op, dv, X + o, Y + o, c, alpha, beta, w, st);
                if (rc != H2_OK) return rc;
                continue;
            }
        }
        const int rc = c == 1       ? launch_chunk<T, 1>(op, dv, X + o, Y + o, c, alpha, beta, w, st, ex)
                     : c <= kChunk  ? launch_chunk<T, kChunk>(op, dv, X + o, Y + o, c, alpha, beta, w, st, ex)
                     : c <= 8       ? launch_wide<T, 8>(op, dv, X + o, Y + o, c, alpha, beta, w, st)
                     : c <= 16      ? launch_wide<T, 16>(op, dv, X + o, Y + o, c, alpha, beta, w, st)
                                    : launch_wide<T, 32>(op, dv, X + o, Y + o, c, alpha, beta, w, st);
        if (rc != H2_OK) return rc;
    }
    return H2_OK;
}

template <typename T>
int generate_blocks(const h2_op &op, h2_device &dv, const int32_t *d_cpl_row, const int32_t *d_dns_row,
                    const int32_t *d_dns_col, const int64_t *d_dns_off, const int32_t *d_cpl_col,
                    const double *d_cheb, const double *d_pts_tree, size_t d_region, cudaStream_t st,
                    int64_t ncpl, int64_t ndns)
{
    h2k::KernelFn f{int(op.ker.kind), op.ker.a, op.ker.b, op.ker.deg};
    if (ncpl > 0)
        h2k::gen_coupling<T><<<unsigned(std::min<int64_t>(ncpl, 1 << 20)), 256, 0, st>>>(
            reinterpret_cast<T *>(dv.vals), d_cpl_row, d_cpl_col, ncpl, d_cheb, op.dim, op.p, op.k, dv.kx, f);
    if (ndns > 0)
        h2k::gen_dense<T><<<unsigned(std::min<int64_t>(ndns, 1 << 20)), 256, 0, st>>>(
            reinterpret_cast<T *>(dv.vals + d_region), d_dns_off, d_dns_row, d_dns_col, ndns, dv.leaf_lo,
            d_pts_tree, op.dim, f);
    return cuda_status(cudaGetLastError());
}

// Coordinates of the matrix-free precision: every cluster's Chebyshev points and every
// leaf's points as float4.
int generate_mf_points(const h2_op &op, h2_device &dv, const double *d_cheb, const double *d_pts, cudaStream_t st)
{
    const int64_t nodes = op.nnodes + 1;
    h2s::k_mf_node_points<<<unsigned(std::min<int64_t>((nodes * op.k + 255) / 256, 65535)), 256, 0, st>>>(
        d_cheb, nodes, op.dim, op.p, op.k, const_cast<float4 *>(dv.mfa.node_pts));
    h2s::k_mf_leaf_points<<<unsigned(std::min<int64_t>((op.nleaves() * dv.mp + 255) / 256, 65535)), 256, 0, st>>>(
        d_pts, dv.leaf_lo, op.nleaves(), op.dim, dv.mp, const_cast<float4 *>(dv.mfa.leaf_pts));
    return cuda_status(cudaGetLastError());
}

int generate_tc_blocks(const h2_op &op, h2_device &dv, const int32_t *d_cpl_row, const int32_t *d_dns_row,
                       const int32_t *d_dns_col, const int32_t *d_cpl_col, const double *d_cheb, const double *d_pts_tree,
                       size_t d_region, cudaStream_t st)
{
    h2k::KernelFn f{int(op.ker.kind), op.ker.a, op.ker.b, op.ker.deg};
    const int64_t ncpl = int64_t(op.cpl_col.size()), ndns = int64_t(op.dns_col.size());
    if (ncpl > 0)
        h2k::gen_coupling_tc<<<unsigned(std::min<int64_t>(ncpl, 1 << 20)), 256, 0, st>>>(
            dv.vals, d_cpl_row, d_cpl_col, ncpl, d_cheb, op.dim, op.p, op.k, f);
    if (ndns > 0)
        h2k::gen_dense_tc<<<unsigned(std::min<int64_t>(ndns, 1 << 20)), 256, 0, st>>>(
            dv.vals + d_region, d_dns_row, d_dns_col, ndns, dv.leaf_lo, d_pts_tree, op.dim, f);
    return cuda_status(cudaGetLastError());
}

// Group a descriptor list (whole block rows, in order) into scheduling chunks of about
// `target` bytes and at most kChunkDesc descriptors: record = (first << 16) | count.
// Returns false if a single row has more than kChunkDesc blocks.
bool make_chunks(const std::vector<h2s::StreamDesc> &d, const std::vector<uint64_t> &bytes, uint64_t target,
                 std::vector<int64_t> &out)
{
    out.clear();
    size_t first = 0, row_first = 0;
    uint64_t acc = 0;
    for (size_t i = 0; i < d.size(); ++i) {
        acc += bytes[i];
        if (!(d[i].flags & h2s::kLast)) continue;
        const size_t row_end = i + 1;
        if (row_end - row_first > size_t(h2s::kChunkDesc)) return false;
        if (row_end - first > size_t(h2s::kChunkDesc)) {  // close the chunk before this row
            out.push_back(int64_t(first) << 16 | int64_t(row_first - first));
            first = row_first;
            acc = 0;
            for (size_t j = row_first; j < row_end; ++j) acc += bytes[j];
        }
        if (acc >= target) {
            out.push_back(int64_t(first) << 16 | int64_t(row_end - first));
            first = row_end;
            acc = 0;
        }
        row_first = row_end;
    }
    if (first < d.size()) out.push_back(int64_t(first) << 16 | int64_t(d.size() - first));
    return true;
}

// ---------------------------------------------------------------- batched products

constexpr int kBatchGroups = 64;  // most merged streams of one batch (width x tile-size classes)

// Width class of a pass of nv vectors (the accumulator the kernels instantiate).
int width_class(int nv) { return nv == 1 ? 1 : nv <= kChunk ? kChunk : nv <= 8 ? 8 : nv <= 16 ? 16 : 32; }

// Launch configuration of one merged stream: CTAs per SM, pipeline stages, chunk target.
struct StreamCfg {
    int per_sm = 1;
    int ns = 0;
    uint64_t chunk_target = 512 * 1024;
};

// Autotuner cache: one line per key, "key per_sm ns chunk_target ms", in the file named by
// H2_TUNE_CACHE or else beside libh2.so.
std::string tune_cache_path()
{
    if (const char *e = std::getenv("H2_TUNE_CACHE")) return e;
    Dl_info info;
    if (dladdr(reinterpret_cast<void *>(&tune_cache_path), &info) && info.dli_fname) {
        std::string f = info.dli_fname;
        const size_t slash = f.rfind('/');
        return (slash == std::string::npos ? std::string(".") : f.substr(0, slash)) + "/h2_autotune.txt";
    }
    return "h2_autotune.txt";
}

std::mutex &tune_mutex()
{
    static std::mutex m;
    return m;
}

bool tune_lookup(const std::string &key, StreamCfg *cfg)
{
    std::lock_guard<std::mutex> lk(tune_mutex());
    std::ifstream in(tune_cache_path());
    std::string line;
    bool found = false;
    while (std::getline(in, line)) {
        std::istringstream ls(line);
        std::string k;
        StreamCfg c;
        double ms = 0;
        if (ls >> k >> c.per_sm >> c.ns >> c.chunk_target >> ms && k == key) {
            *cfg = c;  // the last entry for a key wins
            found = true;
        }
    }
    return found;
}

void tune_store(const std::string &key, const StreamCfg &c, double ms)
{
    std::lock_guard<std::mutex> lk(tune_mutex());
    std::ofstream out(tune_cache_path(), std::ios::app);
    if (out) out << key << ' ' << c.per_sm << ' ' << c.ns << ' ' << c.chunk_target << ' ' << ms << '\n';
}

}  // namespace

// A batch: every member's workspace, the merged descriptor list of each width class and
// the captured graph of the whole batched product.
struct h2_batch {
    struct Member {
        h2_handle op;
        const void *X;
        void *Y;
        int nv;
        Workspace w;
        bool merged = false;  // its sweeps run inside the merged launches of its width
    };
    struct Group {
        int width = 0;
        uint64_t tile_class = 0;             // power of two >= every tile of the group
        std::vector<int> members;            // indices into members
        std::vector<h2s::StreamDesc> desc;   // merged, host
        std::vector<uint64_t> bytes;         // streamed bytes per descriptor
        h2s::StreamDesc *d_desc = nullptr;
        int64_t *d_chunks = nullptr;
        size_t chunk_cap = 0;                // capacity of d_chunks (records)
        int64_t nchunks = 0;
        void *d_ops = nullptr;               // BatchOp<T>[members]
        uint32_t tile_bytes = 0, x_bytes = 0;
        StreamCfg cfg;
        bool tuned = false;
    };
    // merged sweeps: per accumulator width, one launch per sweep step over all members of
    // that width (a task table per launch, all tables of a width in one device allocation)
    struct SweepLaunch {
        int kind = 0;           // kRowsIn, kGather, kUp, kDown, kRowsOut
        size_t task_off = 0;    // first task of this launch in the width's table
        int ntasks = 0;
        int64_t total = 0;      // work items: 32-point tiles, leaves or subtrees
        h2s::Pipe pp{1, 0, 0};  // subtree steps: stages sized for the largest tiles
        int sub_kx = 0;         // subtree steps: the largest subtree buffer (slots x kx)
        int rows = 0;           // gather: from the row-major staging copy
        size_t smem = 0;
        unsigned grid = 1;
    };
    struct SweepClass {
        int width = 0;
        void *d_tasks = nullptr;
        std::vector<SweepLaunch> up, down;
    };
    int device = 0, num_sms = 0;
    size_t esize = 4;
    double alpha = 1, beta = 0;
    std::vector<Member> members;
    std::vector<Group> groups;
    std::vector<SweepClass> sweeps;
    void *ws_mem = nullptr;
    int *d_flags = nullptr;                  // [0, kBatchGroups) tickets per group, [kBatchGroups] error flag
    std::vector<cudaStream_t> branches;
    std::vector<cudaEvent_t> ev_branch;
    cudaEvent_t ev_fork = nullptr, ev_mid = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

template <typename T, int NV>
void batch_member_up(h2_batch::Member &m, double alpha, double beta, cudaStream_t st, bool up)
{
    using namespace h2s;
    const h2_op &op = *m.op;
    h2_device &dv = *op.dev;
    const Op<T> o = make_op<T>(op, dv);
    Vec<T> v{static_cast<const T *>(m.X), static_cast<T *>(m.Y), m.nv, m.nv, T(alpha), T(beta), static_cast<T *>(m.w.xt),
             static_cast<T *>(m.w.yd), static_cast<T *>(m.w.xh), static_cast<T *>(m.w.yh), m.w.tickets, dv.err};
    if (NV >= kWideMin) {
        v.xr = v.yr = static_cast<T *>(m.w.rows);
        v.ldr = round4(m.nv);
    }
    if (up)
        up_all(op, dv, o, v, make_sweep_plan<T, NV>(op, dv), st);
    else
        down_all(op, dv, o, v, make_sweep_plan<T, NV>(op, dv), st);
}

// One member's upsweep (gather included) or downsweep (alpha y + beta Y included).
template <typename T>
void batch_member_sweep(const h2_batch &b, h2_batch::Member &m, cudaStream_t st, bool up)
{
    switch (width_class(m.nv)) {
    case 1: set_kernel_attributes<T, 1>(); return batch_member_up<T, 1>(m, b.alpha, b.beta, st, up);
    case kChunk: set_kernel_attributes<T, kChunk>(); return batch_member_up<T, kChunk>(m, b.alpha, b.beta, st, up);
    case 8: set_kernel_attributes<T, 8>(); return batch_member_up<T, 8>(m, b.alpha, b.beta, st, up);
    case 16: set_kernel_attributes<T, 16>(); return batch_member_up<T, 16>(m, b.alpha, b.beta, st, up);
    default: set_kernel_attributes<T, 32>(); return batch_member_up<T, 32>(m, b.alpha, b.beta, st, up);
    }
}

template <typename T, int NV>
int batch_group_stream(h2_batch &b, h2_batch::Group &g, int gi, cudaStream_t st)
{
    using namespace h2s;
    if (g.nchunks == 0) return H2_OK;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_stream_batch<T, NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(k_stream_batch<T, NV>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        attr = true;
    }
    const Pipe p{g.cfg.ns, g.tile_bytes, g.x_bytes};
    const size_t smem = smem_bytes<T, NV>(p, 0, 0, true);
    const unsigned grid = unsigned(std::max<int64_t>(1, std::min<int64_t>(int64_t(b.num_sms) * g.cfg.per_sm, g.nchunks)));
    k_stream_batch<T, NV><<<grid, kThreads, smem, st>>>(static_cast<const BatchOp<T> *>(g.d_ops), p, g.d_desc,
                                                        g.d_chunks, g.nchunks, b.d_flags + gi, b.d_flags + kBatchGroups);
    return cuda_status(cudaGetLastError());
}

template <typename T>
int batch_group_stream_any(h2_batch &b, h2_batch::Group &g, int gi, cudaStream_t st)
{
    switch (g.width) {
    case 1: return batch_group_stream<T, 1>(b, g, gi, st);
    case kChunk: return batch_group_stream<T, kChunk>(b, g, gi, st);
    case 8: return batch_group_stream<T, 8>(b, g, gi, st);
    case 16: return batch_group_stream<T, 16>(b, g, gi, st);
    default: return batch_group_stream<T, 32>(b, g, gi, st);
    }
}

template <typename T>
size_t batch_group_smem(const h2_batch::Group &g, int ns)
{
    const h2s::Pipe p{ns, g.tile_bytes, g.x_bytes};
    switch (g.width) {
    case 1: return h2s::smem_bytes<T, 1>(p, 0, 0, true);
    case kChunk: return h2s::smem_bytes<T, kChunk>(p, 0, 0, true);
    case 8: return h2s::smem_bytes<T, 8>(p, 0, 0, true);
    case 16: return h2s::smem_bytes<T, 16>(p, 0, 0, true);
    default: return h2s::smem_bytes<T, 32>(p, 0, 0, true);
    }
}

// Stages for per_sm CTAs per SM (budget 200 KB / 110 KB / 72 KB), at most 24 (small tiles
// get deep rings); 0 if fewer than 2 fit.
template <typename T>
int batch_stages(const h2_batch::Group &g, int per_sm)
{
    const size_t budget = per_sm == 1 ? 200 * 1024 : per_sm == 2 ? 110 * 1024 : 72 * 1024;
    for (int ns = 24; ns >= 2; --ns)
        if (batch_group_smem<T>(g, ns) <= budget) return ns;
    return 0;
}

int batch_set_chunks(h2_batch::Group &g, uint64_t target)
{
    std::vector<int64_t> ch;
    if (!make_chunks(g.desc, g.bytes, target, ch)) return H2_EINVAL;
    if (ch.size() > g.chunk_cap) return H2_EINVAL;
    g.nchunks = int64_t(ch.size());
    if (!ch.empty()) {
        const int rc = cuda_status(cudaMemcpy(g.d_chunks, ch.data(), ch.size() * 8, cudaMemcpyHostToDevice));
        if (rc != H2_OK) return rc;
    }
    g.cfg.chunk_target = target;
    return H2_OK;
}

constexpr int kRowsIn = 0, kGather = 1, kUp = 2, kDown = 3, kRowsOut = 4;  // merged sweep steps

// The merged sweeps of the members `mem` (all of accumulator width W): one launch per step --
// [row-major staging], gather, bottom subtrees and each run of upper levels (up), the upper
// levels, bottom subtrees with the leaf epilogue, [staging back] (down) -- each over a task
// table with one task per member, the member with the most work items first. The steps are
// the ones up_all / down_all launch for one operator, in the same order. Returns false when
// a subtree step cannot be staged in 200 KB (the width then keeps per-member sweeps).
template <typename T, int W>
bool batch_build_sweeps(h2_batch &b, const std::vector<int> &mem, h2_batch::SweepClass &sc)
{
    using namespace h2s;
    const size_t es = sizeof(T);
    struct Info {
        SweepTask<T> base;
        SweepPlan<T, W> sp;
        int q;
        uint32_t tile, xseg;
        std::vector<std::array<int, 2>> up_top, down_top;  // (Lr, L) of each run of upper levels
    };
    std::vector<Info> inf;
    for (int i : mem) {
        h2_batch::Member &m = b.members[size_t(i)];
        const h2_op &op = *m.op;
        h2_device &dv = *op.dev;
        Info f;
        f.base.op = make_op<T>(op, dv);
        f.base.vec = Vec<T>{static_cast<const T *>(m.X), static_cast<T *>(m.Y), m.nv, m.nv, T(b.alpha), T(b.beta),
                            static_cast<T *>(m.w.xt), static_cast<T *>(m.w.yd), static_cast<T *>(m.w.xh),
                            static_cast<T *>(m.w.yh), m.w.tickets, dv.err};
        if (W >= kWideMin) {
            f.base.vec.xr = f.base.vec.yr = static_cast<T *>(m.w.rows);
            f.base.vec.ldr = round4(m.nv);
        }
        f.sp = make_sweep_plan<T, W>(op, dv);
        f.q = op.q;
        const int k = op.k, kx = dv.kx, mp = dv.mp;
        f.tile = uint32_t(std::max({size_t(mp) * kx, size_t(k) * kx, size_t(k) * mp}) * es);
        f.xseg = uint32_t(2 * std::max(mp, kx) * W * es);
        for (int lin = op.q - f.sp.Lw; lin > 0;) {
            const int L = std::min(f.sp.Ltop, lin), lr = lin - L;
            f.up_top.push_back({lr, L});
            lin = lr;
        }
        const int Lr0 = op.q - f.sp.Lw;
        for (int lr = 0; lr <= Lr0 - 1;) {
            const int L = std::min(f.sp.Ltop, Lr0 - 1 - lr);
            f.down_top.push_back({lr, L});
            lr += L + 1;
        }
        inf.push_back(f);
    }
    std::vector<SweepTask<T>> all;
    bool ok = true;
    auto push = [&](std::vector<h2_batch::SweepLaunch> &list, int kind, std::vector<SweepTask<T>> tk,
                    uint32_t tile, uint32_t xseg, int sub_kx, int rows) {
        if (!ok || tk.empty()) return;
        std::stable_sort(tk.begin(), tk.end(), [](const SweepTask<T> &x, const SweepTask<T> &y) { return x.nsub > y.nsub; });
        int64_t first = 0;
        for (auto &t : tk) {
            t.first = first;
            first += t.nsub;
        }
        h2_batch::SweepLaunch L;
        L.kind = kind;
        L.task_off = all.size();
        L.ntasks = int(tk.size());
        L.total = first;
        L.rows = rows;
        L.sub_kx = sub_kx;
        if (kind == kUp || kind == kDown) {
            int per_sm = 2;
            L.pp = make_pipe<T, W>(tile, xseg, 1, sub_kx, false, 100 * 1024, 8);
            L.smem = smem_bytes<T, W>(L.pp, 1, sub_kx, false);
            if (L.pp.ns < 2 || L.smem > 100 * 1024) {
                per_sm = 1;
                L.pp = make_pipe<T, W>(tile, xseg, 1, sub_kx, false, 200 * 1024, 8);
                L.smem = smem_bytes<T, W>(L.pp, 1, sub_kx, false);
            }
            if (L.pp.ns < 2 || L.smem > 200 * 1024) {
                ok = false;
                return;
            }
            L.grid = unsigned(std::max<int64_t>(1, std::min<int64_t>(first, int64_t(b.num_sms) * per_sm)));
        } else {
            L.grid = unsigned(std::max<int64_t>(1, std::min<int64_t>(first, 65535)));
        }
        all.insert(all.end(), tk.begin(), tk.end());
        list.push_back(L);
    };
    auto task = [](const Info &f, int Lr, int L, int flag, int64_t nsub) {
        SweepTask<T> t = f.base;
        t.Lr = Lr;
        t.L = L;
        t.flag = flag;
        t.nsub = nsub;
        return t;
    };
    // a subtree step over the given (member, Lr, L, flag) tasks: stages for the largest tiles
    auto subtree_step = [&](std::vector<h2_batch::SweepLaunch> &list, int kind, const std::vector<SweepTask<T>> &tk,
                            const std::vector<const Info *> &who) {
        uint32_t tile = 0, xseg = 0;
        int sub_kx = 0;
        for (size_t j = 0; j < tk.size(); ++j) {
            tile = std::max(tile, who[j]->tile);
            xseg = std::max(xseg, who[j]->xseg);
            sub_kx = std::max(sub_kx, (2 << tk[j].L) * tk[j].op.kx);
        }
        push(list, kind, tk, tile, xseg, sub_kx, 0);
    };
    std::vector<SweepTask<T>> tk;
    std::vector<const Info *> who;
    // ---- up
    if (W >= kWideMin) {
        for (auto &f : inf) tk.push_back(task(f, 0, 0, 0, (f.base.op.n + 31) / 32));
        push(sc.up, kRowsIn, tk, 0, 0, 0, 0);
        tk.clear();
    }
    for (auto &f : inf) tk.push_back(task(f, 0, 0, 0, f.base.op.nleaves));
    push(sc.up, kGather, tk, 0, 0, 0, W >= kWideMin ? 1 : 0);
    tk.clear();
    for (auto &f : inf) {
        tk.push_back(task(f, f.q - f.sp.Lw, f.sp.Lw, 1, f.sp.nsub));
        who.push_back(&f);
    }
    subtree_step(sc.up, kUp, tk, who);
    size_t runs = 0;
    for (auto &f : inf) runs = std::max(runs, f.up_top.size());
    for (size_t j = 0; j < runs; ++j) {
        tk.clear();
        who.clear();
        for (auto &f : inf)
            if (j < f.up_top.size()) {
                tk.push_back(task(f, f.up_top[j][0], f.up_top[j][1], 0, int64_t(1) << f.up_top[j][0]));
                who.push_back(&f);
            }
        subtree_step(sc.up, kUp, tk, who);
    }
    // ---- down
    runs = 0;
    for (auto &f : inf) runs = std::max(runs, f.down_top.size());
    for (size_t j = 0; j < runs; ++j) {
        tk.clear();
        who.clear();
        for (auto &f : inf)
            if (j < f.down_top.size()) {
                tk.push_back(task(f, f.down_top[j][0], f.down_top[j][1], 0, int64_t(1) << f.down_top[j][0]));
                who.push_back(&f);
            }
        subtree_step(sc.down, kDown, tk, who);
    }
    tk.clear();
    who.clear();
    for (auto &f : inf) {
        tk.push_back(task(f, f.q - f.sp.Lw, f.sp.Lw, 1, f.sp.nsub));
        who.push_back(&f);
    }
    subtree_step(sc.down, kDown, tk, who);
    if (W >= kWideMin) {
        tk.clear();
        for (auto &f : inf) tk.push_back(task(f, 0, 0, 0, (f.base.op.n + 31) / 32));
        push(sc.down, kRowsOut, tk, 0, 0, 0, 0);
    }
    if (!ok) {
        sc.up.clear();
        sc.down.clear();
        return false;
    }
    if (cudaMalloc(&sc.d_tasks, std::max<size_t>(1, all.size()) * sizeof(SweepTask<T>)) != cudaSuccess) {
        cudaGetLastError();
        sc.d_tasks = nullptr;
        sc.up.clear();
        sc.down.clear();
        return false;
    }
    if (cudaMemcpy(sc.d_tasks, all.data(), all.size() * sizeof(SweepTask<T>), cudaMemcpyHostToDevice) != cudaSuccess) {
        sc.up.clear();
        sc.down.clear();
        return false;
    }
    static bool attr = false;
    if (!attr) {
        for (const void *fn : {(const void *)k_up_batch<T, W>, (const void *)k_down_batch<T, W>}) {
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        }
        attr = true;
    }
    return true;
}

template <typename T, int W>
void batch_sweep_launch(const h2_batch::SweepClass &sc, const h2_batch::SweepLaunch &L, cudaStream_t st)
{
    using namespace h2s;
    const SweepTask<T> *t = static_cast<const SweepTask<T> *>(sc.d_tasks) + L.task_off;
    switch (L.kind) {
    case kRowsIn: k_rows_in_batch<T><<<L.grid, dim3(32, 8), 0, st>>>(t, L.ntasks, L.total); break;
    case kGather: k_gather_batch<T><<<L.grid, 128, 0, st>>>(t, L.ntasks, L.total, L.rows); break;
    case kUp: k_up_batch<T, W><<<L.grid, kThreads, L.smem, st>>>(t, L.ntasks, L.total, L.pp, L.sub_kx); break;
    case kDown: k_down_batch<T, W><<<L.grid, kThreads, L.smem, st>>>(t, L.ntasks, L.total, L.pp, L.sub_kx); break;
    default: k_rows_out_batch<T><<<L.grid, dim3(32, 8), 0, st>>>(t, L.ntasks, L.total); break;
    }
}

// One width's merged up- (up = true) or downsweep launches, in order, on one stream.
template <typename T>
void batch_sweeps_enqueue(const h2_batch::SweepClass &sc, bool up, cudaStream_t st)
{
    for (const auto &L : up ? sc.up : sc.down) {
        switch (sc.width) {
        case 1: batch_sweep_launch<T, 1>(sc, L, st); break;
        case kChunk: batch_sweep_launch<T, kChunk>(sc, L, st); break;
        case 8: batch_sweep_launch<T, 8>(sc, L, st); break;
        case 16: batch_sweep_launch<T, 16>(sc, L, st); break;
        default: batch_sweep_launch<T, 32>(sc, L, st); break;
        }
    }
}

// Builds the merged sweeps of every width present in the batch.
template <typename T>
int batch_build_all_sweeps(h2_batch &b)
{
    for (int w : {1, kChunk, 8, 16, 32}) {
        std::vector<int> mem;
        for (size_t i = 0; i < b.members.size(); ++i)
            if (width_class(b.members[i].nv) == w) mem.push_back(int(i));
        if (mem.empty()) continue;
        h2_batch::SweepClass sc;
        sc.width = w;
        bool built = false;
        switch (w) {
        case 1: built = batch_build_sweeps<T, 1>(b, mem, sc); break;
        case kChunk: built = batch_build_sweeps<T, kChunk>(b, mem, sc); break;
        case 8: built = batch_build_sweeps<T, 8>(b, mem, sc); break;
        case 16: built = batch_build_sweeps<T, 16>(b, mem, sc); break;
        default: built = batch_build_sweeps<T, 32>(b, mem, sc); break;
        }
        if (!built) {
            if (sc.d_tasks) cudaFree(sc.d_tasks);
            continue;  // this width keeps per-member sweeps
        }
        for (int i : mem) b.members[size_t(i)].merged = true;
        b.sweeps.push_back(sc);
    }
    return cuda_status(cudaGetLastError());
}

// The whole batched product on the capture stream, in three phases on the branch streams:
// upsweeps (each width's merged sweep launches on a branch of its own; members of a width
// without merged sweeps one by one on the other branches), the merged block streams (one per
// group, concurrently: they write disjoint rows, so one group's tail overlaps the others'
// work), downsweeps. Every phase forks all branches from the capture stream and joins them
// back. Without the downsweeps (with_down false) nothing of the members' Y is written.
template <typename T>
int batch_enqueue(h2_batch &b, cudaStream_t st, bool with_down = true)
{
    const size_t nb = b.branches.size();
    auto fork = [&](cudaEvent_t ev) {
        int rc = cuda_status(cudaEventRecord(ev, st));
        for (size_t j = 0; rc == H2_OK && j < nb; ++j) rc = cuda_status(cudaStreamWaitEvent(b.branches[j], ev, 0));
        return rc;
    };
    auto join = [&]() {
        int rc = H2_OK;
        for (size_t j = 0; rc == H2_OK && j < nb; ++j) {
            rc = cuda_status(cudaEventRecord(b.ev_branch[j], b.branches[j]));
            if (rc == H2_OK) rc = cuda_status(cudaStreamWaitEvent(st, b.ev_branch[j], 0));
        }
        return rc;
    };
    auto sweeps = [&](bool up) {
        const size_t nc = b.sweeps.size();
        for (size_t c = 0; c < nc; ++c) batch_sweeps_enqueue<T>(b.sweeps[c], up, b.branches[c % nb]);
        size_t k = 0;
        for (size_t i = 0; i < b.members.size(); ++i)
            if (!b.members[i].merged) batch_member_sweep<T>(b, b.members[i], b.branches[(nc + k++) % nb], up);
        return cuda_status(cudaGetLastError());
    };
    int rc = fork(b.ev_fork);
    if (rc == H2_OK) rc = sweeps(true);
    if (rc == H2_OK) rc = join();
    if (rc == H2_OK) rc = cuda_status(cudaMemsetAsync(b.d_flags, 0, kBatchGroups * sizeof(int), st));
    if (rc == H2_OK) rc = fork(b.ev_mid);
    for (size_t gi = 0; rc == H2_OK && gi < b.groups.size(); ++gi)
        rc = batch_group_stream_any<T>(b, b.groups[gi], int(gi), b.branches[gi % nb]);
    if (rc == H2_OK) rc = join();
    if (rc == H2_OK && with_down) {
        rc = fork(b.ev_mid);
        if (rc == H2_OK) rc = sweeps(false);
        if (rc == H2_OK) rc = join();
    }
    if (rc == H2_OK) rc = cuda_status(cudaGetLastError());
    return rc;
}

// Time one merged stream configuration (median of three launches after one warm-up).
template <typename T>
double batch_time_group(h2_batch &b, size_t gi, cudaStream_t st)
{
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::vector<float> ms;
    for (int r = 0; r < 4; ++r) {
        cudaMemsetAsync(b.d_flags + gi, 0, sizeof(int), st);
        cudaEventRecord(e0, st);
        batch_group_stream_any<T>(b, b.groups[gi], int(gi), st);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float t = 0;
        cudaEventElapsedTime(&t, e0, e1);
        if (r > 0) ms.push_back(t);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::sort(ms.begin(), ms.end());
    return cudaGetLastError() == cudaSuccess ? ms[ms.size() / 2] : 1e30;
}

template <typename T>
std::string batch_tune_key(const h2_batch &b, const h2_batch::Group &g)
{
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, b.device);
    std::string name = prop.name;
    for (char &c : name)
        if (c == ' ') c = '_';
    uint64_t total = 0;
    for (uint64_t x : g.bytes) total += x;
    int lg = 0;
    while ((uint64_t(1) << (lg + 1)) <= total) ++lg;  // log2 of the streamed bytes
    std::ostringstream k;
    k << "stream_batch/" << (sizeof(T) == 8 ? "fp64" : "fp32") << "/w" << g.width << "/tile" << g.tile_bytes
      << "/x" << g.x_bytes << "/log2B" << lg << "/" << name;
    return k.str();
}

// Pick each group's (CTAs per SM, stages, chunk target): from the cache, else by timing
// the candidates (when allowed), else the default (two CTAs per SM where three stages fit).
template <typename T>
int batch_configure(h2_batch &b, bool autotune, cudaStream_t st)
{
    for (size_t gi = 0; gi < b.groups.size(); ++gi) {
        h2_batch::Group &g = b.groups[gi];
        const std::string key = batch_tune_key<T>(b, g);
        StreamCfg c;
        if (tune_lookup(key, &c) && c.ns >= 2 && batch_group_smem<T>(g, c.ns) <= 200 * 1024 &&
            batch_set_chunks(g, c.chunk_target) == H2_OK) {
            g.cfg = c;
            g.tuned = true;
            continue;
        }
        g.cfg.per_sm = batch_stages<T>(g, 2) >= 3 ? 2 : 1;
        g.cfg.ns = batch_stages<T>(g, g.cfg.per_sm);
        int rc = batch_set_chunks(g, 512 * 1024);
        if (rc != H2_OK) return rc;
        if (!autotune || g.nchunks == 0) continue;
        StreamCfg best = g.cfg;
        double best_ms = 1e30;
        for (int per_sm : {1, 2, 3})
            for (uint64_t target : {uint64_t(128) << 10, uint64_t(512) << 10, uint64_t(2) << 20}) {
                const int ns = batch_stages<T>(g, per_sm);
                if (ns < 2) continue;
                g.cfg.per_sm = per_sm;
                g.cfg.ns = ns;
                if (batch_set_chunks(g, target) != H2_OK) continue;
                const double ms = batch_time_group<T>(b, gi, st);
                if (ms < best_ms) {
                    best_ms = ms;
                    best = g.cfg;
                }
            }
        g.cfg = best;
        rc = batch_set_chunks(g, best.chunk_target);
        if (rc != H2_OK) return rc;
        g.tuned = true;
        tune_store(key, best, best_ms);
    }
    return H2_OK;
}

template <typename T>
int batch_build_group_tables(h2_batch &b)
{
    using namespace h2s;
    for (h2_batch::Group &g : b.groups) {
        std::vector<BatchOp<T>> tab;
        for (int mi : g.members) {
            h2_batch::Member &m = b.members[size_t(mi)];
            const h2_device &dv = *m.op->dev;
            BatchOp<T> o;
            o.vals = dv.vals;
            o.xh = static_cast<const T *>(m.w.xh);
            o.xt = static_cast<const T *>(m.w.xt);
            o.yh = static_cast<T *>(m.w.yh);
            o.yd = static_cast<T *>(m.w.yd);
            o.kx = dv.kx;
            o.mp = dv.mp;
            o.vs = m.nv;
            o.nv = m.nv;
            tab.push_back(o);
        }
        int rc = cuda_status(cudaMalloc(&g.d_ops, std::max<size_t>(1, tab.size()) * sizeof(BatchOp<T>)));
        if (rc == H2_OK && !tab.empty())
            rc = cuda_status(cudaMemcpy(g.d_ops, tab.data(), tab.size() * sizeof(BatchOp<T>), cudaMemcpyHostToDevice));
        if (rc != H2_OK) return rc;
    }
    return H2_OK;
}

void batch_free(h2_batch *b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto &g : b->groups) {
        if (g.d_desc) cudaFree(g.d_desc);
        if (g.d_chunks) cudaFree(g.d_chunks);
        if (g.d_ops) cudaFree(g.d_ops);
    }
    for (auto &c : b->sweeps)
        if (c.d_tasks) cudaFree(c.d_tasks);
    for (cudaStream_t s : b->branches) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->ev_branch) cudaEventDestroy(e);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_mid) cudaEventDestroy(b->ev_mid);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->ws_mem) cudaFree(b->ws_mem);
    if (b->d_flags) cudaFree(b->d_flags);
    delete b;
}

}  // namespace

void h2_device_free(h2_op *op)
{
    if (!op || !op->dev) return;
    int prev = -1;
    cudaGetDevice(&prev);
    if (op->dev->device >= 0) cudaSetDevice(op->dev->device);
    if (op->dev->arena) cudaFree(op->dev->arena);
    delete op->dev;  // its destructor frees the stream workspaces and fork/join contexts
    op->dev = nullptr;
    if (prev >= 0) cudaSetDevice(prev);
}

// ---------------------------------------------------------------- internal entry points (h2_internal.h)

int h2_coupling_fp64(const h2_op &op, double *dS, void *cuda_stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int64_t ncpl = int64_t(op.cpl_col.size());
    if (ncpl == 0) return H2_OK;
    if (!op.S.empty()) {
        int rc = cuda_status(cudaMemcpyAsync(dS, op.S.data(), op.S.size() * 8, cudaMemcpyHostToDevice, st));
        return rc == H2_OK ? cuda_status(cudaStreamSynchronize(st)) : rc;
    }
    std::vector<int32_t> row(ncpl);
    for (int64_t t = 1; t <= op.nnodes; ++t)
        for (int64_t b = op.cpl_rowptr[t]; b < op.cpl_rowptr[t + 1]; ++b) row[b] = int32_t(t);
    char *tmp = nullptr;
    const size_t b_rows = align_up(size_t(ncpl) * 4), b_cheb = align_up(op.cheb.size() * 8);
    if (cudaMalloc(&tmp, 2 * b_rows + b_cheb) != cudaSuccess) {
        cudaGetLastError();
        return H2_ENOMEM;
    }
    int32_t *d_row = reinterpret_cast<int32_t *>(tmp), *d_col = reinterpret_cast<int32_t *>(tmp + b_rows);
    double *d_cheb = reinterpret_cast<double *>(tmp + 2 * b_rows);
    int rc = cuda_status(cudaMemcpyAsync(d_row, row.data(), ncpl * 4, cudaMemcpyHostToDevice, st));
    if (rc == H2_OK) rc = cuda_status(cudaMemcpyAsync(d_col, op.cpl_col.data(), ncpl * 4, cudaMemcpyHostToDevice, st));
    if (rc == H2_OK)
        rc = cuda_status(cudaMemcpyAsync(d_cheb, op.cheb.data(), op.cheb.size() * 8, cudaMemcpyHostToDevice, st));
    if (rc == H2_OK) {
        h2k::KernelFn f{int(op.ker.kind), op.ker.a, op.ker.b, op.ker.deg};
        // gen_coupling stores kappa(xi^t_nu, xi^s_mu) at mu * k + nu; with the roles of row
        // and column swapped it stores kappa(xi^s_nu, xi^t_mu) = S_ts[mu][nu] (kappa is
        // symmetric) at mu * k + nu: S_ts row-major
        h2k::gen_coupling<double><<<unsigned(std::min<int64_t>(ncpl, 1 << 20)), 256, 0, st>>>(
            dS, d_col, d_row, ncpl, d_cheb, op.dim, op.p, op.k, op.k, f);
        rc = cuda_status(cudaGetLastError());
    }
    if (rc == H2_OK) rc = cuda_status(cudaStreamSynchronize(st));
    cudaFree(tmp);
    return rc;
}

int h2_exec_create(h2_exec *ex)
{
    if (!ex) return H2_EINVAL;
    *ex = h2_exec{};
    int lo_prio = 0, hi_prio = 0;
    cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
    cudaStream_t side = nullptr;
    cudaEvent_t a = nullptr, b = nullptr, c = nullptr;
    int rc = cuda_status(cudaStreamCreateWithPriority(&side, cudaStreamNonBlocking, hi_prio));
    if (rc == H2_OK) rc = cuda_status(cudaEventCreateWithFlags(&a, cudaEventDisableTiming));
    if (rc == H2_OK) rc = cuda_status(cudaEventCreateWithFlags(&b, cudaEventDisableTiming));
    if (rc == H2_OK) rc = cuda_status(cudaEventCreateWithFlags(&c, cudaEventDisableTiming));
    ex->side = side;
    ex->ev_up = a;
    ex->ev_top = b;
    ex->ev_topup = c;
    if (rc != H2_OK) h2_exec_destroy(ex);
    return rc;
}

void h2_exec_destroy(h2_exec *ex)
{
    if (!ex) return;
    if (ex->ev_up) cudaEventDestroy(static_cast<cudaEvent_t>(ex->ev_up));
    if (ex->ev_top) cudaEventDestroy(static_cast<cudaEvent_t>(ex->ev_top));
    if (ex->ev_topup) cudaEventDestroy(static_cast<cudaEvent_t>(ex->ev_topup));
    if (ex->side) cudaStreamDestroy(static_cast<cudaStream_t>(ex->side));
    *ex = h2_exec{};
}

int h2_device_check(h2_handle h)
{
    if (!h) return H2_EINVAL;
    if (!h->dev) return H2_ESTATE;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) {
        cudaGetLastError();
        return H2_ECUDA;
    }
    return cur == h->dev->device ? H2_OK : H2_EINVAL;
}

namespace {

// Take an idle fork/join context of the handle (creating one if every context is in use by
// another host thread's launch sequence); give it back with exec_release.
int exec_acquire(h2_device &dv, h2_exec *out)
{
    {
        std::lock_guard<std::mutex> lock(dv.exec_mutex);
        if (!dv.exec_idle.empty()) {
            *out = dv.exec_idle.back();
            dv.exec_idle.pop_back();
            return H2_OK;
        }
    }
    h2_exec ex;
    const int rc = h2_exec_create(&ex);
    if (rc != H2_OK) return rc;
    std::lock_guard<std::mutex> lock(dv.exec_mutex);
    dv.exec_all.push_back(ex);
    *out = ex;
    return H2_OK;
}

void exec_release(h2_device &dv, const h2_exec &ex)
{
    std::lock_guard<std::mutex> lock(dv.exec_mutex);
    dv.exec_idle.push_back(ex);
}

}  // namespace

int h2_matvec_exec(h2_handle h, const void *X, void *Y, int nv, double alpha, double beta, void *workspace,
                   size_t ws_bytes, void *cuda_stream, const h2_exec *exp)
{
    h2n::Range range("h2_matvec");
    if (!h || !X || !Y || nv < 1 || !workspace) return H2_EINVAL;
    if (!h->dev) return H2_ESTATE;
    h2_device &dv = *h->dev;
    if (ws_bytes < ws_layout(*h, dv, nv, nullptr, nullptr)) return H2_EINVAL;
    if (reinterpret_cast<uintptr_t>(workspace) % kAlign) return H2_EINVAL;
    // the kernels must run on the GPU that holds the operator (and, for a scratch or pooled
    // workspace, the workspace)
    const int dc = h2_device_check(h);
    if (dc != H2_OK) return dc;
    // a product without its own fork/join context borrows one of the handle's for the time its
    // launches are enqueued; the stream and event orderings it records stay valid after that
    h2_exec own{};
    if (!exp) {
        const int rc = exec_acquire(dv, &own);
        if (rc != H2_OK) return rc;
    }
    const h2_exec &ex = exp ? *exp : own;
    Workspace w;
    ws_layout(*h, dv, nv, &w, workspace);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    dv.products += 1;
    int rc;
    if (dv.tc)
        rc = launch_tc(*h, dv, static_cast<const float *>(X), static_cast<float *>(Y), nv, alpha, beta, w, st);
    else if (dv.esize == 8)
        rc = launch_product<double>(*h, dv, static_cast<const double *>(X), static_cast<double *>(Y), nv, alpha, beta,
                                    w, st, ex);
    else
        rc = launch_product<float>(*h, dv, static_cast<const float *>(X), static_cast<float *>(Y), nv, alpha, beta, w,
                                   st, ex);
    if (!exp) exec_release(dv, own);
    return rc;
}

extern "C" {

int h2_upload(h2_handle h, h2_prec prec, void *cuda_stream)
{
    h2n::Range range("h2_upload");
    if (!h) return H2_EINVAL;
    if (prec != H2_FP64 && prec != H2_FP32 && prec != H2_BF16X2 && prec != H2_FP32_MF) return H2_EINVAL;
    h2_op &op = *h;
    // a compressed operator (p = 0: explicit coupling blocks, no Chebyshev points) uploads in
    // FP64 / FP32 tiles only: the tensor tiles are 64 x 64 and the matrix-free precision
    // evaluates the kernel at the Chebyshev points
    if (op.p == 0 && (prec == H2_BF16X2 || prec == H2_FP32_MF)) return H2_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    h2_device_free(&op);
    h2_device *dv = new (std::nothrow) h2_device;
    if (!dv) return H2_ENOMEM;
    op.dev = dv;
    cudaGetDevice(&dv->device);
    cudaDeviceGetAttribute(&dv->num_sms, cudaDevAttrMultiProcessorCount, dv->device);
    dv->prec = prec;
    dv->esize = prec == H2_FP64 ? 8 : 4;  // bases and transfers: FP32 for H2_BF16X2
    dv->tc = prec == H2_BF16X2;
    dv->mf = prec == H2_FP32_MF;
    const size_t es = dv->esize;
    const int k = op.k;
    const int64_t nleaves = op.nleaves(), first_leaf = op.first_leaf(), ncpl = int64_t(op.cpl_col.size()),
                  ndns = int64_t(op.dns_col.size());

    // ---- layout constants
    std::vector<int32_t> perm32(op.n), leaf_lo(nleaves + 1);
    for (int64_t i = 0; i < op.n; ++i) perm32[i] = int32_t(op.perm[i]);
    for (int64_t t = 0; t < nleaves; ++t) leaf_lo[t] = int32_t(op.lo[first_leaf + t]);
    leaf_lo[nleaves] = int32_t(op.n);
    for (int64_t t = 0; t < nleaves; ++t) dv->max_leaf_rows = std::max(dv->max_leaf_rows, leaf_lo[t + 1] - leaf_lo[t]);
    if (dv->max_leaf_rows > kMaxLeaf) {
        h2_device_free(&op);
        return H2_EINVAL;
    }
    if (dv->tc && (k > 64 || dv->max_leaf_rows > 64)) {  // tensor tiles are 64 x 64
        h2_device_free(&op);
        return H2_EINVAL;
    }
    dv->kx = round4(k);
    dv->mp = round4(dv->max_leaf_rows);
    dv->kkp = int64_t(k) * round4(k);  // entries per stored coupling tile (ld kx)
    dv->tf32_ok = prec == H2_FP32 && k <= 64 && dv->max_leaf_rows <= 64;
    dv->warp_sweeps = !dv->tc && k <= h2s::kWsMaxRank && dv->mp <= 128;
    dv->cta64 = !dv->tc && es == 4 && k > h2s::kWsMaxRank && k <= 64 && dv->mp <= 128;
    dv->L = std::min(op.q, 4);
    dv->Lb = op.q - dv->L;
    dv->root_row = op.cpl_rowptr[2] > op.cpl_rowptr[1];
    const int kx = dv->kx, mp = dv->mp;

    // ---- per-block metadata
    std::vector<int32_t> cpl_row(ncpl), dns_row(ndns);
    std::vector<int64_t> dns_off(ndns + 1);
    for (int64_t t = 1; t <= op.nnodes; ++t)
        for (int64_t b = op.cpl_rowptr[t]; b < op.cpl_rowptr[t + 1]; ++b) cpl_row[b] = int32_t(t);
    dns_off[0] = 0;
    for (int64_t t = 0; t < nleaves; ++t)
        for (int64_t b = op.dns_rowptr[t]; b < op.dns_rowptr[t + 1]; ++b) {
            dns_row[b] = int32_t(t);
            const int64_t s = op.dns_col[b];
            const int64_t cnt = int64_t(round4(leaf_lo[t + 1] - leaf_lo[t])) * (leaf_lo[s + 1] - leaf_lo[s]);
            dns_off[b + 1] = dns_off[b] + (cnt + 31) / 32 * 32;  // 128-byte aligned blocks
        }
    const size_t tcb = h2s::kTcTileBytes;  // split-BF16 tile of one block
    // stored entries; the matrix-free precision keeps coordinates instead, and stores only the
    // coupling blocks of the levels above the bottom subtrees (a prefix of the level-ordered
    // CSR), which its side stream streams like the stored path
    const int64_t ncpl_top = op.cpl_rowptr[std::min<int64_t>(int64_t(1) << dv->Lb, op.nnodes + 1)];
    const size_t s_bytes = dv->mf ? align_up(size_t(ncpl_top) * dv->kkp * es)
                           : dv->tc ? size_t(ncpl) * tcb : align_up(size_t(ncpl) * dv->kkp * es);
    const size_t d_bytes = dv->mf ? 0 : dv->tc ? size_t(ndns) * tcb : align_up(size_t(dns_off[ndns]) * es);

    // ---- stream descriptors: coupling rows of levels >= Lb and all dense rows (bottom),
    //      coupling rows of levels < Lb (top)
    std::vector<h2s::StreamDesc> db, dt;
    std::vector<uint64_t> bb, bt;
    auto level_of = [](int64_t t) {
        int l = 0;
        for (; t > 1; t >>= 1) ++l;
        return l;
    };
    for (int64_t t = 1; t <= op.nnodes; ++t) {
        const int64_t b0 = op.cpl_rowptr[t], b1 = op.cpl_rowptr[t + 1];
        const bool is_top = !dv->tc && level_of(t) < dv->Lb;  // tensor path: one stream
        if (b0 == b1) {  // empty block row: its yhat row is written as zeros
            h2s::StreamDesc d{};
            d.out_node = int32_t(t);
            d.rows = int16_t(k);
            d.ld = int16_t(round4(k));
            d.flags = h2s::kZero | h2s::kLast;
            (is_top ? dt : db).push_back(d);
            (is_top ? bt : bb).push_back(uint64_t(k) * es);
        }
        for (int64_t b = b0; b < b1; ++b) {
            h2s::StreamDesc d{};
            d.src = dv->tc ? uint64_t(b) * tcb : uint64_t(b) * dv->kkp * es;
            d.x_node = op.cpl_col[b];
            d.out_node = int32_t(t);
            d.rows = int16_t(k);
            d.cols = int16_t(k);
            d.ld = int16_t(round4(k));
            d.flags = b + 1 == b1 ? h2s::kLast : 0;
            (is_top ? dt : db).push_back(d);
            (is_top ? bt : bb).push_back(dv->tc ? tcb : uint64_t(d.ld) * k * es);
        }
    }
    for (int64_t t = 0; t < nleaves; ++t) {
        const int64_t b0 = op.dns_rowptr[t], b1 = op.dns_rowptr[t + 1];
        for (int64_t b = b0; b < b1; ++b) {
            const int64_t s = op.dns_col[b];
            h2s::StreamDesc d{};
            d.src = dv->tc ? uint64_t(ncpl + b) * tcb : s_bytes + uint64_t(dns_off[b]) * es;
            d.x_node = int32_t(s);
            d.out_node = int32_t(t);
            d.rows = int16_t(leaf_lo[t + 1] - leaf_lo[t]);
            d.cols = int16_t(leaf_lo[s + 1] - leaf_lo[s]);
            d.ld = int16_t(round4(d.rows));
            d.flags = h2s::kDense | (b + 1 == b1 ? h2s::kLast : 0);
            db.push_back(d);
            bb.push_back(dv->tc ? tcb : uint64_t(d.ld) * d.cols * es);
        }
    }
    std::vector<int64_t> pb, pt, pd;
    dv->tile_cpl = uint32_t((uint64_t(k) * round4(k) * es + 15) / 16 * 16);
    dv->tile_dns = uint32_t((uint64_t(round4(dv->max_leaf_rows)) * dv->max_leaf_rows * es + 15) / 16 * 16);
    const bool split = !dv->tc && !dv->mf && ndns > 0 && dv->tile_dns >= 2 * dv->tile_cpl;
    if (split) {
        // db holds the coupling rows, then the dense rows: chunk the two parts separately
        size_t nc = 0;
        while (nc < db.size() && !(db[nc].flags & h2s::kDense)) ++nc;
        const std::vector<h2s::StreamDesc> dc(db.begin(), db.begin() + nc), dd(db.begin() + nc, db.end());
        const std::vector<uint64_t> bc(bb.begin(), bb.begin() + nc), bd(bb.begin() + nc, bb.end());
        // small tiles: smaller scheduling chunks, for the several CTAs per SM of their stream;
        // with warp sweeps (ranks <= 32) single-vector products take one warp per chunk: about
        // 48 blocks each
        const uint64_t cpl_target =
            dv->warp_sweeps ? std::min<uint64_t>(128 * 1024, 48 * uint64_t(dv->tile_cpl)) : 128 * 1024;
        if (!make_chunks(dc, bc, cpl_target, pb) || !make_chunks(dd, bd, 512 * 1024, pd)) {
            h2_device_free(&op);
            return H2_EINVAL;
        }
        for (auto &c : pd) c += int64_t(nc) << 16;  // descriptor indices of the whole array
    } else if (!make_chunks(db, bb, 512 * 1024, pb)) {
        h2_device_free(&op);
        return H2_EINVAL;  // a block row longer than one scheduling chunk
    }
    // the upper levels' rows: about eight coupling tiles per chunk (at least 8 KB), so that
    // small tiles spread over as many CTAs as large ones
    const uint64_t top_target = std::max<uint64_t>(8 * 1024, std::min<uint64_t>(128 * 1024, 8 * uint64_t(dv->tile_cpl)));
    if (!make_chunks(dt, bt, top_target, pt)) {
        h2_device_free(&op);
        return H2_EINVAL;
    }
    dv->n_chunks_dense = int64_t(pd.size());
    dv->grid_dense = int(std::max<int64_t>(1, std::min<int64_t>(dv->num_sms, dv->n_chunks_dense)));
    dv->n_chunks_bottom = int64_t(pb.size());
    dv->n_chunks_top = int64_t(pt.size());
    dv->n_desc_bottom = int64_t(db.size());
    dv->n_desc_top = int64_t(dt.size());
    dv->grid_bottom = int(std::max<int64_t>(1, std::min<int64_t>(dv->num_sms, dv->n_chunks_bottom)));
    dv->grid_top = int(std::max<int64_t>(1, std::min<int64_t>(dv->num_sms, dv->n_chunks_top)));

    // ---- arena layout
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += align_up(std::max<size_t>(bytes, 1));
        return o;
    };
    const size_t o_perm = take(op.n * 4), o_leaf = take((nleaves + 1) * 4), o_cptr = take((op.nnodes + 2) * 8);
    const size_t o_U = take(size_t(nleaves) * mp * kx * es), o_Ut = take(size_t(nleaves) * kx * mp * es);
    const size_t o_E = take(size_t(op.nnodes + 1) * k * kx * es), o_Et = take(size_t(op.nnodes + 1) * k * kx * es);
    const size_t o_vals = take(s_bytes + d_bytes);
    const size_t o_npts = dv->mf ? take(size_t(op.nnodes + 1) * k * sizeof(float4)) : 0;
    const size_t o_lpts = dv->mf ? take(size_t(nleaves) * mp * sizeof(float4)) : 0;
    const size_t o_db = take(db.size() * sizeof(h2s::StreamDesc)), o_dt = take(dt.size() * sizeof(h2s::StreamDesc));
    const size_t o_pb = take(pb.size() * 8), o_pt = take(pt.size() * 8), o_pd = take(pd.size() * 8), o_err = take(16);
    const size_t persistent = off;
    // temporaries for generation
    const size_t t_cheb = align_up(op.cheb.size() * 8), t_pts = align_up(size_t(op.n) * op.dim * 8);
    const size_t t_crow = align_up(ncpl * 4 + 4), t_ccol = align_up(ncpl * 4 + 4), t_drow = align_up(ndns * 4 + 4),
                 t_dcol = align_up(ndns * 4 + 4), t_doff = align_up((ndns + 1) * 8);
    const size_t tmp_bytes = t_cheb + t_pts + t_crow + t_ccol + t_drow + t_dcol + t_doff;

    char *arena = nullptr, *tmp = nullptr;
    if (cudaMalloc(&arena, persistent) != cudaSuccess) {
        cudaGetLastError();
        h2_device_free(&op);
        return H2_ENOMEM;
    }
    dv->arena = arena;
    dv->arena_bytes = persistent;
    if (cudaMalloc(&tmp, tmp_bytes) != cudaSuccess) {
        cudaGetLastError();
        h2_device_free(&op);
        return H2_ENOMEM;
    }
    dv->perm = reinterpret_cast<int32_t *>(arena + o_perm);
    dv->leaf_lo = reinterpret_cast<int32_t *>(arena + o_leaf);
    dv->cpl_rowptr = reinterpret_cast<int64_t *>(arena + o_cptr);
    dv->U = arena + o_U;
    dv->Ut = arena + o_Ut;
    dv->E = arena + o_E;
    dv->Et = arena + o_Et;
    dv->vals = reinterpret_cast<unsigned char *>(arena + o_vals);
    dv->desc_bottom = reinterpret_cast<h2s::StreamDesc *>(arena + o_db);
    dv->desc_top = reinterpret_cast<h2s::StreamDesc *>(arena + o_dt);
    dv->chunks_bottom = reinterpret_cast<int64_t *>(arena + o_pb);
    dv->chunks_top = reinterpret_cast<int64_t *>(arena + o_pt);
    dv->chunks_dense = reinterpret_cast<int64_t *>(arena + o_pd);
    dv->err = reinterpret_cast<int *>(arena + o_err);
    if (dv->mf) {
        dv->mfa.node_pts = reinterpret_cast<const float4 *>(arena + o_npts);
        dv->mfa.leaf_pts = reinterpret_cast<const float4 *>(arena + o_lpts);
        dv->mfa.k = k;
        dv->mfa.p = op.p;
        dv->mfa.dim = op.dim;
        dv->mfa.lp = (op.p & (op.p - 1)) == 0 ? __builtin_ctz(unsigned(op.p)) : -1;
        dv->mfa.a = float(op.ker.a);
        dv->mfa.neg_inv_a = op.ker.a != 0.0 ? float(-1.0 / op.ker.a) : 0.f;
        dv->mfa.neg_b = float(-op.ker.b);
        dv->mfa.deg = op.ker.deg;
    }
    char *tp = tmp;
    double *d_cheb = reinterpret_cast<double *>(tp);
    tp += t_cheb;
    double *d_pts = reinterpret_cast<double *>(tp);
    tp += t_pts;
    int32_t *d_crow = reinterpret_cast<int32_t *>(tp);
    tp += t_crow;
    int32_t *d_ccol = reinterpret_cast<int32_t *>(tp);
    tp += t_ccol;
    int32_t *d_drow = reinterpret_cast<int32_t *>(tp);
    tp += t_drow;
    int32_t *d_dcol = reinterpret_cast<int32_t *>(tp);
    tp += t_dcol;
    int64_t *d_doff = reinterpret_cast<int64_t *>(tp);

    // ---- bases and transfers in the target precision and tile layouts
    std::vector<unsigned char> Ub(size_t(nleaves) * mp * kx * es, 0), Utb(size_t(nleaves) * kx * mp * es, 0);
    std::vector<unsigned char> Eb(size_t(op.nnodes + 1) * k * kx * es, 0), Etb(size_t(op.nnodes + 1) * k * kx * es, 0);
    auto put = [&](std::vector<unsigned char> &buf, size_t idx, double v) {
        if (es == 8) reinterpret_cast<double *>(buf.data())[idx] = v;
        else reinterpret_cast<float *>(buf.data())[idx] = float(v);
    };
    for (int64_t t = 0; t < nleaves; ++t)
        for (int i = 0; i < leaf_lo[t + 1] - leaf_lo[t]; ++i)
            for (int nu = 0; nu < k; ++nu) {
                const double u = op.U[(int64_t(leaf_lo[t]) + i) * k + nu];
                put(Ub, (size_t(t) * mp + i) * kx + nu, u);
                put(Utb, (size_t(t) * kx + nu) * mp + i, u);
            }
    for (int64_t c = 2; c <= op.nnodes; ++c)
        for (int mu = 0; mu < k; ++mu)
            for (int nu = 0; nu < k; ++nu) {
                const double e = op.E[(size_t(c) * k + mu) * k + nu];
                put(Eb, (size_t(c) * k + mu) * kx + nu, e);
                put(Etb, (size_t(c) * k + nu) * kx + mu, e);
            }
    std::vector<double> pts_tree(size_t(op.n) * op.dim);
    for (int64_t i = 0; i < op.n; ++i)
        for (int d = 0; d < op.dim; ++d) pts_tree[i * op.dim + d] = op.pts[op.perm[i] * op.dim + d];

    int rc = H2_OK;
    auto cp = [&](void *dst, const void *src, size_t bytes) {
        if (rc == H2_OK && bytes) rc = cuda_status(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st));
    };
    cp(dv->perm, perm32.data(), op.n * 4);
    cp(dv->leaf_lo, leaf_lo.data(), (nleaves + 1) * 4);
    cp(dv->cpl_rowptr, op.cpl_rowptr.data(), (op.nnodes + 2) * 8);
    cp(dv->U, Ub.data(), Ub.size());
    cp(dv->Ut, Utb.data(), Utb.size());
    cp(dv->E, Eb.data(), Eb.size());
    cp(dv->Et, Etb.data(), Etb.size());
    cp(dv->desc_bottom, db.data(), db.size() * sizeof(h2s::StreamDesc));
    cp(dv->desc_top, dt.data(), dt.size() * sizeof(h2s::StreamDesc));
    cp(dv->chunks_bottom, pb.data(), pb.size() * 8);
    cp(dv->chunks_top, pt.data(), pt.size() * 8);
    if (!pd.empty()) cp(dv->chunks_dense, pd.data(), pd.size() * 8);
    cp(d_cheb, op.cheb.data(), op.cheb.size() * 8);
    cp(d_pts, pts_tree.data(), pts_tree.size() * 8);
    cp(d_crow, cpl_row.data(), ncpl * 4);
    cp(d_ccol, op.cpl_col.data(), ncpl * 4);
    cp(d_drow, dns_row.data(), ndns * 4);
    cp(d_dcol, op.dns_col.data(), ndns * 4);
    cp(d_doff, dns_off.data(), (ndns + 1) * 8);
    if (rc == H2_OK) rc = cuda_status(cudaMemsetAsync(dv->err, 0, 16, st));
    // explicit coupling blocks, rounded once to the precision, in the tile layout (ld kx)
    const bool explicit_s = !op.S.empty();
    std::vector<unsigned char> Sb(explicit_s ? size_t(ncpl) * dv->kkp * es : 0, 0);
    if (explicit_s) {
        // op.S holds S_ts[nu][mu] row-major; the tiles hold each block transposed (entry
        // (nu, mu) at mu * kx + nu), as gen_coupling writes them
        for (int64_t b = 0; b < ncpl; ++b)
            for (int mu = 0; mu < k; ++mu)
                for (int nu = 0; nu < k; ++nu) put(Sb, (size_t(b) * k + mu) * kx + nu, op.S[(size_t(b) * k + nu) * k + mu]);
        cp(dv->vals, Sb.data(), Sb.size());
    }
    const int64_t ncpl_gen = explicit_s ? 0 : ncpl;
    if (rc == H2_OK)
        rc = dv->mf ? generate_mf_points(op, *dv, d_cheb, d_pts, st)
             : dv->tc ? generate_tc_blocks(op, *dv, d_crow, d_drow, d_dcol, d_ccol, d_cheb, d_pts, s_bytes, st)
             : es == 8 ? generate_blocks<double>(op, *dv, d_crow, d_drow, d_dcol, d_doff, d_ccol, d_cheb, d_pts, s_bytes, st,
                                                 ncpl_gen, ndns)
                       : generate_blocks<float>(op, *dv, d_crow, d_drow, d_dcol, d_doff, d_ccol, d_cheb, d_pts, s_bytes, st,
                                                ncpl_gen, ndns);
    if (rc == H2_OK && dv->mf && ncpl_top > 0)
        rc = generate_blocks<float>(op, *dv, d_crow, d_drow, d_dcol, d_doff, d_ccol, d_cheb, d_pts, s_bytes, st,
                                    ncpl_top, 0);
    if (rc == H2_OK) rc = cuda_status(cudaStreamSynchronize(st));
    cudaFree(tmp);
    if (rc == H2_OK) {  // the first fork/join context
        h2_exec ex;
        rc = h2_exec_create(&ex);
        if (rc == H2_OK) {
            dv->exec_all.push_back(ex);
            dv->exec_idle.push_back(ex);
        }
    }
    if (rc != H2_OK) h2_device_free(&op);
    return rc;
}

size_t h2_workspace_bytes(h2_handle h, int nv)
{
    if (!h || !h->dev || nv < 1) return 0;
    return ws_layout(*h, *h->dev, nv, nullptr, nullptr);
}

int h2_matvec_ws(h2_handle h, const void *X, void *Y, int nv, double alpha, double beta, void *workspace,
                 size_t ws_bytes, void *cuda_stream)
{
    return h2_matvec_exec(h, X, Y, nv, alpha, beta, workspace, ws_bytes, cuda_stream, nullptr);
}

int h2_matvec(h2_handle h, const void *X, void *Y, int nv, double alpha, double beta, void *cuda_stream)
{
    if (!h || !X || !Y || nv < 1) return H2_EINVAL;
    if (!h->dev) return H2_ESTATE;
    const int dc = h2_device_check(h);
    if (dc != H2_OK) return dc;
    h2_device &dv = *h->dev;
    const size_t need = ws_layout(*h, dv, nv, nullptr, nullptr);
    // this stream's workspace (created on its first product)
    h2_device::StreamWs *e = nullptr;
    {
        std::lock_guard<std::mutex> lock(dv.ws_mutex);
        for (auto &w : dv.stream_ws)
            if (w->stream == cuda_stream) e = w.get();
        if (!e) {
            auto w = std::make_unique<h2_device::StreamWs>();
            w->stream = cuda_stream;
            if (cudaEventCreateWithFlags(&w->done, cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                return H2_ECUDA;
            }
            e = w.get();
            dv.stream_ws.push_back(std::move(w));
        }
    }
    std::lock_guard<std::mutex> lock(e->m);
    if (e->bytes < need) {
        if (e->ws) {
            cudaEventSynchronize(e->done);  // the last product on it has finished
            cudaFree(e->ws);
            std::lock_guard<std::mutex> l2(dv.ws_mutex);
            dv.ws_total -= e->bytes;
            e->ws = nullptr;
            e->bytes = 0;
        }
        if (cudaMalloc(&e->ws, need) != cudaSuccess) {
            cudaGetLastError();
            e->ws = nullptr;
            return H2_ENOMEM;
        }
        e->bytes = need;
        std::lock_guard<std::mutex> l2(dv.ws_mutex);
        dv.ws_total += need;
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // a stream handle can be reused after cudaStreamDestroy while the old stream's product is
    // still running: order this product after the previous one on this workspace
    cudaStreamWaitEvent(st, e->done, 0);
    const int rc = h2_matvec_exec(h, X, Y, nv, alpha, beta, e->ws, e->bytes, cuda_stream, nullptr);
    cudaEventRecord(e->done, st);
    return rc;
}

int h2_set_fp32_tensor(h2_handle h, int enable)
{
    if (!h) return H2_EINVAL;
    if (!h->dev) return H2_ESTATE;
    h->dev->tf32_on = enable != 0;
    return H2_OK;
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
        const int64_t l = dv.phase_launches[i].exchange(0);
        if (phase_launches) phase_launches[i] = l;
        dv.phase_ms[i] = 0;
    }
    const int64_t pr = dv.products.exchange(0);
    if (products) *products = pr;
    int flag = 0;
    if (cudaMemcpy(&flag, dv.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return H2_ECUDA;
    return flag ? H2_ETIMEOUT : H2_OK;
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
    h2n::Range range("h2_build");
    if (!out) return H2_EINVAL;
    *out = nullptr;
    if (leaf_size > kMaxLeaf) return H2_EINVAL;
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
    info->device_bytes = op.dev ? op.dev->arena_bytes + op.dev->ws_total : 0;
    return H2_OK;
}

int h2_get_level_ranks(h2_handle h, int *ranks)
{
    if (!h || !ranks) return H2_EINVAL;
    for (int l = 0; l <= h->q; ++l) ranks[l] = h->level_rank.empty() ? h->k : h->level_rank[l];
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
    case H2_ECANCELED: return "cancelled";
    case H2_ENOTCONV: return "not converged";
    default: return "unknown status";
    }
}

// ---------------------------------------------------------------- batched products

int h2_batch_create(const h2_handle *ops, int count, const void *const *X, void *const *Y, const int *nv, double alpha,
                    double beta, int flags, h2_batch_t *out)
{
    h2n::Range range("h2_batch_create");
    if (!out) return H2_EINVAL;
    *out = nullptr;
    if (!ops || count < 1 || !X || !Y || !nv) return H2_EINVAL;
    size_t esize = 0;
    for (int i = 0; i < count; ++i) {
        if (!ops[i] || !X[i] || !Y[i] || nv[i] < 1) return H2_EINVAL;
        const h2_device *dv = ops[i]->dev;
        if (!dv) return H2_ESTATE;
        if (dv->tc || dv->mf) return H2_EINVAL;  // stored FP64 or FP32 members only
        if (esize && dv->esize != esize) return H2_EINVAL;
        esize = dv->esize;
        if (!(nv[i] <= kChunk || (wide_ok(*dv) && nv[i] <= kWidePass))) return H2_EINVAL;  // one pass each
    }
    h2_batch *b = new (std::nothrow) h2_batch;
    if (!b) return H2_ENOMEM;
    b->esize = esize;
    b->alpha = alpha;
    b->beta = beta;
    cudaGetDevice(&b->device);
    cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
    int rc = H2_OK;
    // workspaces, one allocation
    std::vector<size_t> wsz(static_cast<size_t>(count));
    size_t total = 0;
    for (int i = 0; i < count; ++i) {
        wsz[size_t(i)] = align_up(ws_layout(*ops[i], *ops[i]->dev, nv[i], nullptr, nullptr));
        total += wsz[size_t(i)];
    }
    rc = cuda_status(cudaMalloc(&b->ws_mem, total));
    size_t off = 0;
    for (int i = 0; rc == H2_OK && i < count; ++i) {
        h2_batch::Member m;
        m.op = ops[i];
        m.X = X[i];
        m.Y = Y[i];
        m.nv = nv[i];
        ws_layout(*ops[i], *ops[i]->dev, nv[i], &m.w, static_cast<char *>(b->ws_mem) + off);
        off += wsz[size_t(i)];
        b->members.push_back(m);
    }
    // groups by accumulator width and tile-size class (the next power of two of a row's
    // largest tile, so that small tiles get deep pipelines of small stages); descriptors are
    // tagged with the member's index in their group's table, and rows stay whole
    auto tile_class = [](uint64_t bytes) {
        uint64_t c = 1024;
        while (c < bytes) c <<= 1;
        return c;
    };
    for (int i = 0; rc == H2_OK && i < count; ++i) {
        const int wc = width_class(nv[i]);
        const h2_op &op = *ops[i];
        const h2_device &dv = *op.dev;
        std::vector<h2s::StreamDesc> d(size_t(dv.n_desc_bottom + dv.n_desc_top));
        if (dv.n_desc_bottom)
            rc = cuda_status(cudaMemcpy(d.data(), dv.desc_bottom, size_t(dv.n_desc_bottom) * sizeof(h2s::StreamDesc),
                                        cudaMemcpyDeviceToHost));
        if (rc == H2_OK && dv.n_desc_top)
            rc = cuda_status(cudaMemcpy(d.data() + dv.n_desc_bottom, dv.desc_top,
                                        size_t(dv.n_desc_top) * sizeof(h2s::StreamDesc), cudaMemcpyDeviceToHost));
        std::vector<std::pair<size_t, int>> slot_of;  // group index -> this member's slot there
        size_t r0 = 0;
        for (size_t e = 0; rc == H2_OK && e < d.size(); ++e) {
            if (!(d[e].flags & h2s::kLast)) continue;
            // the row d[r0 .. e]
            uint64_t row_max = 0;
            std::vector<uint64_t> tb(e + 1 - r0);
            for (size_t j = r0; j <= e; ++j) {
                tb[j - r0] = (d[j].flags & h2s::kZero) ? uint64_t(op.k) * esize : uint64_t(d[j].ld) * d[j].cols * esize;
                row_max = std::max(row_max, tb[j - r0]);
            }
            const uint64_t cls = tile_class(row_max);
            size_t gi = 0;
            while (gi < b->groups.size() && !(b->groups[gi].width == wc && b->groups[gi].tile_class == cls)) ++gi;
            if (gi == b->groups.size()) {
                b->groups.emplace_back();
                b->groups.back().width = wc;
                b->groups.back().tile_class = cls;
            }
            h2_batch::Group &g = b->groups[gi];
            int slot = -1;
            for (auto &sv : slot_of)
                if (sv.first == gi) slot = sv.second;
            if (slot < 0) {
                slot = int(g.members.size());
                g.members.push_back(i);
                slot_of.push_back({gi, slot});
                g.x_bytes = std::max<uint32_t>(g.x_bytes, uint32_t(std::max(dv.mp, dv.kx) * wc * esize));
            }
            for (size_t j = r0; j <= e; ++j) {
                h2s::StreamDesc x = d[j];
                x.pad1 = slot;
                g.desc.push_back(x);
                g.bytes.push_back(tb[j - r0]);
                g.tile_bytes = std::max<uint32_t>(g.tile_bytes, uint32_t((tb[j - r0] + 15) / 16 * 16));
            }
            r0 = e + 1;
        }
    }
    for (h2_batch::Group &g : b->groups) {
        if (rc != H2_OK) break;
        g.chunk_cap = std::max<size_t>(1, g.desc.size());
        rc = cuda_status(cudaMalloc(&g.d_desc, std::max<size_t>(1, g.desc.size()) * sizeof(h2s::StreamDesc)));
        if (rc == H2_OK && !g.desc.empty())
            rc = cuda_status(cudaMemcpy(g.d_desc, g.desc.data(), g.desc.size() * sizeof(h2s::StreamDesc),
                                        cudaMemcpyHostToDevice));
        if (rc == H2_OK) rc = cuda_status(cudaMalloc(&g.d_chunks, g.chunk_cap * 8));
    }
    if (rc == H2_OK) rc = esize == 8 ? batch_build_group_tables<double>(*b) : batch_build_group_tables<float>(*b);
    if (rc == H2_OK && !(flags & H2_BATCH_MEMBER_SWEEPS))
        rc = esize == 8 ? batch_build_all_sweeps<double>(*b) : batch_build_all_sweeps<float>(*b);
    if (rc == H2_OK && b->groups.size() > size_t(kBatchGroups)) rc = H2_EINVAL;
    if (rc == H2_OK) rc = cuda_status(cudaMalloc(&b->d_flags, (kBatchGroups + 1) * sizeof(int)));
    if (rc == H2_OK) rc = cuda_status(cudaMemset(b->d_flags, 0, (kBatchGroups + 1) * sizeof(int)));
    if (rc == H2_OK) rc = cuda_status(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    const int nb = std::min(count, 16);
    for (int j = 0; rc == H2_OK && j < nb; ++j) {
        cudaStream_t s = nullptr;
        cudaEvent_t e = nullptr;
        rc = cuda_status(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        if (rc == H2_OK) b->branches.push_back(s);
        if (rc == H2_OK) rc = cuda_status(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        if (rc == H2_OK) b->ev_branch.push_back(e);
    }
    if (rc == H2_OK) rc = cuda_status(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
    if (rc == H2_OK) rc = cuda_status(cudaEventCreateWithFlags(&b->ev_mid, cudaEventDisableTiming));
    // default configuration, one eager upsweep and merged stream (kernel attributes, valid
    // trees for tuning; X is read, Y is not written), then the tuned configuration and the
    // captured graph
    auto configure = [&](bool tune) {
        return esize == 8 ? batch_configure<double>(*b, tune, b->cap) : batch_configure<float>(*b, tune, b->cap);
    };
    auto enqueue = [&](cudaStream_t st, bool with_down) {
        return esize == 8 ? batch_enqueue<double>(*b, st, with_down) : batch_enqueue<float>(*b, st, with_down);
    };
    if (rc == H2_OK) rc = configure(false);
    if (rc == H2_OK) rc = enqueue(b->cap, false);  // leaves every Y untouched
    if (rc == H2_OK) rc = cuda_status(cudaStreamSynchronize(b->cap));
    if (rc == H2_OK && (flags & H2_BATCH_AUTOTUNE)) {
        for (auto &g : b->groups) g.tuned = false;
        rc = configure(true);
        if (rc == H2_OK) rc = cuda_status(cudaStreamSynchronize(b->cap));
    }
    if (rc == H2_OK) rc = cuda_status(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    if (rc == H2_OK) {
        int rc2 = enqueue(b->cap, true);
        const int rc3 = cuda_status(cudaStreamEndCapture(b->cap, &b->graph));
        rc = rc2 != H2_OK ? rc2 : rc3;
    }
    if (rc == H2_OK) rc = cuda_status(cudaGraphInstantiate(&b->exec, b->graph, 0));
    if (rc != H2_OK) {
        cudaGetLastError();
        batch_free(b);
        return rc;
    }
    *out = b;
    return H2_OK;
}

int h2_batch_run(h2_batch_t b, void *cuda_stream)
{
    h2n::Range range("h2_batch_run");
    if (!b || !b->exec) return H2_EINVAL;
    return cuda_status(cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(cuda_stream)));
}

int h2_batch_check(h2_batch_t b)
{
    if (!b) return H2_EINVAL;
    int flag = 0;
    if (cudaMemcpy(&flag, b->d_flags + kBatchGroups, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return H2_ECUDA;
    for (const auto &m : b->members) {
        int f = 0;
        if (cudaMemcpy(&f, m.op->dev->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return H2_ECUDA;
        flag |= f;
    }
    return flag ? H2_ETIMEOUT : H2_OK;
}

int h2_batch_describe(h2_batch_t b, char *buf, size_t len)
{
    if (!b || !buf || len == 0) return H2_EINVAL;
    std::ostringstream o;
    o << "members " << b->members.size() << " branches " << b->branches.size();
    for (const auto &g : b->groups)
        o << "; width " << g.width << ": members " << g.members.size() << " blocks " << g.desc.size() << " chunks "
          << g.nchunks << " ctas/sm " << g.cfg.per_sm << " stages " << g.cfg.ns << " chunk " << g.cfg.chunk_target
          << (g.tuned ? " (tuned)" : " (default)") << " tiles<=" << g.tile_class;
    size_t own = 0;
    for (const auto &m : b->members) own += m.merged ? 0 : 1;
    for (const auto &c : b->sweeps)
        o << "; sweeps width " << c.width << ": " << c.up.size() << " up + " << c.down.size() << " down launches";
    o << "; members with their own sweeps " << own;
    const std::string str = o.str();
    const size_t n = std::min(len - 1, str.size());
    std::memcpy(buf, str.data(), n);
    buf[n] = 0;
    return H2_OK;
}

int h2_batch_destroy(h2_batch_t b)
{
    if (!b) return H2_EINVAL;
    if (b->cap) cudaStreamSynchronize(b->cap);
    batch_free(b);
    return H2_OK;
}

}  // extern "C\"
