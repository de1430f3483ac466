// h2_stream.cuh -- pipelined kernels of the H^2 product (FP64 / FP32 entries, nv <= NVMAX).
//
// Every matrix tile (coupling block, dense block, leaf basis, transfer) streams from HBM
// into a ring of shared-memory stages through 1-D bulk copies issued by one producer
// thread (warp 4); four consumer warps (128 threads) multiply each tile with a vector
// segment and reduce in a fixed order (deterministic, no atomics on data).
//
//   k_up_sub      upsweep xhat^{l-1}_p = sum_c E_c^T xhat^l_c over CTA-resident subtrees of a
//                 few levels, starting from the leaf projections xhat^q_t = U_t^T x_t or from
//                 a level computed by an earlier launch (Sec. 3.1, Alg 1);
//   k_stream      block rows of coupling blocks (yhat^l_t = sum_s S_ts xhat^l_s, Sec. 3.2,
//                 Alg 4) and of dense blocks (A_de x, Sec. 3) from one flat descriptor list,
//                 handed out to persistent CTAs in chunks of whole rows by an atomic ticket;
//                 an empty block row is written as zeros, so every yhat row is defined;
//   k_down_sub    downsweep yhat^l_c = E_c yhat^{l-1}_p + yhat^l_c over CTA-resident subtrees
//                 of a few levels, ending either in a level handed to the next launch or in
//                 the leaf expansion y_t = U_t yhat^q_t (Sec. 3.3, Alg 6), the dense partial
//                 result and the epilogue Y[perm] = alpha y + beta Y.
//
// Tile layouts (element type T, ld = leading dimension): the consumer always computes
// out[o] = sum_j tile[j * ld + o] * x[j], so each tile is stored with the output index
// contiguous: U_t as [i][nu] (ld kx) for the upsweep, U_t^T as [nu][i] (ld mp) for the
// expansion, E_c as [mu][nu] (ld kx) for the upsweep, E_c^T as [nu][mu] (ld kx) for the
// downsweep, S_ts^T as [mu][nu] (ld k) and D_ts^T as [j][i] (ld rows_t).
// Vector trees: xh, yh as [node][v][kx]; permuted input xt and dense result yd as
// [leaf][v][mp]; kx = k rounded up to 4, mp = largest leaf rounded up to 4, so every
// segment starts on a 16-byte boundary.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>
#include <type_traits>

#include "h2_pipe.cuh"

namespace h2s {

constexpr int kConsumers = 128;  // 4 consumer warps
constexpr int kThreads = 160;    // + 1 producer warp
constexpr int kChunkDesc = 256;  // most descriptors in one scheduling chunk
constexpr int kRedElems = 512;   // group-exchange buffer per vector (elements of T)

struct alignas(16) StreamDesc {
    uint64_t src;     // byte offset of the tile in the value buffer
    int32_t x_node;   // heap index (coupling) or leaf index (dense) of the input segment
    int32_t out_node; // heap index (coupling) or leaf index (dense) of the output segment
    int16_t rows, cols;
    int16_t flags;    // kDense | kLast | kZero | kEnd
    int16_t ld;       // leading dimension of the stored tile: rows rounded up to 4, zero-padded
    int32_t pad1;
};
constexpr int16_t kDense = 1;  // dense block (else coupling block)
constexpr int16_t kLast = 2;   // last block of its row: reduce and store the row
constexpr int16_t kZero = 4;   // empty row: no data, store zeros
constexpr int16_t kEnd = 8;    // no more work (consumers stop)

template <typename T>
struct Op {
    int64_t n, nleaves, first_leaf;
    int k, kx, mp, q;
    const int32_t *perm, *leaf_lo;
    const T *U, *Ut, *E, *Et;
    const unsigned char *vals;
};

template <typename T>
struct Vec {
    const T *X;
    T *Y;
    int nv;  // vectors in this pass
    int vs;  // vectors per node in the tree layouts (>= nv)
    T alpha, beta;
    T *xt, *yd, *xh, *yh;
    int *tickets;  // kTickets scheduling words of this product (zeroed by k_gather)
    int *err;
    // tensor-core path only: split-BF16 B-operand tiles of every node's xhat (written by the
    // upsweep) and of every leaf's permuted input (written by the gather), np rows each
    unsigned char *xb = nullptr, *xtb = nullptr;
    int np = 0;
    // wide passes: row-major copies of X and of the result in user order ([row][v], ld ldr),
    // so that the gather and the leaf epilogue move whole rows of nv values
    T *xr = nullptr, *yr = nullptr;
    int ldr = 0;
    // warp-per-node sweeps (h2_warpsweep.cuh): the nodes' completion flags, zeroed by k_gather
    int *flags = nullptr;
    int64_t nflags = 0;
};

// Scheduling words of a product: [0] bottom block stream, [1] top block stream, [2] dense
// stream, [4 .. 7] the warp sweeps' launches, [8] their abort word.
constexpr int kTickets = 16;

// Bytes of one node's split-BF16 vector tile: np rows (vectors) x 64 bf16, hi then lo.
__host__ __device__ constexpr uint32_t vec_tile_bytes(int np) { return 2u * uint32_t(np) * 128u; }

// Byte offset of element (row r, column k) in a K-major bf16 tile with 64 columns per
// 128-byte row, 128-byte swizzle (the 16-byte chunk index XORed with the row index mod 8).
__host__ __device__ inline uint32_t sw128(int r, int k)
{
    const uint32_t o = uint32_t(r) * 128u + uint32_t(k) * 2u;
    return o ^ (((o >> 7) & 7u) << 4);
}

// Byte offset of element (row r, column k < 64) in a K-major tf32 tile of `rows` rows: two
// K-blocks of 32 columns (128 bytes per row), each `rows` x 128 bytes with the 128-byte swizzle.
__host__ __device__ inline uint32_t sw128_tf32(int r, int k, int rows)
{
    const uint32_t o = uint32_t(r) * 128u + uint32_t(k & 31) * 4u;
    return uint32_t(k >> 5) * uint32_t(rows) * 128u + (o ^ (((o >> 7) & 7u) << 4));
}

// The split-TF32 pair of x: hi = x with its 13 low mantissa bits cleared (exact as a TF32
// operand), lo = x - hi (exact in FP32, |lo| < 2^-10 |x|; the tensor core keeps it to TF32
// precision).
__device__ __forceinline__ void split_tf32(float x, float &hi, float &lo)
{
    hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
    lo = x - hi;
}

struct Pipe {
    int ns;               // stages
    uint32_t tile_bytes;  // bytes of one tile slot
    uint32_t x_bytes;     // bytes of one vector slot
};

__host__ __device__ constexpr int rpad(int r) { return r <= 32 ? 32 : (r <= 64 ? 64 : 128); }

template <typename T>
struct Smem {
    unsigned char *tiles, *xs;
    StreamDesc *desc;
    uint64_t *full, *empty;
    T *red, *sub;
    StreamDesc *dbuf;  // [2][kChunkDesc] (k_stream only)
    uint64_t *dbar;    // [2]
    int *abort_flag;
};

// Vectors per pass from which the wide accumulator (AccW) replaces the group-reduced one.
constexpr int kWideMin = 8;

// Elements of the column-group exchange buffer per vector: the narrow accumulator's groups,
// or, in the block streams (stream = true), the split-column slices of AccWK (S - 1 slices
// of 64 outputs: S = 4, 2 at 8, 16 vectors); AccW (sweeps; streams of 32 vectors) needs none.
template <int NVMAX>
__host__ __device__ constexpr int red_elems(bool stream)
{
    return NVMAX < kWideMin ? kRedElems : (!stream || NVMAX >= 32) ? 0 : NVMAX == 8 ? 3 * 64 : 64;
}

template <typename T, int NVMAX>
__host__ __device__ inline size_t smem_bytes(const Pipe &p, int sub_nodes, int kx, bool chunks)
{
    size_t b = size_t(p.ns) * (p.tile_bytes + p.x_bytes);
    b += size_t(p.ns) * sizeof(StreamDesc);
    b += size_t(2 * p.ns) * sizeof(uint64_t);
    b += size_t(red_elems<NVMAX>(chunks)) * NVMAX * sizeof(T);
    b += size_t(sub_nodes) * kx * NVMAX * sizeof(T);
    if (chunks) b += 2 * kChunkDesc * sizeof(StreamDesc) + 2 * sizeof(uint64_t);
    b += 16;
    return b;
}

template <typename T, int NVMAX>
__device__ inline Smem<T> carve(unsigned char *base, const Pipe &p, int sub_nodes, int kx, bool chunks)
{
    Smem<T> s;
    unsigned char *c = base;
    s.tiles = c;
    c += size_t(p.ns) * p.tile_bytes;
    s.xs = c;
    c += size_t(p.ns) * p.x_bytes;
    s.desc = reinterpret_cast<StreamDesc *>(c);
    c += size_t(p.ns) * sizeof(StreamDesc);
    s.full = reinterpret_cast<uint64_t *>(c);
    s.empty = s.full + p.ns;
    c += size_t(2 * p.ns) * sizeof(uint64_t);
    s.red = reinterpret_cast<T *>(c);
    c += size_t(red_elems<NVMAX>(chunks)) * NVMAX * sizeof(T);
    s.sub = reinterpret_cast<T *>(c);
    c += size_t(sub_nodes) * kx * NVMAX * sizeof(T);
    s.dbuf = nullptr;
    s.dbar = nullptr;
    if (chunks) {
        s.dbuf = reinterpret_cast<StreamDesc *>(c);
        c += 2 * kChunkDesc * sizeof(StreamDesc);
        s.dbar = reinterpret_cast<uint64_t *>(c);
        c += 2 * sizeof(uint64_t);
    }
    s.abort_flag = reinterpret_cast<int *>(c);
    return s;
}

template <typename T>
__device__ inline void init_pipe(Smem<T> &s, const Pipe &p, int consumers = kConsumers)
{
    if (threadIdx.x == 0) {
        for (int i = 0; i < p.ns; ++i) {
            h2p::mbar_init(&s.full[i], 1);
            h2p::mbar_init(&s.empty[i], consumers / 32);
        }
        if (s.dbar) {
            h2p::mbar_init(&s.dbar[0], 1);
            h2p::mbar_init(&s.dbar[1], 1);
        }
        *s.abort_flag = 0;
        h2p::fence_barrier_init();
    }
    __syncthreads();
}

// Ring position shared by the producer and the consumers (they walk the same sequence).
struct Ring {
    int stage = 0;
    uint32_t phase = 0;
    int ns;
    uint32_t issued = 0;  // producer only: stages that received a copy (bit per stage)
    uint32_t parity = 0;  // producer only: phase parity of each stage's last copy
    __device__ explicit Ring(int n) : ns(n) {}
    __device__ void next()
    {
        if (++stage == ns) {
            stage = 0;
            phase ^= 1u;
        }
    }
};

// Producer epilogue: after an abort, wait (bounded, about a second per stage) until every
// copy this CTA started has landed, so that no bulk copy is still writing into shared
// memory when the CTA exits.
template <typename T>
__device__ inline void drain_on_abort(Smem<T> &s, const Ring &r)
{
    if (!*s.abort_flag) return;
    for (int i = 0; i < r.ns; ++i) {
        if (!(r.issued >> i & 1u)) continue;
        const uint32_t par = r.parity >> i & 1u;
        const long long t0 = clock64();
        while (!h2p::mbar_try_wait(&s.full[i], par) && clock64() - t0 < h2p::kWaitCycles) {
        }
    }
}

// Producer side: claim the next stage and start copying a tile and up to two vector
// segments (into the first and the second half of the stage's vector slot). Returns false
// if the pipeline aborted.
template <typename T>
__device__ inline bool produce(Smem<T> &s, const Pipe &p, Ring &r, const void *tile, uint32_t tile_bytes,
                               const void *x, uint32_t x_bytes, const void *x2, uint32_t x2_bytes,
                               const StreamDesc *d, int *err)
{
    if (!h2p::mbar_wait(&s.empty[r.stage], r.phase ^ 1u, s.abort_flag, err)) return false;
    if (d) s.desc[r.stage] = *d;
    unsigned char *xs = s.xs + size_t(r.stage) * p.x_bytes;
    h2p::mbar_arrive_expect_tx(&s.full[r.stage], tile_bytes + x_bytes + x2_bytes);
    if (tile_bytes) h2p::bulk_g2s(s.tiles + size_t(r.stage) * p.tile_bytes, tile, tile_bytes, &s.full[r.stage]);
    if (x_bytes) h2p::bulk_g2s(xs, x, x_bytes, &s.full[r.stage]);
    if (x2_bytes) h2p::bulk_g2s(xs + p.x_bytes / 2, x2, x2_bytes, &s.full[r.stage]);
    r.issued |= 1u << r.stage;
    r.parity = (r.parity & ~(1u << r.stage)) | (r.phase << r.stage);
    r.next();
    return true;
}

template <typename T>
__device__ __forceinline__ const T *stage_tile(const Smem<T> &s, const Pipe &p, int stage)
{
    return reinterpret_cast<const T *>(s.tiles + size_t(stage) * p.tile_bytes);
}
template <typename T>
__device__ __forceinline__ const T *stage_x(const Smem<T> &s, const Pipe &p, int stage, int half = 0)
{
    return reinterpret_cast<const T *>(s.xs + size_t(stage) * p.x_bytes + (half ? p.x_bytes / 2 : 0));
}

// Consumer: release a stage once this warp is done reading it.
__device__ __forceinline__ void release(uint64_t *empty, int lane)
{
    __syncwarp();
    if (lane == 0) h2p::mbar_arrive(empty);
}

// Consumer accumulator: out[o] = sum_j tile[j*ld + o] * x[v*xld + j] over the tiles of one
// output. The CONS consumer threads (128, or 256 for the FP64 single-vector stream) are split
// into `lanes` output lanes x G column groups (both powers of two). With ld a multiple of VEC
// (16 bytes of T) each lane owns VEC consecutive outputs and reads them with one 16-byte
// shared-memory load per column; otherwise it owns one output (scalar path). Column group g
// takes j = g, g+G, ...; the groups are summed in a fixed order, so the result is
// deterministic.
template <typename T, int NVMAX, int CONS = kConsumers>
struct Acc {
    static_assert(CONS == kConsumers || (CONS == 2 * kConsumers && sizeof(T) == 8),
                  "256 consumers: FP64 only (the group-exchange buffer holds (G - 1) x 64 doubles)");
    static constexpr int VEC = 16 / int(sizeof(T));
    T a[NVMAX][VEC];
    int per, shift, g, G, o0, Rp;

    __device__ __forceinline__ void setup(int R, int ld, int tid)
    {
        Rp = rpad(R);
        per = (ld % VEC == 0) ? VEC : 1;
        const int lanes = Rp / per;
        shift = __ffs(lanes) - 1;
        g = tid >> shift;
        G = CONS >> shift;
        o0 = (tid & (lanes - 1)) * per;
    }
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int v = 0; v < NVMAX; ++v)
#pragma unroll
            for (int e = 0; e < VEC; ++e) a[v][e] = T(0);
    }
    // Square tiles with RC rows = columns = leading dimension, all shapes known at compile
    // time: fully unrolled, constant offsets (the common case: rank 64 with leaf size 64).
    template <int RC>
    __device__ __forceinline__ void gemv_fixed(const T *__restrict__ tile, const T *__restrict__ x, int xld, int nv)
    {
        using VT = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
        constexpr int LANES = rpad(RC) / VEC, GG = CONS / LANES, ITER = RC / GG;
        const T *tb = tile + g * RC + o0;
        const T *xb = x + g;
#pragma unroll
        for (int i = 0; i < ITER; ++i) {
            T t[VEC];
            *reinterpret_cast<VT *>(t) = *reinterpret_cast<const VT *>(tb + i * GG * RC);
#pragma unroll
            for (int v = 0; v < NVMAX; ++v)
                if (v < nv) {
                    const T xv = xb[v * xld + i * GG];
#pragma unroll
                    for (int e = 0; e < VEC; ++e) a[v][e] += t[e] * xv;
                }
        }
    }
    __device__ __forceinline__ void gemv(const T *__restrict__ tile, int ld, int R, int C, const T *__restrict__ x,
                                         int xld, int nv)
    {
        if (o0 >= R) return;
        if (R == 64 && C == 64 && ld == 64 && per == VEC) {
            gemv_fixed<64>(tile, x, xld, nv);
            return;
        }
        if (per == VEC) {
            using VT = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
#pragma unroll 4
            for (int j = g; j < C; j += G) {
                T t[VEC];
                *reinterpret_cast<VT *>(t) = *reinterpret_cast<const VT *>(tile + j * ld + o0);
#pragma unroll
                for (int v = 0; v < NVMAX; ++v)
                    if (v < nv) {
                        const T xv = x[v * xld + j];
#pragma unroll
                        for (int e = 0; e < VEC; ++e) a[v][e] += t[e] * xv;
                    }
            }
        } else {
#pragma unroll 4
            for (int j = g; j < C; j += G) {
                const T t = tile[j * ld + o0];
#pragma unroll
                for (int v = 0; v < NVMAX; ++v)
                    if (v < nv) a[v][0] += t * x[v * xld + j];
            }
        }
    }
    // Sum the column groups; true for the threads (g == 0, o0 < R) holding final values.
    __device__ __forceinline__ bool reduce(int R, int nv, T *red)
    {
        if (G > 1) {
            if (g > 0 && o0 < R) {
#pragma unroll
                for (int v = 0; v < NVMAX; ++v)
#pragma unroll
                    for (int e = 0; e < VEC; ++e)
                        if (v < nv && e < per) red[((g - 1) * NVMAX + v) * Rp + o0 + e] = a[v][e];
            }
            h2p::consumer_sync(CONS);
            if (g == 0 && o0 < R)
                for (int gg = 1; gg < G; ++gg)
#pragma unroll
                    for (int v = 0; v < NVMAX; ++v)
#pragma unroll
                        for (int e = 0; e < VEC; ++e)
                            if (v < nv && e < per) a[v][e] += red[((gg - 1) * NVMAX + v) * Rp + o0 + e];
        }
        return g == 0 && o0 < R;
    }
    // Store the held outputs o0 .. o0+per-1 (< R) of every vector v < nv at dst[v*ld + o].
    __device__ __forceinline__ void store(T *dst, int ld, int nv, int R) const
    {
#pragma unroll
        for (int v = 0; v < NVMAX; ++v)
#pragma unroll
            for (int e = 0; e < VEC; ++e)
                if (v < nv && e < per && o0 + e < R) dst[v * ld + o0 + e] = a[v][e];
    }
    __device__ __forceinline__ void add(const T *src, int ld, int nv, int R)
    {
#pragma unroll
        for (int v = 0; v < NVMAX; ++v)
#pragma unroll
            for (int e = 0; e < VEC; ++e)
                if (v < nv && e < per && o0 + e < R) a[v][e] += src[v * ld + o0 + e];
    }
    // Leaf epilogue: user-order rows of the held outputs (fetched before the tile arrives),
    // then Y[v*n + row] = alpha y + beta Y for the threads holding final values.
    int64_t u[VEC];
    __device__ __forceinline__ void fetch_rows(const int32_t *perm, int r0, int R)
    {
#pragma unroll
        for (int e = 0; e < VEC; ++e) u[e] = (g == 0 && e < per && o0 + e < R) ? perm[r0 + o0 + e] : 0;
    }
    __device__ __forceinline__ void write_out(T *Y, int64_t n, T alpha, T beta, int nv, int R) const
    {
#pragma unroll
        for (int e = 0; e < VEC; ++e)
            if (e < per && o0 + e < R) {
#pragma unroll
                for (int v = 0; v < NVMAX; ++v)
                    if (v < nv) {
                        T *dst = Y + int64_t(v) * n + u[e];
                        const T y = a[v][e];
                        *dst = (beta == T(0)) ? alpha * y : alpha * y + beta * *dst;
                    }
            }
    }
};

// Wide accumulator for passes of NV >= 8 vectors and tiles of at most 64 outputs: thread
// (og, vg) = (tid % 16, tid / 16) owns outputs o0 .. o0+3 (o0 = 4 og) of vectors
// v0 .. v0+VT-1 (v0 = VT vg, VT = NV / 8), a 4 x VT register block of the 64 x NV result.
// Each column step j reads four tile entries and VT vector entries; with 16-byte aligned
// rows four steps are read at once (16-byte loads along j for the vectors), so every loaded
// value feeds 4 or VT fused multiply-adds. Each thread sums its columns in ascending order;
// there is no cross-thread reduction, and the result is deterministic.
template <typename T, int NV>
struct AccW {
    static constexpr int VT = NV / 8;
    static constexpr int VEC = 4;
    static_assert(NV % 8 == 0 && NV >= 8, "wide accumulator: NV is a multiple of 8");
    T a[VT][4];
    int o0, v0;
    int64_t u[4];

    __device__ __forceinline__ void setup(int /*R*/, int /*ld*/, int tid)
    {
        o0 = (tid & 15) * 4;
        v0 = (tid >> 4) * VT;
    }
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int v = 0; v < VT; ++v)
#pragma unroll
            for (int e = 0; e < 4; ++e) a[v][e] = T(0);
    }
    __device__ static __forceinline__ void load4(T (&d)[4], const T *p)
    {
        if constexpr (sizeof(T) == 4) {
            *reinterpret_cast<float4 *>(d) = *reinterpret_cast<const float4 *>(p);
        } else {
            *reinterpret_cast<double2 *>(d) = *reinterpret_cast<const double2 *>(p);
            *reinterpret_cast<double2 *>(d + 2) = *reinterpret_cast<const double2 *>(p + 2);
        }
    }
    __device__ static __forceinline__ void store4(T *p, const T (&d)[4])
    {
        if constexpr (sizeof(T) == 4) {
            *reinterpret_cast<float4 *>(p) = *reinterpret_cast<const float4 *>(d);
        } else {
            *reinterpret_cast<double2 *>(p) = *reinterpret_cast<const double2 *>(d);
            *reinterpret_cast<double2 *>(p + 2) = *reinterpret_cast<const double2 *>(d + 2);
        }
    }
    // Columns j0 .. j0+3 with 16-byte aligned tile rows and vector segments.
    __device__ __forceinline__ void step4(const T *__restrict__ tb, int ld, const T *__restrict__ xb, int xld)
    {
        T xv[VT][4];
#pragma unroll
        for (int v = 0; v < VT; ++v) load4(xv[v], xb + v * xld);
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            T t[4];
            load4(t, tb + jj * ld);
#pragma unroll
            for (int v = 0; v < VT; ++v)
#pragma unroll
                for (int e = 0; e < 4; ++e) a[v][e] += t[e] * xv[v][jj];
        }
    }
    // out[o][v] += sum_{j < C} tile[j*ld + o] * x[v*xld + j] for o < R, v < nv.
    __device__ __forceinline__ void gemv(const T *__restrict__ tile, int ld, int R, int C, const T *__restrict__ x,
                                         int xld, int nv)
    {
        if (o0 >= R || v0 >= nv) return;
        const T *tb = tile + o0;
        const T *xb = x + v0 * xld;
        if (ld == 64 && xld == 64 && C == 64) {  // the common square tile: constant offsets
#pragma unroll
            for (int j = 0; j < 64; j += 4) step4(tb + j * 64, 64, xb + j, 64);
            return;
        }
        // every tile is zero-padded up to its leading dimension, so a group of four outputs
        // that straddles R reads zeros beyond it (and the stores mask them)
        if ((ld & 3) == 0 && (xld & 3) == 0 && o0 + 4 <= ld) {
            int j = 0;
#pragma unroll 2
            for (; j + 4 <= C; j += 4) step4(tb + j * ld, ld, xb + j, xld);
            for (; j < C; ++j) {
                T t[4];
                load4(t, tb + j * ld);
#pragma unroll
                for (int v = 0; v < VT; ++v) {
                    const T xs = xb[v * xld + j];
#pragma unroll
                    for (int e = 0; e < 4; ++e) a[v][e] += t[e] * xs;
                }
            }
            return;
        }
        for (int j = 0; j < C; ++j) {  // unaligned rows or a ragged last output group
            T t[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) t[e] = o0 + e < R ? tb[j * ld + e] : T(0);
#pragma unroll
            for (int v = 0; v < VT; ++v) {
                const T xs = xb[v * xld + j];
#pragma unroll
                for (int e = 0; e < 4; ++e) a[v][e] += t[e] * xs;
            }
        }
    }
    __device__ __forceinline__ bool reduce(int R, int nv, T * /*red*/) const { return o0 < R && v0 < nv; }
    __device__ __forceinline__ void store(T *dst, int ld, int nv, int R) const
    {
        const bool vec = (ld & 3) == 0 && o0 + 4 <= R;
#pragma unroll
        for (int v = 0; v < VT; ++v) {
            if (v0 + v >= nv) break;
            T *d = dst + (v0 + v) * ld + o0;
            if (vec) {
                store4(d, a[v]);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (o0 + e < R) d[e] = a[v][e];
            }
        }
    }
    __device__ __forceinline__ void add(const T *src, int ld, int nv, int R)
    {
        const bool vec = (ld & 3) == 0 && o0 + 4 <= R;
#pragma unroll
        for (int v = 0; v < VT; ++v) {
            if (v0 + v >= nv) break;
            const T *p = src + (v0 + v) * ld + o0;
            T s[4];
            if (vec) {
                load4(s, p);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) s[e] = o0 + e < R ? p[e] : T(0);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) a[v][e] += s[e];
        }
    }
    __device__ __forceinline__ void fetch_rows(const int32_t *perm, int r0, int R)
    {
#pragma unroll
        for (int e = 0; e < 4; ++e) u[e] = o0 + e < R ? perm[r0 + o0 + e] : 0;
    }
    // Leaf result rows in user order into the row-major buffer: yr[u*ldr + v] = y (the
    // epilogue alpha y + beta Y follows in k_rows_out). VT consecutive vectors of a row are
    // one 16-byte store when VT = 4.
    __device__ __forceinline__ void write_rows(T *yr, int ldr, int nv, int R) const
    {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (o0 + e >= R) continue;
            T *d = yr + u[e] * ldr + v0;
            if (VT == 4 && v0 + 4 <= nv && (ldr & 3) == 0) {
                const T t[4] = {a[0][e], a[VT > 1 ? 1 : 0][e], a[VT > 2 ? 2 : 0][e], a[VT > 3 ? 3 : 0][e]};
                store4(d, t);
            } else {
#pragma unroll
                for (int v = 0; v < VT; ++v)
                    if (v0 + v < nv) d[v] = a[v][e];
            }
        }
    }
    // Split-BF16 B-operand tile of the held block (rows = vectors v < np, columns = outputs):
    // hi = bf16(a), lo = bf16(a - hi), zero for v >= nv or output >= R. Four consecutive
    // outputs are 8 contiguous bytes of one swizzled 16-byte chunk.
    __device__ __forceinline__ void store_tile(unsigned char *tile, int np, int nv, int R) const
    {
        if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int v = 0; v < VT; ++v) {
                const int r = v0 + v;
                if (r >= np) break;
                __nv_bfloat16 hi[4], lo[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float x = (r < nv && o0 + e < R) ? a[v][e] : 0.f;
                    hi[e] = __float2bfloat16_rn(x);
                    lo[e] = __float2bfloat16_rn(x - __bfloat162float(hi[e]));
                }
                const uint32_t off = sw128(r, o0);
                *reinterpret_cast<uint2 *>(tile + off) = *reinterpret_cast<const uint2 *>(hi);
                *reinterpret_cast<uint2 *>(tile + np * 128 + off) = *reinterpret_cast<const uint2 *>(lo);
            }
        }
    }
    __device__ __forceinline__ void write_out(T *Y, int64_t n, T alpha, T beta, int nv, int R) const
    {
#pragma unroll
        for (int v = 0; v < VT; ++v)
            if (v0 + v < nv)
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (o0 + e < R) {
                        T *dst = Y + int64_t(v0 + v) * n + u[e];
                        const T y = a[v][e];
                        *dst = (beta == T(0)) ? alpha * y : alpha * y + beta * *dst;
                    }
    }
};

template <typename T, int NVMAX>
using AccOf = typename std::conditional<(NVMAX >= kWideMin), AccW<T, NVMAX>, Acc<T, NVMAX>>::type;

// Wide accumulator of the block streams (k_stream, k_stream_batch): every thread holds an
// OUT-output x 4-vector register block, and the 128 consumer threads split the columns into
// S = 128 / ((64 / OUT) (NV / 4)) slices of four-column steps (slice ks takes the steps
// ks, ks + S, ...). With 8 and 16 vectors (OUT = 4; S = 4, 2) every loaded tile value feeds
// 4 FMAs where AccW's 4 x NV/8 block feeds 1 or 2. At the end of a row the slices are summed
// through shared memory in a fixed order (slice 0 adds 1 .. S-1) and slice 0 stores, so the
// result stays deterministic.
template <typename T, int NV, int OUT>
struct AccWK {
    static constexpr int VT = 4;
    static constexpr int NVG = NV / 4;        // vector groups
    static constexpr int OG = 64 / OUT;       // output groups
    static constexpr int S = kConsumers / (OG * NVG);  // column slices
    static constexpr int QS = 64 / (OUT / 4);  // distance between a thread's output quads
    static_assert(S >= 2 && OG * NVG * S == kConsumers, "split-column wide accumulator: 8, 16 or 32 vectors");
    // outputs of element e: quad e / 4 at o0 + QS * (e / 4) (16-byte loads of neighbouring
    // threads stay adjacent in shared memory: no bank conflicts)
    T a[VT][OUT];
    int o0, v0, ks;

    __device__ __forceinline__ static int off(int e) { return (e & 3) + QS * (e >> 2); }
    __device__ __forceinline__ void setup(int /*R*/, int /*ld*/, int tid)
    {
        o0 = (tid % OG) * 4;
        const int rest = tid / OG;
        v0 = (rest % NVG) * VT;
        ks = rest / NVG;
    }
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int v = 0; v < VT; ++v)
#pragma unroll
            for (int e = 0; e < OUT; ++e) a[v][e] = T(0);
    }
    __device__ __forceinline__ void step4(const T *__restrict__ tb, int ld, const T *__restrict__ xb, int xld)
    {
        T xv[VT][4];
#pragma unroll
        for (int v = 0; v < VT; ++v) AccW<T, 32>::load4(xv[v], xb + v * xld);
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            T t[OUT];
#pragma unroll
            for (int h = 0; h < OUT / 4; ++h)
                AccW<T, 32>::load4(*reinterpret_cast<T(*)[4]>(t + 4 * h), tb + jj * ld + QS * h);
#pragma unroll
            for (int v = 0; v < VT; ++v)
#pragma unroll
                for (int e = 0; e < OUT; ++e) a[v][e] += t[e] * xv[v][jj];
        }
    }
    __device__ __forceinline__ void column(const T *__restrict__ tb, int ld, int R, const T *__restrict__ xb, int xld,
                                           int j)
    {
        T t[OUT];
#pragma unroll
        for (int e = 0; e < OUT; ++e) t[e] = o0 + off(e) < R ? tb[j * ld + off(e)] : T(0);
#pragma unroll
        for (int v = 0; v < VT; ++v) {
            const T xs = xb[v * xld + j];
#pragma unroll
            for (int e = 0; e < OUT; ++e) a[v][e] += t[e] * xs;
        }
    }
    // out[o][v] += sum over this slice's columns j < C of tile[j*ld + o] * x[v*xld + j].
    __device__ __forceinline__ void gemv(const T *__restrict__ tile, int ld, int R, int C, const T *__restrict__ x,
                                         int xld, int nv)
    {
        if (o0 >= R || v0 >= nv) return;
        const T *tb = tile + o0;
        const T *xb = x + v0 * xld;
        if (ld == 64 && xld == 64 && C == 64) {
#pragma unroll
            for (int j = 4 * ks; j < 64; j += 4 * S) step4(tb + j * 64, 64, xb + j, 64);
            return;
        }
        // zero-padded, 16-byte aligned rows whose padding covers this thread's outputs
        if ((ld & 3) == 0 && (xld & 3) == 0 && o0 + off(OUT - 1) < ld) {
            for (int j = 4 * ks; j + 4 <= C; j += 4 * S) step4(tb + j * ld, ld, xb + j, xld);
            const int jt = C & ~3;  // the partial last step belongs to slice (C / 4) % S
            if (jt < C && (C >> 2) % S == ks)
                for (int j = jt; j < C; ++j) column(tb, ld, R, xb, xld, j);
            return;
        }
        for (int q = ks; 4 * q < C; q += S)  // unaligned rows or outputs past the padding
            for (int j = 4 * q; j < C && j < 4 * q + 4; ++j) column(tb, ld, R, xb, xld, j);
    }
    // Sum the slices (every consumer thread calls this; it holds a consumer barrier).
    __device__ __forceinline__ bool reduce(int R, int nv, T *red)
    {
        const bool mine = o0 < R && v0 < nv;
        if (ks > 0 && mine)
#pragma unroll
            for (int v = 0; v < VT; ++v)
#pragma unroll
                for (int e = 0; e < OUT; ++e) red[((ks - 1) * 64 + o0 + off(e)) * NV + v0 + v] = a[v][e];
        h2p::consumer_sync(kConsumers);
        if (ks == 0 && mine)
            for (int sl = 1; sl < S; ++sl)
#pragma unroll
                for (int v = 0; v < VT; ++v)
#pragma unroll
                    for (int e = 0; e < OUT; ++e) a[v][e] += red[((sl - 1) * 64 + o0 + off(e)) * NV + v0 + v];
        return ks == 0 && mine;
    }
    __device__ __forceinline__ void store(T *dst, int ld, int nv, int R) const
    {
#pragma unroll
        for (int v = 0; v < VT; ++v) {
            if (v0 + v >= nv) break;
            T *d = dst + (v0 + v) * ld + o0;
#pragma unroll
            for (int h = 0; h < OUT / 4; ++h) {
                if ((ld & 3) == 0 && o0 + QS * h + 4 <= R) {
                    AccW<T, 32>::store4(d + QS * h, *reinterpret_cast<const T(*)[4]>(a[v] + 4 * h));
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (o0 + QS * h + e < R) d[QS * h + e] = a[v][4 * h + e];
                }
            }
        }
    }
};

// Accumulator of the block streams (k_stream, k_stream_batch): the split-column form for 8
// and 16 vectors; at 32 vectors AccW's unsplit 4 x 4 block (the split 8 x 4 form measured
// 41.8 against 38.7 ms for the 2^21-point FP32 product: its second output quad doubles the
// tile loads per thread without raising the FMAs per vector load).
template <typename T, int NVMAX>
using AccStreamOf =
    typename std::conditional<(NVMAX >= kWideMin && NVMAX < 32), AccWK<T, NVMAX, 4>, AccOf<T, NVMAX>>::type;

// ------------------------------------------------------------------ gather

// xt[leaf][v][i] = X[v*n + perm[leaf_lo[leaf] + i]]: one CTA per leaf (grid-stride). Also
// resets the scheduling tickets and the warp sweeps' node flags of this product. With
// vec.xtb (tensor-core passes) it also writes each leaf's split-BF16 tile.
template <typename T>
__global__ void k_gather(Op<T> op, Vec<T> vec)
{
    if (blockIdx.x == 0 && threadIdx.x < kTickets) vec.tickets[threadIdx.x] = 0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < vec.nflags; i += int64_t(gridDim.x) * blockDim.x)
        vec.flags[i] = 0;
    for (int64_t leaf = blockIdx.x; leaf < op.nleaves; leaf += gridDim.x) {
        const int r0 = op.leaf_lo[leaf], R = op.leaf_lo[leaf + 1] - r0;
        if (vec.xtb == nullptr) {
            for (int e = threadIdx.x; e < R * vec.nv; e += blockDim.x) {
                const int i = e % R, v = e / R;
                vec.xt[(leaf * vec.vs + v) * op.mp + i] = vec.X[int64_t(v) * op.n + op.perm[r0 + i]];
            }
        } else if constexpr (sizeof(T) == 4) {
            unsigned char *tile = vec.xtb + leaf * vec_tile_bytes(vec.np);
            for (int e = threadIdx.x; e < vec.np * 64; e += blockDim.x) {
                const int i = e % 64, v = e / 64;
                float x = 0.f;
                if (i < R && v < vec.nv) {
                    x = vec.X[int64_t(v) * op.n + op.perm[r0 + i]];
                    vec.xt[(leaf * vec.vs + v) * op.mp + i] = x;
                }
                const __nv_bfloat16 hi = __float2bfloat16_rn(x);
                const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
                const uint32_t off = sw128(v, i);
                *reinterpret_cast<__nv_bfloat16 *>(tile + off) = hi;
                *reinterpret_cast<__nv_bfloat16 *>(tile + vec.np * 128 + off) = lo;
            }
        }
    }
}

// The gather of wide passes (leaves of at most 64 points, at most 32 vectors): each permuted
// point's nv values are one row of the row-major copy vec.xr (coalesced reads), staged in
// shared memory and written per vector, with the split-BF16 tile when vec.xtb is set. Also
// resets the scheduling tickets.
template <typename T>
__global__ void k_gather_rows(Op<T> op, Vec<T> vec)
{
    __shared__ T rows[64 * 33];
    if (blockIdx.x == 0 && threadIdx.x < kTickets) vec.tickets[threadIdx.x] = 0;
    for (int64_t leaf = blockIdx.x; leaf < op.nleaves; leaf += gridDim.x) {
        const int r0 = op.leaf_lo[leaf], R = op.leaf_lo[leaf + 1] - r0;
        for (int e = threadIdx.x; e < R * vec.nv; e += blockDim.x) {
            const int i = e / vec.nv, v = e % vec.nv;
            rows[i * 33 + v] = vec.xr[int64_t(op.perm[r0 + i]) * vec.ldr + v];
        }
        __syncthreads();
        for (int e = threadIdx.x; e < R * vec.nv; e += blockDim.x) {
            const int v = e / R, i = e % R;
            vec.xt[(leaf * vec.vs + v) * op.mp + i] = rows[i * 33 + v];
        }
        if constexpr (sizeof(T) == 4) {
            if (vec.xtb != nullptr) {
                unsigned char *tile = vec.xtb + leaf * vec_tile_bytes(vec.np);
                for (int e = threadIdx.x; e < vec.np * 64; e += blockDim.x) {
                    const int i = e % 64, v = e / 64;
                    const float x = (i < R && v < vec.nv) ? rows[i * 33 + v] : 0.f;
                    const __nv_bfloat16 hi = __float2bfloat16_rn(x);
                    const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
                    const uint32_t off = sw128(v, i);
                    *reinterpret_cast<__nv_bfloat16 *>(tile + off) = hi;
                    *reinterpret_cast<__nv_bfloat16 *>(tile + vec.np * 128 + off) = lo;
                }
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ row-major staging

// xr[u*ldr + v] = X[v*n + u] for u < n, v < nv: 32 x 32 tiles through shared memory, so
// that both sides are read and written along their contiguous index. Block 32 x 8.
template <typename T>
__global__ void k_rows_in(const T *__restrict__ X, int64_t n, int nv, T *__restrict__ xr, int ldr)
{
    __shared__ T t[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t u0 = int64_t(blockIdx.x) * 32;
    const int v0 = blockIdx.y * 32;
    for (int j = ty; j < 32; j += 8) {
        const int64_t u = u0 + tx;
        const int v = v0 + j;
        if (u < n && v < nv) t[j][tx] = X[int64_t(v) * n + u];
    }
    __syncthreads();
    for (int j = ty; j < 32; j += 8) {
        const int64_t u = u0 + j;
        const int v = v0 + tx;
        if (u < n && v < nv) xr[u * ldr + v] = t[tx][j];
    }
}

// Epilogue of a wide pass: Y[v*n + u] = alpha yr[u*ldr + v] + beta Y[v*n + u] (Y is not read
// when beta = 0), through the same 32 x 32 shared-memory tiles.
template <typename T>
__global__ void k_rows_out(const T *__restrict__ yr, int ldr, T *__restrict__ Y, int64_t n, int nv, T alpha, T beta)
{
    __shared__ T t[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t u0 = int64_t(blockIdx.x) * 32;
    const int v0 = blockIdx.y * 32;
    for (int j = ty; j < 32; j += 8) {
        const int64_t u = u0 + j;
        const int v = v0 + tx;
        if (u < n && v < nv) t[j][tx] = yr[u * ldr + v];
    }
    __syncthreads();
    for (int j = ty; j < 32; j += 8) {
        const int64_t u = u0 + tx;
        const int v = v0 + j;
        if (u < n && v < nv) {
            T *dst = Y + int64_t(v) * n + u;
            const T y = t[tx][j];
            *dst = (beta == T(0)) ? alpha * y : alpha * y + beta * *dst;
        }
    }
}

// ------------------------------------------------------------------ subtree upsweep

// Upsweep of subtrees rooted at level Lr with depth L (inputs on level Lr+L). With leaf
// input (Lr+L = q) the inputs are the leaf projections xhat^q_t = U_t^T x_t; otherwise they
// are the coefficient vectors of level Lr+L computed by an earlier launch. Writes xhat for
// levels Lr .. Lr+L (the input level only with leaf input).
//
// The work of one subtree st is split into its producer part (the tiles in the order the
// consumers use them) and its consumer part, so that one kernel (k_up_sub) walks the
// subtrees of one operator and another (k_up_batch) a merged list over many operators.

// One subtree's tiles into the ring; false once the pipeline aborted.
template <typename T, int NVMAX>
__device__ bool up_sub_produce(const Op<T> &op, const Vec<T> &vec, Smem<T> &s, const Pipe &pp, Ring &ring, int Lr,
                               int L, int64_t st, int leaf_input)
{
    const int k = op.k, kx = op.kx, mp = op.mp, nv = vec.nv, vs = vec.vs;
    const int Lin = Lr + L;
    const uint32_t es = sizeof(T);
    bool ok = true;
    if (leaf_input) {
        const int64_t leaf0 = st << L;
        for (int j = 0; ok && j < (1 << L); ++j) {
            const int64_t leaf = leaf0 + j;
            ok = produce(s, pp, ring, op.U + leaf * mp * kx, mp * kx * es, vec.xt + leaf * mp * vs, mp * nv * es,
                         nullptr, 0, nullptr, vec.err);
        }
    }
    for (int lev = Lin; ok && lev > Lr; --lev) {
        const int64_t cnt = int64_t(1) << (lev - Lr);
        const int64_t c0 = (int64_t(1) << lev) + st * cnt;
        // an input level from an earlier launch travels with its transfer tiles
        const bool with_x = !leaf_input && lev == Lin;
        for (int64_t c = c0; ok && c < c0 + cnt; ++c)
            ok = produce(s, pp, ring, op.E + c * k * kx, k * kx * es, with_x ? vec.xh + c * kx * vs : nullptr,
                         with_x ? kx * nv * es : 0, nullptr, 0, nullptr, vec.err);
    }
    return ok;
}

// One subtree's products (consumer warps); false once the pipeline aborted.
template <typename T, int NVMAX>
__device__ bool up_sub_consume(const Op<T> &op, const Vec<T> &vec, Smem<T> &s, const Pipe &pp, Ring &ring,
                               AccOf<T, NVMAX> &acc, int Lr, int L, int64_t st, int leaf_input)
{
    const int lane = threadIdx.x % 32;
    const int k = op.k, kx = op.kx, mp = op.mp, nv = vec.nv, vs = vec.vs;
    const int Lin = Lr + L;
    const int wstride = kx * NVMAX;
    if (leaf_input) {
        // leaf projections into local slots 2^L + j
        const int64_t leaf0 = st << L;
        for (int j = 0; j < (1 << L); ++j) {
            const int64_t leaf = leaf0 + j;
            const int R = op.leaf_lo[leaf + 1] - op.leaf_lo[leaf];
            acc.zero();
            if (!h2p::mbar_wait(&s.full[ring.stage], ring.phase, s.abort_flag, vec.err)) return false;
            acc.gemv(stage_tile(s, pp, ring.stage), kx, k, R, stage_x(s, pp, ring.stage), mp, nv);
            release(&s.empty[ring.stage], lane);
            ring.next();
            if (acc.reduce(k, nv, s.red)) {
                acc.store(s.sub + ((1 << L) + j) * wstride, kx, nv, k);
                acc.store(vec.xh + (op.first_leaf + leaf) * kx * vs, kx, nv, k);
            }
            if constexpr (NVMAX >= kWideMin)
                if (vec.xb) acc.store_tile(vec.xb + (op.first_leaf + leaf) * vec_tile_bytes(vec.np), vec.np, nv, k);
            h2p::consumer_sync(kConsumers);
        }
    }
    // transfers, level by level (the input level of a launch without leaf input arrives in
    // the stages, next to its transfer tiles)
    for (int lev = Lin; lev > Lr; --lev) {
        const int rel = lev - Lr;
        const int64_t cnt = int64_t(1) << rel;
        const bool staged_x = !leaf_input && lev == Lin;
        for (int64_t pi = 0; pi < cnt / 2; ++pi) {
            acc.zero();
            for (int c = 0; c < 2; ++c) {
                const int child_slot = (1 << rel) + int(2 * pi + c);
                if (!h2p::mbar_wait(&s.full[ring.stage], ring.phase, s.abort_flag, vec.err)) return false;
                const T *xc = staged_x ? stage_x(s, pp, ring.stage) : s.sub + child_slot * wstride;
                acc.gemv(stage_tile(s, pp, ring.stage), kx, k, k, xc, kx, nv);
                release(&s.empty[ring.stage], lane);
                ring.next();
            }
            const int64_t par = (int64_t(1) << (lev - 1)) + st * (cnt / 2) + pi;
            if (acc.reduce(k, nv, s.red)) {
                const int pslot = (1 << (rel - 1)) + int(pi);
                acc.store(s.sub + pslot * wstride, kx, nv, k);
                acc.store(vec.xh + par * kx * vs, kx, nv, k);
            }
            if constexpr (NVMAX >= kWideMin)
                if (vec.xb) acc.store_tile(vec.xb + par * vec_tile_bytes(vec.np), vec.np, nv, k);
            h2p::consumer_sync(kConsumers);
        }
    }
    return true;
}

template <typename T, int NVMAX>
__global__ void __launch_bounds__(kThreads)
    k_up_sub(Op<T> op, Vec<T> vec, Pipe pp, int Lr, int L, int64_t nsub, int leaf_input)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem<T> s = carve<T, NVMAX>(smem_raw, pp, 2 << L, op.kx, false);
    init_pipe(s, pp);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    Ring ring(pp.ns);
    if (warp == 4) {  // producer: fixed-size tiles, so no per-leaf metadata is needed
        if (lane == 0) {
            bool ok = true;
            for (int64_t st = blockIdx.x; ok && st < nsub; st += gridDim.x)
                ok = up_sub_produce<T, NVMAX>(op, vec, s, pp, ring, Lr, L, st, leaf_input);
            drain_on_abort(s, ring);
        }
        return;
    }
    AccOf<T, NVMAX> acc;
    acc.setup(op.k, op.kx, threadIdx.x);
    for (int64_t st = blockIdx.x; st < nsub; st += gridDim.x)
        if (!up_sub_consume<T, NVMAX>(op, vec, s, pp, ring, acc, Lr, L, st, leaf_input)) return;
}

// A sweep step of one operator inside a merged launch: its subtrees are the global work
// items first .. first + nsub - 1.
template <typename T>
struct SweepTask {
    Op<T> op;
    Vec<T> vec;
    int Lr, L, flag;  // flag: leaf input (upsweep) or leaf output (downsweep)
    int64_t first, nsub;
};

// The task holding global item g (tasks ordered by first, every nsub >= 1).
template <typename T>
__device__ inline int sweep_task_of(const SweepTask<T> *__restrict__ tasks, int ntasks, int64_t g)
{
    int lo = 0, hi = ntasks - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (tasks[mid].first <= g)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Merged upsweep step: every task's subtrees in one persistent launch. Shared memory is
// carved for the largest subtree buffer of the tasks (sub_kx = the most subtree slots x kx
// over the tasks) and the pipe's slots for the largest tiles.
template <typename T, int NVMAX>
__global__ void __launch_bounds__(kThreads)
    k_up_batch(const SweepTask<T> *__restrict__ tasks, int ntasks, int64_t total, Pipe pp, int sub_kx)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem<T> s = carve<T, NVMAX>(smem_raw, pp, 1, sub_kx, false);
    init_pipe(s, pp);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    Ring ring(pp.ns);
    if (warp == 4) {
        if (lane == 0) {
            bool ok = true;
            for (int64_t g = blockIdx.x; ok && g < total; g += gridDim.x) {
                const SweepTask<T> &t = tasks[sweep_task_of(tasks, ntasks, g)];
                ok = up_sub_produce<T, NVMAX>(t.op, t.vec, s, pp, ring, t.Lr, t.L, g - t.first, t.flag);
            }
            drain_on_abort(s, ring);
        }
        return;
    }
    AccOf<T, NVMAX> acc;
    for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
        const SweepTask<T> &t = tasks[sweep_task_of(tasks, ntasks, g)];
        acc.setup(t.op.k, t.op.kx, threadIdx.x);
        if (!up_sub_consume<T, NVMAX>(t.op, t.vec, s, pp, ring, acc, t.Lr, t.L, g - t.first, t.flag)) return;
    }
}

// ------------------------------------------------------------------ block-row stream

// chunks[c] = (first descriptor << 16) | descriptor count: whole rows, in order.
// CONS consumer threads (warps 0 .. CONS/32 - 1) and one producer warp after them. The FP64
// single-vector stream runs 256 consumers: the FP64 pipe is the bound there, and eight
// consumer warps per SM keep it busier than four (a 64 x 64 tile product from shared memory
// measured 1.19 against 1.03 Tflop/s per GPU).
template <typename T, int NVMAX, int CONS = kConsumers>
__global__ void __launch_bounds__(CONS + 32, 1)
    k_stream(Op<T> op, Vec<T> vec, Pipe pp, const StreamDesc *__restrict__ desc, const int64_t *__restrict__ chunks,
             int64_t nchunks, int ticket_index)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem<T> s = carve<T, NVMAX>(smem_raw, pp, 0, op.kx, true);
    init_pipe(s, pp, CONS);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int kx = op.kx, mp = op.mp, nv = vec.nv, vs = vec.vs;
    const uint32_t es = sizeof(T);
    Ring ring(pp.ns);

    if (warp == CONS / 32) {
        if (lane == 0) {
            int *ticket = vec.tickets + ticket_index;
            // a chunk's descriptors are bulk-copied into one of two shared-memory slots while
            // the previous chunk is being issued; tickets are fetched one chunk ahead
            auto fetch_desc = [&](int slot, int64_t rec) {
                const int64_t b0 = rec >> 16;
                const uint32_t bytes = uint32_t(rec & 0xffff) * uint32_t(sizeof(StreamDesc));
                h2p::fence_proxy_async_shared();
                h2p::mbar_arrive_expect_tx(&s.dbar[slot], bytes);
                h2p::bulk_g2s(s.dbuf + slot * kChunkDesc, desc + b0, bytes, &s.dbar[slot]);
            };
            int64_t tA = atomicAdd(ticket, 1);
            int64_t tB = atomicAdd(ticket, 1);
            int64_t recA = tA < nchunks ? chunks[tA] : 0;
            int slot = 0;
            uint32_t dphase = 0;  // bit per slot
            bool ok = true;
            if (tA < nchunks) fetch_desc(0, recA);
            while (ok && tA < nchunks) {
                const int64_t recB = tB < nchunks ? chunks[tB] : 0;
                const int64_t tC = atomicAdd(ticket, 1);
                ok = h2p::mbar_wait(&s.dbar[slot], dphase >> slot & 1u, s.abort_flag, vec.err);
                dphase ^= 1u << slot;
                const int cnt = int(recA & 0xffff);
                const int pre = cnt - 1 < 4 ? cnt - 1 : 4;
                for (int i = 0; ok && i < cnt; ++i) {
                    if (i == pre && tB < nchunks) fetch_desc(slot ^ 1, recB);
                    const StreamDesc d = s.dbuf[slot * kChunkDesc + i];
                    if (d.flags & kZero) {
                        ok = produce(s, pp, ring, nullptr, 0, nullptr, 0, nullptr, 0, &d, vec.err);
                    } else {
                        const bool dense = d.flags & kDense;
                        const uint32_t tb = (uint32_t(d.ld) * d.cols * es + 15u) & ~15u;
                        const T *x = dense ? vec.xt + int64_t(d.x_node) * mp * vs : vec.xh + int64_t(d.x_node) * kx * vs;
                        const uint32_t xb = (dense ? mp : kx) * nv * es;
                        ok = produce(s, pp, ring, op.vals + d.src, tb, x, xb, nullptr, 0, &d, vec.err);
                    }
                }
                slot ^= 1;
                tA = tB;
                recA = recB;
                tB = tC;
            }
            if (ok && h2p::mbar_wait(&s.empty[ring.stage], ring.phase ^ 1u, s.abort_flag, vec.err)) {
                s.desc[ring.stage].flags = kEnd;  // sentinel: completes the stage with no data
                h2p::mbar_arrive(&s.full[ring.stage]);
            }
            drain_on_abort(s, ring);
        }
        return;
    }

    const int tid = threadIdx.x;
    typename std::conditional<CONS == kConsumers, AccStreamOf<T, NVMAX>, Acc<T, NVMAX, CONS>>::type acc;
    bool fresh = true;
    for (;;) {
        if (!h2p::mbar_wait(&s.full[ring.stage], ring.phase, s.abort_flag, vec.err)) return;
        const StreamDesc d = s.desc[ring.stage];
        if (d.flags & kEnd) break;
        const bool dense = d.flags & kDense;
        const int xld = dense ? mp : kx;
        if (fresh) {
            acc.setup(d.rows, d.ld, tid);
            acc.zero();
            fresh = false;
        }
        if (!(d.flags & kZero))
            acc.gemv(stage_tile(s, pp, ring.stage), d.ld, d.rows, d.cols, stage_x(s, pp, ring.stage), xld, nv);
        release(&s.empty[ring.stage], lane);
        ring.next();
        if (d.flags & kLast) {
            if (acc.reduce(d.rows, nv, s.red)) {
                T *out = dense ? vec.yd + int64_t(d.out_node) * mp * vs : vec.yh + int64_t(d.out_node) * kx * vs;
                acc.store(out, xld, nv, d.rows);
            }
            h2p::consumer_sync(CONS);
            fresh = true;
        }
    }
}

// ------------------------------------------------------------------ subtree downsweep

// Downsweep of subtrees rooted at level Lr with depth L: yhat^l_c = E_c yhat^{l-1}_p + own_c
// for levels Lr .. Lr+L, where own_c is node c's coupling row (every row is defined: empty
// rows were written as zeros) and the parent total of a root at level Lr >= 1 comes from
// an earlier launch. With leaf output (Lr+L = q) it finishes with the leaf expansion
// y_t = U_t yhat^q_t, the dense partial result and Y[perm] = alpha y + beta Y; otherwise it
// writes the totals of level Lr+L over their coupling rows, for the next launch. As for the
// upsweep, one subtree's producer and consumer parts serve k_down_sub (one operator) and
// k_down_batch (a merged list).
//
// Each node's own coupling vector travels with its transfer tile in the second half of the
// stage's vector slot; the root's parent total in the first half.
template <typename T, int NVMAX>
__device__ bool down_sub_produce(const Op<T> &op, const Vec<T> &vec, Smem<T> &s, const Pipe &pp, Ring &ring,
                                 int Lr, int L, int64_t st, int leaf_output)
{
    const int k = op.k, kx = op.kx, mp = op.mp, nv = vec.nv, vs = vec.vs;
    const int Lo = Lr + L;
    const uint32_t es = sizeof(T);
    const uint32_t vb = kx * nv * es;  // bytes of one node's coefficient vector
    bool ok = true;
    const int64_t r = (int64_t(1) << Lr) + st;
    if (Lr >= 1)
        ok = produce(s, pp, ring, op.Et + r * k * kx, k * kx * es, vec.yh + (r / 2) * kx * vs, vb,
                     vec.yh + r * kx * vs, vb, nullptr, vec.err);
    else
        ok = produce(s, pp, ring, nullptr, 0, nullptr, 0, vec.yh + r * kx * vs, vb, nullptr, vec.err);
    for (int lev = Lr + 1; ok && lev <= Lo; ++lev) {
        const int64_t cnt = int64_t(1) << (lev - Lr);
        const int64_t c0 = (int64_t(1) << lev) + st * cnt;
        for (int64_t c = c0; ok && c < c0 + cnt; ++c)
            ok = produce(s, pp, ring, op.Et + c * k * kx, k * kx * es, nullptr, 0, vec.yh + c * kx * vs, vb, nullptr,
                         vec.err);
    }
    if (leaf_output) {
        const int64_t leaf0 = st << L;
        for (int j = 0; ok && j < (1 << L); ++j) {
            const int64_t leaf = leaf0 + j;
            ok = produce(s, pp, ring, op.Ut + leaf * kx * mp, k * mp * es, vec.yd + leaf * mp * vs, mp * nv * es,
                         nullptr, 0, nullptr, vec.err);
        }
    }
    return ok;
}

template <typename T, int NVMAX>
__device__ bool down_sub_consume(const Op<T> &op, const Vec<T> &vec, Smem<T> &s, const Pipe &pp, Ring &ring,
                                 AccOf<T, NVMAX> &acc, int Lr, int L, int64_t st, int leaf_output)
{
    const int lane = threadIdx.x % 32, tid = threadIdx.x;
    const int k = op.k, kx = op.kx, mp = op.mp, nv = vec.nv, vs = vec.vs;
    const int Lo = Lr + L;
    const int wstride = kx * NVMAX;
    // subtree root: E_r yhat_parent + own
    acc.setup(k, kx, tid);
    acc.zero();
    if (!h2p::mbar_wait(&s.full[ring.stage], ring.phase, s.abort_flag, vec.err)) return false;
    if (Lr >= 1) acc.gemv(stage_tile(s, pp, ring.stage), kx, k, k, stage_x(s, pp, ring.stage), kx, nv);
    if (acc.reduce(k, nv, s.red)) {
        acc.add(stage_x(s, pp, ring.stage, 1), kx, nv, k);
        acc.store(s.sub + 1 * wstride, kx, nv, k);
        if (L == 0 && !leaf_output) acc.store(vec.yh + ((int64_t(1) << Lr) + st) * kx * vs, kx, nv, k);
    }
    release(&s.empty[ring.stage], lane);
    ring.next();
    h2p::consumer_sync(kConsumers);
    for (int lev = Lr + 1; lev <= Lo; ++lev) {
        const int rel = lev - Lr;
        const int64_t cnt = int64_t(1) << rel;
        for (int64_t ci = 0; ci < cnt; ++ci) {
            const int slot = (1 << rel) + int(ci);
            acc.zero();
            if (!h2p::mbar_wait(&s.full[ring.stage], ring.phase, s.abort_flag, vec.err)) return false;
            acc.gemv(stage_tile(s, pp, ring.stage), kx, k, k, s.sub + (slot / 2) * wstride, kx, nv);
            if (acc.reduce(k, nv, s.red)) {
                acc.add(stage_x(s, pp, ring.stage, 1), kx, nv, k);
                acc.store(s.sub + slot * wstride, kx, nv, k);
                if (lev == Lo && !leaf_output)
                    acc.store(vec.yh + ((int64_t(1) << lev) + st * cnt + ci) * kx * vs, kx, nv, k);
            }
            release(&s.empty[ring.stage], lane);
            ring.next();
            h2p::consumer_sync(kConsumers);
        }
    }
    if (!leaf_output) return true;
    // leaves: y = U_t yhat_t + yd_t; Y[perm] = alpha y + beta Y
    const int64_t leaf0 = st << L;
    for (int j = 0; j < (1 << L); ++j) {
        const int64_t leaf = leaf0 + j;
        const int r0 = op.leaf_lo[leaf], R = op.leaf_lo[leaf + 1] - r0;
        acc.setup(R, mp, tid);
        acc.zero();
        acc.fetch_rows(op.perm, r0, R);  // output rows, fetched while the tile is in flight
        if (!h2p::mbar_wait(&s.full[ring.stage], ring.phase, s.abort_flag, vec.err)) return false;
        acc.gemv(stage_tile(s, pp, ring.stage), mp, R, k, s.sub + ((1 << L) + j) * wstride, kx, nv);
        if (acc.reduce(R, nv, s.red)) {
            acc.add(stage_x(s, pp, ring.stage), mp, nv, R);
            // narrow passes write Y directly (a runtime choice here slowed the nv = 1 leaf
            // epilogue measurably); wide passes may stage rows for k_rows_out
            if constexpr (NVMAX >= kWideMin) {
                if (vec.yr)
                    acc.write_rows(vec.yr, vec.ldr, nv, R);
                else
                    acc.write_out(vec.Y, op.n, vec.alpha, vec.beta, nv, R);
            } else {
                acc.write_out(vec.Y, op.n, vec.alpha, vec.beta, nv, R);
            }
        }
        release(&s.empty[ring.stage], lane);
        ring.next();
        h2p::consumer_sync(kConsumers);
    }
    return true;
}

template <typename T, int NVMAX>
__global__ void __launch_bounds__(kThreads)
    k_down_sub(Op<T> op, Vec<T> vec, Pipe pp, int Lr, int L, int64_t nsub, int leaf_output)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem<T> s = carve<T, NVMAX>(smem_raw, pp, 2 << L, op.kx, false);
    init_pipe(s, pp);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    Ring ring(pp.ns);
    if (warp == 4) {
        if (lane == 0) {
            bool ok = true;
            for (int64_t st = blockIdx.x; ok && st < nsub; st += gridDim.x)
                ok = down_sub_produce<T, NVMAX>(op, vec, s, pp, ring, Lr, L, st, leaf_output);
            drain_on_abort(s, ring);
        }
        return;
    }
    AccOf<T, NVMAX> acc;
    for (int64_t st = blockIdx.x; st < nsub; st += gridDim.x)
        if (!down_sub_consume<T, NVMAX>(op, vec, s, pp, ring, acc, Lr, L, st, leaf_output)) return;
}

// Merged downsweep step over the tasks' subtrees (see k_up_batch).
template <typename T, int NVMAX>
__global__ void __launch_bounds__(kThreads)
    k_down_batch(const SweepTask<T> *__restrict__ tasks, int ntasks, int64_t total, Pipe pp, int sub_kx)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem<T> s = carve<T, NVMAX>(smem_raw, pp, 1, sub_kx, false);
    init_pipe(s, pp);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    Ring ring(pp.ns);
    if (warp == 4) {
        if (lane == 0) {
            bool ok = true;
            for (int64_t g = blockIdx.x; ok && g < total; g += gridDim.x) {
                const SweepTask<T> &t = tasks[sweep_task_of(tasks, ntasks, g)];
                ok = down_sub_produce<T, NVMAX>(t.op, t.vec, s, pp, ring, t.Lr, t.L, g - t.first, t.flag);
            }
            drain_on_abort(s, ring);
        }
        return;
    }
    AccOf<T, NVMAX> acc;
    for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
        const SweepTask<T> &t = tasks[sweep_task_of(tasks, ntasks, g)];
        if (!down_sub_consume<T, NVMAX>(t.op, t.vec, s, pp, ring, acc, t.Lr, t.L, g - t.first, t.flag)) return;
    }
}

}  // namespace h2s
