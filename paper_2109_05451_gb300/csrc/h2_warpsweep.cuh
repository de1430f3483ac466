// h2_warpsweep.cuh -- sweeps and coupling rows of operators of small rank (k <= 32), and the
// bottom downsweep of FP32 ranks 33 .. 64, one vector.
//
// With k <= 32 a node's coefficient vector fits one warp and a transfer or leaf-basis tile is
// a few hundred bytes to a few KB. The staged kernels of h2_stream.cuh (one tile per pipeline
// stage, reductions across four consumer warps, one producer thread) are then bound by their
// per-tile latency, not by HBM. The kernels here work at warp granularity and read their tiles
// straight from global memory:
//
//   k_up_cta     bottom subtrees, one CTA of eight warps each: leaf projections
//                xhat^q_t = U_t^T x_t (Sec. 3.1), then xhat^{l-1}_p = sum_c E_c^T xhat^l_c
//                (Alg 1) level by level, the vectors exchanged through shared memory;
//   k_down_cta   bottom subtrees: yhat^l_c = E_c yhat^{l-1}_p + yhat^l_c (the node's own
//                coupling row) level by level, then y_t = U_t yhat^q_t + (A_de x)_t and
//                Y[perm] = alpha y + beta Y at the leaves (Sec. 3.3, Alg 6);
//   k_down_cta2  the same downsweep for FP32 ranks 33 .. 64, two warps per node;
//   k_up_warp,   the upper levels (few nodes per level), one warp per node, ordered by
//   k_down_warp  flags in global memory;
//   k_rows_warp  coupling rows (Sec. 3.2, Alg 4), one warp per chunk of rows.
//
// Every product of a node or block is formed the same way: each lane accumulates a partial
// vector of KM (16 or 32 >= k) outputs from the tile entries it loaded (lane j takes row j of
// a transfer or coupling tile, lane i row i of the leaf basis), and one reduce-scatter over
// the warp (31 shuffles) leaves output o in lane o. A node issues its tile loads before it
// waits for the nodes it reads, so one memory latency, not one per tile row, lies on each
// dependency. Tiles are read in the layouts of h2_stream.cuh: U_t^T as [nu][i] (ld mp), E_c,
// E_c^T and S_ts^T as [j][o] (ld kx), where j is the input and o the output coefficient.
//
// Ordering of the flag-based sweeps: a node's work item comes after the items of the nodes it
// reads (its children in the upsweep, its parent in the downsweep), and a warp takes a ticket
// only while it runs, so each wait is for a warp that is already running and that itself
// waits only on earlier items; the waits end. Each one is still bounded (about a second): a
// wait that runs out raises the launch's abort word and the operator's error flag, and every
// warp then returns. A node publishes its vector by a release store of its flag after its
// lanes' stores and a fence; a reader acquires the flag in every lane and reads the vector
// through L2.
#pragma once

#include <cstdint>

#include "h2_pipe.cuh"
#include "h2_stream.cuh"

namespace h2s {

// Two warps per CTA: small CTAs also become resident next to a persistent block stream (the
// upper levels' sweeps run on a side stream while the lower levels' rows stream).
constexpr int kWsThreads = 64;
constexpr int kWsWarps = kWsThreads / 32;
constexpr int kWsChunk = 2;      // consecutive work items per ticket
constexpr int kWsMaxRank = 32;

// One launch of a warp sweep.
struct WarpSweep {
    int *ticket;  // this launch's work counter (zeroed by the gather)
    int *abort;   // raised by a wait that ran out (zeroed by the gather)
    int *flag;    // per heap node: set once the node's vector is final (zeroed by the gather)
    int lo, hi;   // upsweep: levels hi-1 .. lo from the vectors of level hi; downsweep: levels
                  // lo .. hi from the totals of level lo - 1
};

__device__ __forceinline__ int ld_acquire_gpu(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(int *p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Waits (lane 0) until *flag is set, then acquires it in every lane. False, in every lane,
// once this launch aborted: another wait raised the abort word, or this one saw no flag for
// `budget` clock cycles and raised it (and the error flag) itself.
__device__ __forceinline__ bool ws_wait_for(const int *flag, int *abort, int *err, long long budget)
{
    const int lane = threadIdx.x & 31;
    int ok = 1;
    if (lane == 0 && !ld_acquire_gpu(flag)) {
        const long long t0 = clock64();
        for (;;) {
            if (ld_acquire_gpu(flag)) break;
            if (*reinterpret_cast<volatile int *>(abort)) {
                ok = 0;
                break;
            }
            if (clock64() - t0 > budget) {
                atomicExch(abort, 1);
                if (err) atomicExch(err, 1);
                ok = 0;
                break;
            }
        }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (ok) (void)ld_acquire_gpu(flag);
    return ok != 0;
}

__device__ __forceinline__ bool ws_wait(const int *flag, int *abort, int *err)
{
    return ws_wait_for(flag, abort, err, h2p::kWaitCycles);
}

// After the lanes' stores of a node's vector: every lane fences, then lane 0 sets the flag.
__device__ __forceinline__ void ws_publish(int *flag)
{
    __threadfence();
    __syncwarp();
    if ((threadIdx.x & 31) == 0) st_release_gpu(flag, 1);
}

// Next ticket of the warp (lane 0 draws, all lanes get it).
__device__ __forceinline__ int64_t ws_ticket(int *ticket)
{
    int t = 0;
    if ((threadIdx.x & 31) == 0) t = atomicAdd(ticket, 1);
    return int64_t(__shfl_sync(0xffffffffu, t, 0));
}

// Sum over the warp of the lanes' partial vectors p[0 .. KM): afterwards p[0] of lane l holds
// output l mod KM. Pairs of lanes halve the outputs they keep at each step (KM = 32) or first
// add their whole vectors (the step of offset 16 with KM = 16).
template <typename T, int KM>
__device__ __forceinline__ T ws_reduce(T (&p)[KM])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        if (s >= KM) {
#pragma unroll
            for (int j = 0; j < KM; ++j) p[j] += __shfl_xor_sync(0xffffffffu, p[j], s);
        } else {
            const bool upper = (lane & s) != 0;
#pragma unroll
            for (int j = 0; j < s; ++j) {
                const T send = upper ? p[j] : p[j + s];
                const T keep = upper ? p[j + s] : p[j];
                p[j] = keep + __shfl_xor_sync(0xffffffffu, send, s);
            }
        }
    }
    return p[0];
}

// Row j of a tile ([j][o], ld kx): r[o] for o < KM, zero beyond kx and when not active.
// 16-byte loads (kx is a multiple of 4, tile rows start on 16 bytes).
template <typename T, int KM>
__device__ __forceinline__ void ws_load_row_at(const T *__restrict__ tile, int j, bool active, int kx, T (&r)[KM])
{
    constexpr int V = 16 / sizeof(T);  // elements per 16-byte load
    const T *__restrict__ row = tile + int64_t(j) * kx;
#pragma unroll
    for (int q = 0; q < KM / V; ++q) {
        if (active && q * V < kx) {
            if constexpr (V == 4) {
                const float4 v = __ldg(reinterpret_cast<const float4 *>(row) + q);
                r[4 * q] = v.x, r[4 * q + 1] = v.y, r[4 * q + 2] = v.z, r[4 * q + 3] = v.w;
            } else {
                const double2 v = __ldg(reinterpret_cast<const double2 *>(row) + q);
                r[2 * q] = v.x, r[2 * q + 1] = v.y;
            }
        } else {
#pragma unroll
            for (int e = 0; e < V; ++e) r[V * q + e] = T(0);
        }
    }
}

// Row j = lane of a transfer tile (zero for lanes j >= k).
template <typename T, int KM>
__device__ __forceinline__ void ws_load_row(const T *__restrict__ tile, int k, int kx, T (&r)[KM])
{
    const int lane = threadIdx.x & 31;
    ws_load_row_at<T, KM>(tile, lane, lane < k, kx, r);
}

// Leaf projection xhat_t = U_t^T x_t (Sec. 3.1): lane i takes rows i, i + 32, ... of U_t
// (column i of U_t^T, ld mp); returns entry o of xhat_t in lane o (o < KM, lane mod KM).
template <typename T, int KM>
__device__ __forceinline__ T ws_project_leaf(const Op<T> &op, const Vec<T> &vec, int64_t t)
{
    const int lane = threadIdx.x & 31;
    const int k = op.k, kx = op.kx, mp = op.mp;
    const int R = op.leaf_lo[t + 1] - op.leaf_lo[t];
    const T *__restrict__ x = vec.xt + t * mp * vec.vs;
    const T *__restrict__ ut = op.Ut + t * kx * mp;
    T p[KM];
#pragma unroll
    for (int j = 0; j < KM; ++j) p[j] = T(0);
    for (int rb = 0; rb < mp; rb += 64) {  // two row blocks per round of loads
        const int i0 = rb + lane, i1 = rb + 32 + lane;
        const T x0 = i0 < R ? x[i0] : T(0), x1 = i1 < R ? x[i1] : T(0);
        T u0[KM], u1[KM];
#pragma unroll
        for (int j = 0; j < KM; ++j) {
            u0[j] = j < k && i0 < mp ? __ldg(ut + j * mp + i0) : T(0);
            u1[j] = j < k && i1 < mp ? __ldg(ut + j * mp + i1) : T(0);
        }
#pragma unroll
        for (int j = 0; j < KM; ++j) p[j] = fma(u1[j], x1, fma(u0[j], x0, p[j]));
    }
    return ws_reduce<T, KM>(p);
}

// Upsweep of the levels hi - 1 .. lo from the vectors of level hi (computed by an earlier
// launch): items bottom-up, item g of level l being node 3 * 2^l + g - 2^hi.
template <typename T, int KM>
__global__ void __launch_bounds__(kWsThreads, 8) k_up_warp(Op<T> op, Vec<T> vec, WarpSweep ws)
{
    const int lane = threadIdx.x & 31;
    const int k = op.k, kx = op.kx, vs = vec.vs;
    const int top = ws.hi - 1;
    if (top < ws.lo) return;
    const int64_t span = int64_t(2) << top;  // 2^(top+1)
    const int64_t total = span - (int64_t(1) << ws.lo);
    for (;;) {
        const int64_t g0 = ws_ticket(ws.ticket) * kWsChunk;
        if (g0 >= total) return;
        const int64_t g1 = g0 + kWsChunk < total ? g0 + kWsChunk : total;
        for (int64_t g = g0; g < g1; ++g) {
            const int l = 63 - __clzll(static_cast<unsigned long long>(span - g - 1));
            const int64_t node = (int64_t(3) << l) + g - span;
            // xhat_p = sum over the two children of E_c^T xhat_c; lane j takes row j of each
            // child's tile (loaded before the children are waited for) and entry j of its vector
            const int64_t c0 = 2 * node;
            T e0[KM], e1[KM];
            ws_load_row<T, KM>(op.E + c0 * k * kx, k, kx, e0);
            ws_load_row<T, KM>(op.E + (c0 + 1) * k * kx, k, kx, e1);
            const bool wait = l + 1 <= top;  // the children are items of this launch
            if (wait && !ws_wait(ws.flag + c0, ws.abort, vec.err)) return;
            if (wait && !ws_wait(ws.flag + c0 + 1, ws.abort, vec.err)) return;
            const T x0 = lane < k ? __ldcg(vec.xh + c0 * kx * vs + lane) : T(0);
            const T x1 = lane < k ? __ldcg(vec.xh + (c0 + 1) * kx * vs + lane) : T(0);
            T p[KM];
#pragma unroll
            for (int j = 0; j < KM; ++j) p[j] = fma(e1[j], x1, e0[j] * x0);
            const T r = ws_reduce<T, KM>(p);
            if (lane < k) vec.xh[node * kx * vs + lane] = r;
            if (l > ws.lo) ws_publish(ws.flag + node);
        }
    }
}

// Downsweep of the levels lo .. hi (the totals of level lo - 1 from an earlier launch): items
// top-down, item g being heap node 2^lo + g; every total is written to yhat for the next
// launch or level.
template <typename T, int KM>
__global__ void __launch_bounds__(kWsThreads, 8) k_down_warp(Op<T> op, Vec<T> vec, WarpSweep ws)
{
    const int lane = threadIdx.x & 31;
    const int k = op.k, kx = op.kx, vs = vec.vs;
    if (ws.hi < ws.lo) return;
    const int64_t first = int64_t(1) << ws.lo;
    const int64_t total = (int64_t(2) << ws.hi) - first;
    for (;;) {
        const int64_t g0 = ws_ticket(ws.ticket) * kWsChunk;
        if (g0 >= total) return;
        const int64_t g1 = g0 + kWsChunk < total ? g0 + kWsChunk : total;
        for (int64_t g = g0; g < g1; ++g) {
            const int64_t node = first + g;
            const int l = 63 - __clzll(static_cast<unsigned long long>(node));
            // everything that does not depend on the parent is loaded first
            const T own = lane < k ? vec.yh[node * kx * vs + lane] : T(0);  // the node's coupling row
            T e[KM];
            if (l >= 1) ws_load_row<T, KM>(op.Et + node * k * kx, k, kx, e);
            T acc = T(0);
            if (l >= 1) {
                const int64_t p = node >> 1;
                // a parent of level lo - 1 was completed by an earlier launch
                if (l - 1 >= ws.lo && !ws_wait(ws.flag + p, ws.abort, vec.err)) return;
                const T yp = lane < k ? __ldcg(vec.yh + p * kx * vs + lane) : T(0);
                T q[KM];
#pragma unroll
                for (int j = 0; j < KM; ++j) q[j] = e[j] * yp;
                acc = ws_reduce<T, KM>(q);
            }
            acc += own;
            if (lane < k) vec.yh[node * kx * vs + lane] = acc;
            if (l < ws.hi) ws_publish(ws.flag + node);
        }
    }
}

// ---- bottom subtrees: one CTA of eight warps per subtree, vectors in shared memory

constexpr int kCtaWarps = 8;
constexpr int kCtaThreads = 32 * kCtaWarps;

// Shared memory of a subtree CTA: one KM-entry slot per node of a subtree of depth L (local
// heap order: slot 1 is the root, slots 2^L .. 2^(L+1)-1 the leaves).
template <typename T, int KM>
__host__ __device__ constexpr size_t cta_smem_bytes(int L)
{
    return (size_t(2) << L) * KM * sizeof(T);
}

// Upsweep of the subtree st rooted at level Lr with depth L = q - Lr (Sec. 3.1, Alg 1): the
// warps project the 2^L leaves, then compute the levels q - 1 .. Lr one barrier apart, every
// warp taking the nodes w, w + 8, ... of a level; each vector is written to xhat (for the block
// streams and the upper levels) and to the CTA's slot of the node. A warp loads the transfer
// rows of its next node before it waits at the barrier.
template <typename T, int KM>
__global__ void __launch_bounds__(kCtaThreads, 2) k_up_cta(Op<T> op, Vec<T> vec, int Lr, int L)
{
    extern __shared__ __align__(16) unsigned char ws_smem[];
    T *sx = reinterpret_cast<T *>(ws_smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = op.k, kx = op.kx, vs = vec.vs;
    const int64_t st = blockIdx.x;
    const int nleaf = 1 << L;
    for (int j = warp; j < nleaf; j += kCtaWarps) {
        const int64_t t = st * nleaf + j;
        const T r = ws_project_leaf<T, KM>(op, vec, t);
        if (lane < k) {
            vec.xh[(op.first_leaf + t) * kx * vs + lane] = r;
            sx[(nleaf + j) * KM + lane] = r;
        }
    }
    T e0[KM], e1[KM];
    auto load_rows = [&](int rel, int i) {  // transfer rows of the children of local node (rel, i)
        const int64_t c0 = 2 * ((int64_t(1) << (Lr + rel)) + st * (int64_t(1) << rel) + i);
        ws_load_row<T, KM>(op.E + c0 * k * kx, k, kx, e0);
        ws_load_row<T, KM>(op.E + (c0 + 1) * k * kx, k, kx, e1);
    };
    if (L >= 1 && warp < (1 << (L - 1))) load_rows(L - 1, warp);
    __syncthreads();
    for (int rel = L - 1; rel >= 0; --rel) {
        const int cnt = 1 << rel;
        for (int i = warp; i < cnt; i += kCtaWarps) {
            if (i != warp) load_rows(rel, i);  // nodes beyond the first of this warp
            const int slot = cnt + i;
            const T x0 = lane < k ? sx[(2 * slot) * KM + lane] : T(0);
            const T x1 = lane < k ? sx[(2 * slot + 1) * KM + lane] : T(0);
            T p[KM];
#pragma unroll
            for (int j = 0; j < KM; ++j) p[j] = fma(e1[j], x1, e0[j] * x0);
            const T r = ws_reduce<T, KM>(p);
            if (lane < k) {
                vec.xh[((int64_t(1) << (Lr + rel)) + st * cnt + i) * kx * vs + lane] = r;
                sx[slot * KM + lane] = r;
            }
        }
        if (rel >= 1 && warp < (cnt >> 1)) load_rows(rel - 1, warp);
        __syncthreads();
    }
}

// Downsweep of the subtree st rooted at level Lr with depth L = q - Lr (Sec. 3.3, Alg 6): the
// root's total yhat_r = E_r yhat_parent + own_r (the parent's total from an earlier launch;
// none at the tree root), then the levels below one barrier apart (totals in the CTA's slots
// only), and at the leaves the expansion and epilogue. A warp loads its next node's transfer
// rows, coupling row and, for a leaf, basis rows, dense result and output rows before it
// waits at the barrier.
template <typename T, int KM>
__global__ void __launch_bounds__(kCtaThreads, 2) k_down_cta(Op<T> op, Vec<T> vec, int Lr, int L)
{
    extern __shared__ __align__(16) unsigned char ws_smem[];
    T *sy = reinterpret_cast<T *>(ws_smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = op.k, kx = op.kx, mp = op.mp, vs = vec.vs;
    const int64_t st = blockIdx.x;
    T e[KM], own = T(0);
    auto node_of = [&](int rel, int i) { return (int64_t(1) << (Lr + rel)) + st * (int64_t(1) << rel) + i; };
    auto load_node = [&](int rel, int i) {
        const int64_t node = node_of(rel, i);
        own = lane < k ? vec.yh[node * kx * vs + lane] : T(0);
        if (Lr + rel >= 1) ws_load_row<T, KM>(op.Et + node * k * kx, k, kx, e);
    };
    // the parent's vector (lane j: entry j): the CTA's slot, or for the root the total of an
    // earlier launch
    auto parent_of = [&](int rel, int i) -> T {
        if (rel >= 1) return lane < k ? sy[((1 << (rel - 1)) + (i >> 1)) * KM + lane] : T(0);
        if (Lr == 0) return T(0);
        return lane < k ? __ldcg(vec.yh + (node_of(0, 0) >> 1) * kx * vs + lane) : T(0);
    };
    auto total_of = [&](int rel, int i) -> T {
        T acc = T(0);
        if (Lr + rel >= 1) {
            const T yp = parent_of(rel, i);
            T q[KM];
#pragma unroll
            for (int j = 0; j < KM; ++j) q[j] = e[j] * yp;
            acc = ws_reduce<T, KM>(q);
        }
        return acc + own;
    };
    // internal levels Lr .. q - 1
    if (L >= 1 && warp == 0) load_node(0, 0);
    for (int rel = 0; rel < L; ++rel) {
        const int cnt = 1 << rel;
        for (int i = warp; i < cnt; i += kCtaWarps) {
            if (i != warp) load_node(rel, i);
            const T acc = total_of(rel, i);
            if (lane < k) sy[(cnt + i) * KM + lane] = acc;
        }
        if (rel + 1 < L && warp < 2 * cnt) load_node(rel + 1, warp);
        __syncthreads();
    }
    // leaves: y_i = sum_nu U_t[i][nu] yhat_nu + (A_de x)_i, Y[perm] = alpha y + beta Y
    const int nleaf = 1 << L;
    for (int j = warp; j < nleaf; j += kCtaWarps) {
        const int64_t t = st * nleaf + j;
        load_node(L, j);
        const int r0 = op.leaf_lo[t], R = op.leaf_lo[t + 1] - r0;
        const T *__restrict__ ut = op.Ut + t * kx * mp;
        const T *__restrict__ yd = vec.yd + t * mp * vs;
        const int i0 = lane, i1 = 32 + lane;
        T u0[KM], u1[KM], d0 = T(0), d1 = T(0);
        int perm0 = 0, perm1 = 0;
#pragma unroll
        for (int jj = 0; jj < KM; ++jj) {
            u0[jj] = jj < k && i0 < mp ? __ldg(ut + jj * mp + i0) : T(0);
            u1[jj] = jj < k && i1 < mp ? __ldg(ut + jj * mp + i1) : T(0);
        }
        if (i0 < R) d0 = yd[i0], perm0 = op.perm[r0 + i0];
        if (i1 < R) d1 = yd[i1], perm1 = op.perm[r0 + i1];
        const T acc = total_of(L, j);
        T y0 = T(0), y1 = T(0);
#pragma unroll
        for (int jj = 0; jj < KM; ++jj) {
            const T a = __shfl_sync(0xffffffffu, acc, jj);
            y0 = fma(u0[jj], a, y0);
            y1 = fma(u1[jj], a, y1);
        }
        if (i0 < R) {
            const T v = y0 + d0;
            T *dst = vec.Y + perm0;
            *dst = (vec.beta == T(0)) ? vec.alpha * v : vec.alpha * v + vec.beta * *dst;
        }
        if (i1 < R) {
            const T v = y1 + d1;
            T *dst = vec.Y + perm1;
            *dst = (vec.beta == T(0)) ? vec.alpha * v : vec.alpha * v + vec.beta * *dst;
        }
        for (int ib = 64; ib < R; ib += 32) {  // rows beyond 64, uniform over the warp
            const int i = ib + lane;
            T y = T(0);
            for (int jj = 0; jj < k; ++jj) {
                const T a = __shfl_sync(0xffffffffu, acc, jj);
                if (i < mp) y = fma(__ldg(ut + jj * mp + i), a, y);
            }
            if (i < R) {
                const T v = y + yd[i];
                T *dst = vec.Y + op.perm[r0 + i];
                *dst = (vec.beta == T(0)) ? vec.alpha * v : vec.alpha * v + vec.beta * *dst;
            }
        }
    }
}

// ---- bottom downsweep of ranks 33 .. 64 (FP32): two warps per node
//
// A 64-output product does not fit one warp's registers, so each node is taken by a pair of
// warps: warp h of the pair forms the outputs 32h .. 32h + 31, lane j accumulating rows j and
// j + 32 of the tile, and one reduce-scatter leaves output 32h + o in lane o. The CTA's four
// pairs take the nodes of a level in turn, one barrier apart, as in k_down_cta; the
// shared-memory slots hold 64 entries per node (cta_smem_bytes<float, 64>). (The same scheme
// for the upsweep measured slower than the staged k_up_sub at these ranks: its leaf
// projections read 16 KB tiles per warp pair without the bulk-copy pipeline's depth.)

constexpr int kCtaPairs = kCtaWarps / 2;

// Barrier of the 64 threads of warp pair `pair` (named barrier 1 + pair; barrier 0 is
// __syncthreads).
__device__ __forceinline__ void ws_pair_sync(int pair)
{
    asm volatile("bar.sync %0, 64;" ::"r"(1 + pair) : "memory");
}

// Rows j = lane and j + 32 of a tile ([j][o], ld kx), columns 32h .. 32h + 31: zero for rows
// >= k and columns >= kx. 16-byte loads (kx is a multiple of 4, tile rows start on 16 bytes).
__device__ __forceinline__ void wp_load_rows(const float *__restrict__ tile, int k, int kx, int h, float (&a)[32],
                                             float (&b)[32])
{
    const int lane = threadIdx.x & 31;
    const float4 *ra = reinterpret_cast<const float4 *>(tile + int64_t(lane) * kx + 32 * h);
    const float4 *rb = reinterpret_cast<const float4 *>(tile + int64_t(lane + 32) * kx + 32 * h);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const bool col = 32 * h + 4 * q < kx;
        const float4 va = col && lane < k ? __ldg(ra + q) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 vb = col && lane + 32 < k ? __ldg(rb + q) : make_float4(0.f, 0.f, 0.f, 0.f);
        a[4 * q] = va.x, a[4 * q + 1] = va.y, a[4 * q + 2] = va.z, a[4 * q + 3] = va.w;
        b[4 * q] = vb.x, b[4 * q + 1] = vb.y, b[4 * q + 2] = vb.z, b[4 * q + 3] = vb.w;
    }
}

// p[o] += a[o] x_j + b[o] x_{j+32} with the inputs of a node in slot `slot` (lane j: j, j + 32)
__device__ __forceinline__ void wp_accumulate(const float *__restrict__ s, int slot, int k, const float (&a)[32],
                                              const float (&b)[32], float (&p)[32])
{
    const int lane = threadIdx.x & 31;
    const float xa = lane < k ? s[slot * 64 + lane] : 0.f;
    const float xb = lane + 32 < k ? s[slot * 64 + lane + 32] : 0.f;
#pragma unroll
    for (int o = 0; o < 32; ++o) p[o] = fmaf(b[o], xb, fmaf(a[o], xa, p[o]));
}

// Downsweep of the subtree st rooted at level Lr with depth L = q - Lr (Sec. 3.3, Alg 6), ranks
// 33 .. 64: the totals level by level in the CTA's slots (the root's parent total from an
// earlier launch), then per leaf its total, the expansion (warp h of the pair takes the rows
// 32h + lane, 32h + lane + 64, ...) and the epilogue.
template <typename T>
__global__ void __launch_bounds__(kCtaThreads, 2) k_down_cta2(Op<T> op, Vec<T> vec, int Lr, int L)
{
    static_assert(sizeof(T) == 4, "FP32 only: 64 FP64 outputs per warp pair would not fit the registers");
    extern __shared__ __align__(16) unsigned char ws_smem[];
    float *sy = reinterpret_cast<float *>(ws_smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int pair = warp >> 1, h = warp & 1, o = 32 * h + lane;
    const int k = op.k, kx = op.kx, mp = op.mp, vs = vec.vs;
    const int64_t st = blockIdx.x;
    // the total of node (rel, i) into its slot: E_node yhat_parent + own
    auto total = [&](int rel, int i) {
        const int64_t node = (int64_t(1) << (Lr + rel)) + st * (int64_t(1) << rel) + i;
        const float own = o < k ? vec.yh[node * kx * vs + o] : 0.f;
        float p[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) p[q] = 0.f;
        float r = 0.f;
        if (Lr + rel >= 1) {
            float a[32], b[32];
            wp_load_rows(op.Et + node * k * kx, k, kx, h, a, b);
            if (rel >= 1) {
                wp_accumulate(sy, (1 << (rel - 1)) + (i >> 1), k, a, b, p);
            } else {  // the subtree root: its parent's total from an earlier launch
                const float *yp = vec.yh + (node >> 1) * kx * vs;
                const float xa = lane < k ? __ldcg(yp + lane) : 0.f;
                const float xb = lane + 32 < k ? __ldcg(yp + lane + 32) : 0.f;
#pragma unroll
                for (int q = 0; q < 32; ++q) p[q] = fmaf(b[q], xb, fmaf(a[q], xa, p[q]));
            }
            r = ws_reduce<float, 32>(p);
        }
        if (o < k) sy[((1 << rel) + i) * 64 + o] = r + own;
    };
    for (int rel = 0; rel < L; ++rel) {
        for (int i = pair; i < (1 << rel); i += kCtaPairs) total(rel, i);
        __syncthreads();
    }
    const int nleaf = 1 << L;
    for (int j = pair; j < nleaf; j += kCtaPairs) {
        total(L, j);
        ws_pair_sync(pair);  // both halves of the leaf's total are in its slot
        const int64_t t = st * nleaf + j;
        const int r0 = op.leaf_lo[t], R = op.leaf_lo[t + 1] - r0;
        const float *__restrict__ ut = op.Ut + t * kx * mp;
        const float *__restrict__ yd = vec.yd + t * mp * vs;
        const float *__restrict__ yl = sy + (nleaf + j) * 64;
        for (int ib = 32 * h; ib < R; ib += 64) {  // uniform over the warp
            const int i = ib + lane;
            float y = 0.f;
            if (i < mp) {
#pragma unroll 16
                for (int nu = 0; nu < k; ++nu) y = fmaf(__ldg(ut + nu * mp + i), yl[nu], y);
            }
            if (i < R) {
                const float v = y + yd[i];
                float *dst = vec.Y + op.perm[r0 + i];
                *dst = (vec.beta == 0.f) ? vec.alpha * v : vec.alpha * v + vec.beta * *dst;
            }
        }
    }
}

// Block rows of small coupling blocks (k <= 32), one vector (Sec. 3.2, Alg 4): one warp per
// scheduling chunk of whole rows (chunks[c] = (first descriptor << 16) | count), taken from
// the ticket vec.tickets[ticket_index]. With KM = 16 each half-warp takes its own block (H = 2
// blocks per load slot), with KM = 32 the whole warp one; lane j of a group takes row j of the
// block's tile S_ts^T ([j][o], ld kx) and entry j of xhat_s, so a row's partial vectors need
// one reduce-scatter at its end. The blocks are added in order (the groups of a slot one
// after the other), so a row that ends inside a slot is reduced before the next row's block
// is added. The tiles of NB slots are loaded at once (NB x KM values per lane), and the next
// chunk's ticket is drawn while the current one is processed. An empty row (kZero) is stored
// as zeros. Rows are independent: no warp waits for another.
template <typename T, int KM>
__global__ void __launch_bounds__(kWsThreads, 8)
    k_rows_warp(Op<T> op, Vec<T> vec, const StreamDesc *__restrict__ desc, const int64_t *__restrict__ chunks,
                int64_t nchunks, int ticket_index)
{
    constexpr int NB = (64 * 4 / int(sizeof(T))) / KM;  // load slots: 64 registers of tiles
    constexpr int H = 32 / KM;                          // blocks per slot, one per lane group
    const int lane = threadIdx.x & 31;
    const int grp = lane / KM, j = lane % KM;
    const int k = op.k, kx = op.kx, vs = vec.vs;
    int *ticket = vec.tickets + ticket_index;
    int64_t c = ws_ticket(ticket);
    T p[KM];
#pragma unroll
    for (int q = 0; q < KM; ++q) p[q] = T(0);
    while (c < nchunks) {
        int next = 0;
        if (lane == 0) next = atomicAdd(ticket, 1);  // used after this chunk
        const int64_t rec = chunks[c];
        const int64_t b0 = rec >> 16;
        const int cnt = int(rec & 0xffff);
        for (int gb = 0; gb < cnt; gb += 32) {
            const int n = cnt - gb < 32 ? cnt - gb : 32;
            // lane i holds descriptor gb + i of the chunk
            uint64_t src = 0;
            int xn = 0, on = 0, fl = 0;
            if (lane < n) {
                const StreamDesc d = desc[b0 + gb + lane];
                src = d.src;
                xn = d.x_node;
                on = d.out_node;
                fl = d.flags;
            }
            for (int b = 0; b < n; b += NB * H) {
                T t[NB][KM], xv[NB];
                int fb[NB][H], ob[NB][H];
#pragma unroll
                for (int u = 0; u < NB; ++u) {
#pragma unroll
                    for (int e = 0; e < H; ++e) {
                        const int be = b + H * u + e < n ? b + H * u + e : n - 1;
                        fb[u][e] = __shfl_sync(0xffffffffu, fl, be);
                        ob[u][e] = __shfl_sync(0xffffffffu, on, be);
                    }
                    const int mine = b + H * u + grp;  // this lane group's block
                    const int bi = mine < n ? mine : n - 1;
                    const uint64_t sb = __shfl_sync(0xffffffffu, src, bi);
                    const int xb = __shfl_sync(0xffffffffu, xn, bi);
                    const int fm = __shfl_sync(0xffffffffu, fl, bi);
                    const bool live = mine < n && !(fm & kZero) && j < k;
                    ws_load_row_at<T, KM>(reinterpret_cast<const T *>(op.vals + sb), j, live, kx, t[u]);
                    xv[u] = live ? vec.xh[int64_t(xb) * kx * vs + j] : T(0);
                }
#pragma unroll
                for (int u = 0; u < NB; ++u) {
#pragma unroll
                    for (int e = 0; e < H; ++e) {
                        if (b + H * u + e >= n) break;
                        if (grp == e) {
#pragma unroll
                            for (int q = 0; q < KM; ++q) p[q] = fma(t[u][q], xv[u], p[q]);
                        }
                        if (fb[u][e] & kLast) {
                            const T r = ws_reduce<T, KM>(p);
                            if (lane < k) vec.yh[int64_t(ob[u][e]) * kx * vs + lane] = r;
#pragma unroll
                            for (int q = 0; q < KM; ++q) p[q] = T(0);
                        }
                    }
                }
            }
        }
        c = __shfl_sync(0xffffffffu, next, 0);
    }
}

}  // namespace h2s
