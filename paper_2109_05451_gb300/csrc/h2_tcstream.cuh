// h2_tcstream.cuh -- multi-vector block rows on the tensor cores (split-BF16, FP32 accumulate).
//
// With nv vectors the per-level products of Sec. 3.2 (Alg 4) and the dense product become
// small GEMMs: for block (t, s), ( yhat_t )_{64 x N} += S_ts (64 x 64) * xhat_s (64 x N), N = nv
// padded to a multiple of 16. Each entry a is stored as a_hi + a_lo with a_hi = bf16(a),
// a_lo = bf16(a - a_hi); vectors are split the same way, and the product of the two split
// representations accumulates in FP32 in tensor memory.
//
// A block's tile is [S_hi; S_lo] (128 x 64, K-major) and a node's vector tile [x_hi; x_lo]
// (2N x 64), so one M = 128, N = 2N MMA per K-step forms all four partial products at once:
//   D = [ S_hi x_hi   S_hi x_lo ]   rows 0..63
//       [ S_lo x_hi   S_lo x_lo ]   rows 64..127,
// and the row result is the sum of the four N-column quadrants, added in the epilogue.
//
// Roles per CTA (persistent, work handed out in chunks of whole rows by an atomic ticket):
//   warp 4 (one lane): producer -- bulk-copies each block's hi/lo tiles (16 KB) and the input
//                      vector's hi/lo tiles (2 x N x 128 B) into a ring of stages;
//   warp 5 (one lane): MMA issuer -- 4 K-steps of tcgen05.mma per block into one of two TMEM
//                      accumulators; tcgen05.commit frees the stage when the MMAs of the
//                      block are done and signals the epilogue at the end of a row;
//   warps 0-3:         epilogue -- tcgen05.ld of the 128 x 2N accumulator (warp w: rows
//                      32w..32w+31); each thread adds its row's two column halves, warps 2-3
//                      hand their sums (the S_lo rows) to warps 0-1 through shared memory,
//                      and warps 0-1 store the FP32 row into the coefficient trees.
#pragma once

#include <cstdint>

#include "h2_stream.cuh"
#include "h2_tc.cuh"

namespace h2s {

constexpr int kTcThreads = 192;
constexpr uint32_t kTcTileBytes = 16384;  // hi (8 KB) + lo (8 KB) of one 64 x 64 block

struct TcArgs {
    const unsigned char *vals;       // block tiles (hi, lo), 16 KB each, in descriptor order
    const StreamDesc *desc;          // src = byte offset of the block's tiles
    const int64_t *chunks;
    int64_t nchunks;
    const unsigned char *xb;         // input vector tiles of the coefficient tree, per node
    const unsigned char *xtb;        // input vector tiles of the permuted input, per leaf
    float *yh, *yd;                  // FP32 output trees: (node, v, i) at (node*nv + v)*ld + i
    int nv;                          // vectors
    int kx, mp;                      // ld of yh / yd
    int *ticket;
    int *err;
    int ns;                          // pipeline stages
};

struct TcRowInfo {
    int32_t out_node;
    int16_t rows;
    int16_t flags;
};

// Two accumulator slots of 2 NP columns each.
__host__ __device__ constexpr uint32_t tc_tmem_cols(int np)
{
    return 4 * np <= 32 ? 32u : (4 * np <= 64 ? 64u : (4 * np <= 128 ? 128u : 256u));
}

__host__ __device__ constexpr size_t tc_smem_bytes(int np, int ns)
{
    return size_t(ns) * (kTcTileBytes + 2u * np * 128u) + 2u * 64u * np * sizeof(float) +
           size_t(ns) * sizeof(StreamDesc) + 2 * kChunkDesc * sizeof(StreamDesc) + (2 * ns + 13) * sizeof(uint64_t) +
           2 * 8 + 16;
}

// Grid: persistent; block: kTcThreads; NP = N (padded vectors, 16..64).
template <int NP>
__global__ void __launch_bounds__(kTcThreads, 1) k_stream_tc(TcArgs a)
{
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    constexpr uint32_t kVecBytes = 2u * NP * 128u;  // hi + lo tiles of one node's vectors
    constexpr uint32_t kStage = kTcTileBytes + kVecBytes;
    const int ns = a.ns;
    // layout: stages (1 KB aligned) | row exchange | descriptors | barriers | TMEM address | flags
    unsigned char *stages = tc_smem;
    float *xch = reinterpret_cast<float *>(stages + size_t(ns) * kStage);  // [2][NP][64]
    StreamDesc *sdesc = reinterpret_cast<StreamDesc *>(xch + 2 * 64 * NP);
    StreamDesc *dbuf = sdesc + ns;  // [2][kChunkDesc]
    uint64_t *full = reinterpret_cast<uint64_t *>(dbuf + 2 * kChunkDesc);
    uint64_t *empty = full + ns;
    uint64_t *dbar = empty + ns;     // [2]
    uint64_t *rowdone = dbar + 2;    // [2]
    uint64_t *accfree = rowdone + 2; // [2]
    uint64_t *fin = accfree + 2;     // the issuer's last MMAs have completed
    uint64_t *xready = fin + 1;      // [2] warps 2-3 have written their row sums
    uint64_t *xfree = xready + 2;    // [2] warps 0-1 have read them
    TcRowInfo *rowinfo = reinterpret_cast<TcRowInfo *>(xfree + 2);  // [2]
    uint32_t *taddr_s = reinterpret_cast<uint32_t *>(rowinfo + 2);
    int *abort_flag = reinterpret_cast<int *>(taddr_s + 1);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) {
        for (int i = 0; i < ns; ++i) {
            h2p::mbar_init(&full[i], 1);
            h2p::mbar_init(&empty[i], 1);  // arrived by tcgen05.commit of the issuer
        }
        h2p::mbar_init(&dbar[0], 1);
        h2p::mbar_init(&dbar[1], 1);
        for (int i = 0; i < 2; ++i) {
            h2p::mbar_init(&rowdone[i], 2);  // the issuer's arrive + its tcgen05.commit
            h2p::mbar_init(&accfree[i], 4);  // the four epilogue warps
            h2p::mbar_init(&xready[i], 2);   // lane 0 of warps 2 and 3
            h2p::mbar_init(&xfree[i], 2);    // lane 0 of warps 0 and 1
        }
        h2p::mbar_init(fin, 1);
        *abort_flag = 0;
        h2p::fence_barrier_init();
    }
    if (warp == 0) h2t::tmem_alloc(taddr_s, tc_tmem_cols(NP));
    h2t::fence_before_sync();
    __syncthreads();
    h2t::fence_after_sync();
    const uint32_t tmem = *taddr_s;

    if (warp == 4) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0, issued = 0, parity = 0;
            auto fetch_desc = [&](int slot, int64_t rec) {
                const int64_t b0 = rec >> 16;
                const uint32_t bytes = uint32_t(rec & 0xffff) * uint32_t(sizeof(StreamDesc));
                h2p::fence_proxy_async_shared();
                h2p::mbar_arrive_expect_tx(&dbar[slot], bytes);
                h2p::bulk_g2s(dbuf + slot * kChunkDesc, a.desc + b0, bytes, &dbar[slot]);
            };
            int64_t tA = atomicAdd(a.ticket, 1), tB = atomicAdd(a.ticket, 1);
            int64_t recA = tA < a.nchunks ? a.chunks[tA] : 0;
            int slot = 0;
            uint32_t dphase = 0;
            bool ok = true;
            if (tA < a.nchunks) fetch_desc(0, recA);
            while (ok && tA < a.nchunks) {
                const int64_t recB = tB < a.nchunks ? a.chunks[tB] : 0;
                const int64_t tC = atomicAdd(a.ticket, 1);
                ok = h2p::mbar_wait(&dbar[slot], dphase >> slot & 1u, abort_flag, a.err);
                dphase ^= 1u << slot;
                const int cnt = int(recA & 0xffff);
                const int pre = cnt - 1 < 4 ? cnt - 1 : 4;
                for (int i = 0; ok && i < cnt; ++i) {
                    if (i == pre && tB < a.nchunks) fetch_desc(slot ^ 1, recB);
                    const StreamDesc d = dbuf[slot * kChunkDesc + i];
                    ok = h2p::mbar_wait(&empty[stage], phase ^ 1u, abort_flag, a.err);
                    if (!ok) break;
                    sdesc[stage] = d;
                    unsigned char *st = stages + size_t(stage) * kStage;
                    if (d.flags & kZero) {
                        h2p::mbar_arrive(&full[stage]);
                    } else {
                        const unsigned char *x = (d.flags & kDense) ? a.xtb + size_t(d.x_node) * kVecBytes
                                                                    : a.xb + size_t(d.x_node) * kVecBytes;
                        h2p::mbar_arrive_expect_tx(&full[stage], kStage);
                        h2p::bulk_g2s(st, a.vals + d.src, kTcTileBytes, &full[stage]);
                        h2p::bulk_g2s(st + kTcTileBytes, x, kVecBytes, &full[stage]);
                        issued |= 1u << stage;
                        parity = (parity & ~(1u << stage)) | (phase << stage);
                    }
                    if (++stage == ns) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                slot ^= 1;
                tA = tB;
                recA = recB;
                tB = tC;
            }
            if (ok && h2p::mbar_wait(&empty[stage], phase ^ 1u, abort_flag, a.err)) {
                sdesc[stage].flags = kEnd;
                h2p::mbar_arrive(&full[stage]);
            }
            if (*abort_flag) {  // let every started copy land before the CTA can exit
                for (int i = 0; i < ns; ++i)
                    if (issued >> i & 1u) {
                        const long long t0 = clock64();
                        while (!h2p::mbar_try_wait(&full[i], parity >> i & 1u) && clock64() - t0 < h2p::kWaitCycles) {
                        }
                    }
            }
        }
    } else if (warp == 5) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = h2t::idesc_bf16_f32(128, 2 * NP);
            int stage = 0;
            uint32_t phase = 0;
            int acc = 0;              // accumulator slot
            uint32_t accphase = 0;    // parity of the slot's accfree phase to wait for
            bool fresh = true;        // next block starts a row
            for (;;) {
                if (!h2p::mbar_wait(&full[stage], phase, abort_flag, a.err)) break;
                const StreamDesc d = sdesc[stage];
                // a new row -- and the end marker, which travels like one -- may only take an
                // accumulator slot once the epilogue is done with the slot's previous row
                if (fresh || (d.flags & kEnd)) {
                    if (!h2p::mbar_wait(&accfree[acc], accphase ^ 1u, abort_flag, a.err)) break;
                    h2t::fence_after_sync();
                }
                if (d.flags & kEnd) {
                    rowinfo[acc].flags = kEnd;
                    h2p::mbar_arrive(&rowdone[acc]);
                    h2t::commit(&rowdone[acc]);
                    break;
                }
                if (!(d.flags & kZero)) {
                    const unsigned char *st = stages + size_t(stage) * kStage;
                    const uint64_t ad = h2t::smem_desc_sw128(st);                 // [S_hi; S_lo]
                    const uint64_t bd = h2t::smem_desc_sw128(st + kTcTileBytes);  // [x_hi; x_lo]
                    const uint32_t dt = tmem + uint32_t(acc * 2 * NP);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        h2t::mma_bf16(dt, ad + uint64_t(2 * kk), bd + uint64_t(2 * kk), idesc,
                                      (fresh && kk == 0) ? 0u : 1u);
                    fresh = false;
                } else {
                    fresh = true;  // a zero row is a whole row by itself
                }
                h2t::commit(&empty[stage]);  // stage free once these MMAs have read it
                if (d.flags & kLast) {
                    rowinfo[acc].out_node = d.out_node;
                    rowinfo[acc].rows = d.rows;
                    rowinfo[acc].flags = d.flags;
                    h2p::mbar_arrive(&rowdone[acc]);
                    h2t::commit(&rowdone[acc]);
                    if (acc == 1) accphase ^= 1u;
                    acc ^= 1;
                    fresh = true;
                }
                if (++stage == ns) {
                    stage = 0;
                    phase ^= 1u;
                }
            }
            // no MMA may be in flight when the accumulators are freed (also after an abort)
            h2t::commit(fin);
            const long long t0 = clock64();
            while (!h2p::mbar_try_wait(fin, 0) && clock64() - t0 < h2p::kWaitCycles) {
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue (warps 0-3)
        int acc = 0;
        uint32_t phase = 0;
        const bool lo_rows = warp >= 2;            // D rows 64..127: the S_lo products
        const int row = 32 * (warp & 1) + lane;    // output row of this thread
        const uint32_t lanes = uint32_t(32 * warp) << 16;
        for (;;) {
            if (!h2p::mbar_wait(&rowdone[acc], phase, abort_flag, a.err)) break;
            const TcRowInfo info = rowinfo[acc];
            if (info.flags & kEnd) break;
            h2t::fence_after_sync();
            float sum[NP];
            if (!(info.flags & kZero)) {
#pragma unroll
                for (int c = 0; c < NP; c += 16) {
                    uint32_t t0[16], t1[16];
                    h2t::tmem_ld16(tmem + uint32_t(acc * 2 * NP + c) + lanes, t0);
                    h2t::tmem_ld16(tmem + uint32_t(acc * 2 * NP + NP + c) + lanes, t1);
                    h2t::tmem_wait_ld();
#pragma unroll
                    for (int e = 0; e < 16; ++e) sum[c + e] = __uint_as_float(t0[e]) + __uint_as_float(t1[e]);
                }
            } else {
#pragma unroll
                for (int e = 0; e < NP; ++e) sum[e] = 0.f;
            }
            h2t::fence_before_sync();
            __syncwarp();
            if (lane == 0) h2p::mbar_arrive(&accfree[acc]);
            float *xs = xch + acc * 64 * NP;
            if (lo_rows) {
                if (!h2p::mbar_wait(&xfree[acc], phase ^ 1u, abort_flag, a.err)) break;
#pragma unroll
                for (int e = 0; e < NP; ++e) xs[e * 64 + row] = sum[e];
                __syncwarp();
                if (lane == 0) h2p::mbar_arrive(&xready[acc]);
            } else {
                if (!h2p::mbar_wait(&xready[acc], phase, abort_flag, a.err)) break;
                if (row < info.rows) {
                    const bool dense = info.flags & kDense;
                    const int ld = dense ? a.mp : a.kx;
                    float *base = (dense ? a.yd : a.yh) + int64_t(info.out_node) * ld * a.nv + row;
#pragma unroll
                    for (int e = 0; e < NP; ++e)
                        if (e < a.nv) base[e * ld] = sum[e] + xs[e * 64 + row];
                }
                __syncwarp();
                if (lane == 0) h2p::mbar_arrive(&xfree[acc]);
            }
            if (acc == 1) phase ^= 1u;
            acc ^= 1;
        }
    }
    h2t::fence_before_sync();
    __syncthreads();
    if (warp == 0) h2t::tmem_dealloc(tmem, tc_tmem_cols(NP));
}

}  // namespace h2s
