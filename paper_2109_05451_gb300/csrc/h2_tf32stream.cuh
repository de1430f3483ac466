// h2_tf32stream.cuh -- multi-vector block rows of the FP32 operator on the tensor cores (3xTF32).
//
// With nv vectors the per-level products of Sec. 3.2 (Alg 4) and the dense product are small
// GEMMs: for block (t, s), yhat_t (64 x N) += S_ts (64 x 64) * xhat_s (64 x N). The FP32 blocks
// are the ones the single-vector stream reads (column-major tiles, rows padded to 4), and the
// vectors are the FP32 coefficient and leaf trees the sweeps write ([node][v][i]); nothing is
// stored twice. Each value a is split as a = a_hi + a_lo with a_hi = a with its 13 low
// mantissa bits cleared (exact as a TF32 operand) and a_lo = a - a_hi (exact in FP32,
// |a_lo| < 2^-10 |a|); the tensor core keeps a_lo to TF32 precision whether it truncates or
// rounds its low bits, so a_hi + a_lo carries a to about 2^-21 relative. The MMA operands are
//   A = [S_hi; S_lo]  (128 x 64, in tensor memory)     B = [x_hi | x_lo]  (64 x 2N, K-major)
// so one M = 128, N = 2N MMA per K-step forms all four partial products, and the row result is
// the sum of the four N-column quadrants of D (FP32, in tensor memory).
//
// A 1-D bulk copy stages each block's tile and its input node's FP32 vector rows (the same
// 24 KB per block at 32 vectors as the split-BF16 stream, so the same L2 footprint); eight
// converter warps split both and free the stage at once: S goes to tensor memory
// (tcgen05.st), x to a swizzled B slot in shared memory, so the MMA reads only B from shared
// memory. Warp w may access TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31, hence the numbering:
//   warps 0-3:  epilogue -- tcgen05.ld of the 128 x 2N accumulator (warp w: rows 32w..32w+31),
//               row sums of the two column halves, warps 2-3 (the S_lo rows) hand theirs to
//               warps 0-1 through shared memory, warps 0-1 store the FP32 row;
//   warps 4-19: converters, two groups of eight that take alternate descriptors (a block's
//               split is a chain of shared-memory loads, TMEM stores and barrier hand-offs, so
//               two blocks are split at once) -- warp 4 + 8g + q + 4h writes TMEM lanes
//               32q..32q+31, columns 32h..32h+31 of an A slot: S_hi rows (q = 0, 1) or S_lo
//               rows (q = 2, 3), one tile row per thread; the group also writes the block's B
//               slot; every descriptor (also the empty-row and end markers) passes to the MMA
//               issuer through an A/B slot pair;
//   warp 20:    producer (one lane) -- chunk tickets, bulk copies into a ring of stages;
//   warp 21:    MMA issuer (one lane) -- 8 K-steps of tcgen05.mma.kind::tf32 per block into one
//               of two accumulator slots; tcgen05.commit frees the A/B slot pair.
// Every wait is bounded; on timeout the kernel raises the error flag and unwinds (the
// producer lets its copies in flight land first, and TMEM is freed after the last MMA).
#pragma once

#include <cstdint>

#include "h2_stream.cuh"
#include "h2_tc.cuh"

namespace h2s {

constexpr int kTfConverters = 8;          // converter warps per group
constexpr int kTfGroups = 2;              // converter groups; group g splits blocks j = g mod 2
constexpr int kTfThreads = 32 * (4 + kTfGroups * kTfConverters + 2);
constexpr int kTfAslots = 3;              // A (TMEM) / B (shared memory) operand slot pairs
constexpr uint32_t kTfTileBytes = 16384;  // largest FP32 block tile: 64 x 64

struct TfArgs {
    const unsigned char *vals;       // FP32 block tiles (column-major, ld = rows rounded up to 4)
    const StreamDesc *desc;          // src = byte offset of the block's tile
    const int64_t *chunks;
    int64_t nchunks;
    const float *xh, *xt;            // FP32 input trees: (node, v, i) at (node*nv + v)*ld + i
    float *yh, *yd;                  // FP32 output trees, same layouts
    int nv;                          // vectors
    int kx, mp;                      // ld of the coefficient / leaf trees
    int *ticket;
    int *err;
    int ns;                          // pipeline stages (<= 16)
};

// TMEM columns: two accumulator slots of 2 NP columns, then kTfAslots A slots of 64 columns.
__host__ __device__ constexpr uint32_t tf_tmem_cols(int np) { return 4 * np + 64 * kTfAslots <= 256 ? 256u : 512u; }

__host__ __device__ constexpr uint32_t tf_x_bytes(int np) { return uint32_t(np) * 64u * 4u; }    // staged x rows
__host__ __device__ constexpr uint32_t tf_b_bytes(int np) { return 2u * np * 256u; }            // [x_hi; x_lo]
__host__ __device__ constexpr uint32_t tf_stage_bytes(int np) { return kTfTileBytes + tf_x_bytes(np); }

__host__ __device__ constexpr size_t tf_smem_bytes(int np, int ns)
{
    return size_t(kTfAslots) * tf_b_bytes(np) + size_t(ns) * tf_stage_bytes(np) + 2u * 64u * np * sizeof(float) +
           size_t(ns + kTfAslots) * sizeof(StreamDesc) + 2 * kChunkDesc * sizeof(StreamDesc) +
           (2 * ns + 13 + 2 * kTfAslots) * sizeof(uint64_t) + 2 * 8 + 16;
}

// Grid: persistent; block: kTfThreads; NP = vectors padded to 16 or 32.
template <int NP>
__global__ void __launch_bounds__(kTfThreads, 1) k_stream_tf32(TfArgs a)
{
    extern __shared__ __align__(1024) unsigned char tf_smem[];
    constexpr uint32_t kB = tf_b_bytes(NP);
    constexpr uint32_t kStage = tf_stage_bytes(NP);
    constexpr uint32_t kAcol = 4u * NP;  // first column of the A slots
    const int ns = a.ns;
    // layout: B slots (1 KB aligned) | stages (tile, then x rows) | row exchange | descriptors |
    //         barriers | row info | TMEM address | abort flag
    unsigned char *bslots = tf_smem;
    unsigned char *stages = bslots + size_t(kTfAslots) * kB;
    float *xch = reinterpret_cast<float *>(stages + size_t(ns) * kStage);  // [2][NP][64]
    StreamDesc *sdesc = reinterpret_cast<StreamDesc *>(xch + 2 * 64 * NP);
    StreamDesc *adesc = sdesc + ns;         // [kTfAslots] descriptor of the block in each slot pair
    StreamDesc *dbuf = adesc + kTfAslots;   // [2][kChunkDesc]
    uint64_t *full = reinterpret_cast<uint64_t *>(dbuf + 2 * kChunkDesc);
    uint64_t *empty = full + ns;
    uint64_t *dbar = empty + ns;     // [2]
    uint64_t *rowdone = dbar + 2;    // [2]
    uint64_t *accfree = rowdone + 2; // [2]
    uint64_t *fin = accfree + 2;     // the issuer's last MMAs have completed
    uint64_t *xready = fin + 1;      // [2] warps 2-3 have written their row sums
    uint64_t *xfree = xready + 2;    // [2] warps 0-1 have read them
    uint64_t *afull = xfree + 2;              // [kTfAslots] the converters have filled a slot pair
    uint64_t *afree = afull + kTfAslots;      // [kTfAslots] the MMAs reading a slot pair have completed
    TcRowInfo *rowinfo = reinterpret_cast<TcRowInfo *>(afree + kTfAslots);  // [2]
    uint32_t *taddr_s = reinterpret_cast<uint32_t *>(rowinfo + 2);
    int *abort_flag = reinterpret_cast<int *>(taddr_s + 1);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) {
        for (int i = 0; i < ns; ++i) {
            h2p::mbar_init(&full[i], 1);
            h2p::mbar_init(&empty[i], kTfConverters);  // lane 0 of every converter warp
        }
        h2p::mbar_init(&dbar[0], 1);
        h2p::mbar_init(&dbar[1], 1);
        for (int i = 0; i < 2; ++i) {
            h2p::mbar_init(&rowdone[i], 2);  // the issuer's arrive + its tcgen05.commit
            h2p::mbar_init(&accfree[i], 4);  // the four epilogue warps
            h2p::mbar_init(&xready[i], 2);   // lane 0 of warps 2 and 3
            h2p::mbar_init(&xfree[i], 2);    // lane 0 of warps 0 and 1
        }
        for (int i = 0; i < kTfAslots; ++i) {
            h2p::mbar_init(&afull[i], kTfConverters);
            h2p::mbar_init(&afree[i], 1);    // the issuer's tcgen05.commit
        }
        h2p::mbar_init(fin, 1);
        *abort_flag = 0;
        h2p::fence_barrier_init();
    }
    if (warp == 0) h2t::tmem_alloc(taddr_s, tf_tmem_cols(NP));
    h2t::fence_before_sync();
    __syncthreads();
    h2t::fence_after_sync();
    const uint32_t tmem = *taddr_s;

    constexpr int kProducerWarp = 4 + kTfGroups * kTfConverters, kMmaWarp = kProducerWarp + 1;
    if (warp == kProducerWarp) {
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
            auto put = [&](const StreamDesc &d) -> bool {
                if (!h2p::mbar_wait(&empty[stage], phase ^ 1u, abort_flag, a.err)) return false;
                sdesc[stage] = d;
                unsigned char *st = stages + size_t(stage) * kStage;
                if (d.flags & (kZero | kEnd)) {
                    h2p::mbar_arrive(&full[stage]);
                } else {
                    const bool dense = d.flags & kDense;
                    const int xld = dense ? a.mp : a.kx;
                    const float *x = (dense ? a.xt : a.xh) + int64_t(d.x_node) * xld * a.nv;
                    const uint32_t tb = uint32_t(d.ld) * uint32_t(d.cols) * 4u;  // <= kTfTileBytes
                    const uint32_t xb = uint32_t(xld) * uint32_t(a.nv) * 4u;    // <= tf_x_bytes(NP)
                    h2p::mbar_arrive_expect_tx(&full[stage], tb + xb);
                    h2p::bulk_g2s(st, a.vals + d.src, tb, &full[stage]);
                    h2p::bulk_g2s(st + kTfTileBytes, x, xb, &full[stage]);
                    issued |= 1u << stage;
                    parity = (parity & ~(1u << stage)) | (phase << stage);
                }
                if (++stage == ns) {
                    stage = 0;
                    phase ^= 1u;
                }
                return true;
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
                    ok = put(dbuf[slot * kChunkDesc + i]);
                }
                slot ^= 1;
                tA = tB;
                recA = recB;
                tB = tC;
            }
            if (ok) {  // one end marker per converter group (each sees every other descriptor)
                StreamDesc end{};
                end.flags = kEnd;
                for (int g = 0; ok && g < kTfGroups; ++g) ok = put(end);
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
    } else if (warp >= 4 && warp < kProducerWarp) {
        // ------------------------------------------------------------ converters
        const int gw = warp - 4;
        const int g = gw / kTfConverters;  // group: descriptors j = g, g + 2, g + 4, ...
        const int q = warp & 3;            // TMEM lane quarter of this warp
        const int h = (gw % kTfConverters) >> 2;  // column half of this warp
        const bool lo_rows = q >= 2;       // A rows 64..127: S_lo
        const int r = 32 * (q & 1) + lane; // tile row of this thread
        const int ct = (gw % kTfConverters) * 32 + lane;  // 0..255 within the group
        const uint32_t lanes = uint32_t(32 * q) << 16;
        // this thread's float4 items of the B slot (vector row fv, columns 4 fk .. 4 fk + 3):
        // their shared-memory offsets do not change from block to block
        constexpr int kItems = NP * 16 / 256;
        uint32_t bhi[kItems], blo[kItems], xk[kItems], xm[kItems];
        int c4[kItems];
        bool vrow[kItems];
#pragma unroll
        for (int it = 0; it < kItems; ++it) {
            const int f = ct + 256 * it;
            const int fv = f >> 4, fk = f & 15;
            bhi[it] = sw128_tf32(fv, 4 * fk, 2 * NP);
            blo[it] = sw128_tf32(NP + fv, 4 * fk, 2 * NP);
            xk[it] = uint32_t(fv * a.kx + 4 * fk);
            xm[it] = uint32_t(fv * a.mp + 4 * fk);
            c4[it] = 4 * fk;
            vrow[it] = fv < a.nv;
        }
        for (int64_t j = g;; j += kTfGroups) {
            const int stage = int(j % ns), aslot = int(j % kTfAslots);
            const uint32_t phase = uint32_t(j / ns) & 1u, aphase = uint32_t(j / kTfAslots) & 1u;
            if (!h2p::mbar_wait(&full[stage], phase, abort_flag, a.err)) break;
            const StreamDesc d = sdesc[stage];
            // every descriptor takes a slot pair, so that it reaches the MMA issuer in order
            if (!h2p::mbar_wait(&afree[aslot], aphase ^ 1u, abort_flag, a.err)) break;
            h2t::fence_after_sync();
            if (!(d.flags & (kZero | kEnd))) {
                const unsigned char *st = stages + size_t(stage) * kStage;
                const float *tile = reinterpret_cast<const float *>(st);
                const int R = d.rows, C = d.cols, ld = d.ld;
                const bool full_tile = R == 64 && C == 64 && ld == 64;  // rank 64 / 64-point leaves
                const float *trow = tile + r;
                const uint32_t ta = tmem + kAcol + 64u * uint32_t(aslot) + lanes;
#pragma unroll
                for (int c0 = 32 * h; c0 < 32 * h + 32; c0 += 16) {
                    float x[16];
                    if (full_tile) {
#pragma unroll
                        for (int e = 0; e < 16; ++e) x[e] = trow[(c0 + e) * 64];
                    } else {
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            const int c = c0 + e;
                            x[e] = (r < R && c < C) ? tile[c * ld + r] : 0.f;
                        }
                    }
                    uint32_t v[16];
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const uint32_t hi = __float_as_uint(x[e]) & 0xFFFFE000u;
                        v[e] = lo_rows ? __float_as_uint(x[e] - __uint_as_float(hi)) : hi;
                    }
                    h2t::tmem_st16(ta + uint32_t(c0), v);
                }
                // B = [x_hi; x_lo]: rows v (hi) and NP + v (lo), K-blocks of 32 columns, 128-byte
                // swizzle; four consecutive columns per item, zero beyond the block's columns
                // and beyond the pass's vectors
                const bool dense = d.flags & kDense;
                const float *xs = reinterpret_cast<const float *>(st + kTfTileBytes);
                unsigned char *b = bslots + size_t(aslot) * kB;
#pragma unroll
                for (int it = 0; it < kItems; ++it) {
                    float4 xv = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (vrow[it]) {
                        const float *src = xs + (dense ? xm[it] : xk[it]);
                        if (c4[it] + 4 <= C) {
                            xv = *reinterpret_cast<const float4 *>(src);
                        } else if (c4[it] < C) {
                            float *dst = &xv.x;
                            for (int e = 0; e < 4; ++e)
                                if (c4[it] + e < C) dst[e] = src[e];
                        }
                    }
                    float4 hv, lv;
                    split_tf32(xv.x, hv.x, lv.x);
                    split_tf32(xv.y, hv.y, lv.y);
                    split_tf32(xv.z, hv.z, lv.z);
                    split_tf32(xv.w, hv.w, lv.w);
                    *reinterpret_cast<float4 *>(b + bhi[it]) = hv;
                    *reinterpret_cast<float4 *>(b + blo[it]) = lv;
                }
                h2p::fence_proxy_async_shared();  // B is read by the MMA (async proxy)
            }
            if (gw % kTfConverters == 0 && lane == 0) adesc[aslot] = d;
            __syncwarp();
            if (lane == 0) h2p::mbar_arrive(&empty[stage]);  // the stage has been read
            if (d.flags & kEnd) {
                if (lane == 0) h2p::mbar_arrive(&afull[aslot]);
                break;
            }
            h2t::tmem_wait_st();
            h2t::fence_before_sync();
            __syncwarp();
            if (lane == 0) h2p::mbar_arrive(&afull[aslot]);
        }
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = h2t::idesc_tf32_f32(128, 2 * NP);
            constexpr uint32_t kKb = 2u * NP * 128u;  // bytes of one 32-column K-block of B
            int aslot = 0;
            uint32_t aphase = 0;
            int acc = 0;              // accumulator slot
            uint32_t accphase = 0;    // parity of the slot's accfree phase to wait for
            bool fresh = true;        // next block starts a row
            for (;;) {
                if (!h2p::mbar_wait(&afull[aslot], aphase, abort_flag, a.err)) break;
                h2t::fence_after_sync();
                const StreamDesc d = adesc[aslot];
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
                    const unsigned char *bt = bslots + size_t(aslot) * kB;  // [x_hi; x_lo]
                    const uint32_t at = tmem + kAcol + 64u * uint32_t(aslot);
                    const uint32_t dt = tmem + uint32_t(acc * 2 * NP);
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk) {
                        const uint64_t bd = h2t::smem_desc_sw128(bt + (kk >> 2) * kKb) + uint64_t(2 * (kk & 3));
                        h2t::mma_tf32_ts(dt, at + uint32_t(8 * kk), bd, idesc, (fresh && kk == 0) ? 0u : 1u);
                    }
                    fresh = false;
                } else {
                    fresh = true;  // a zero row is a whole row by itself
                }
                h2t::commit(&afree[aslot]);  // slot pair free once these MMAs have read it
                if (++aslot == kTfAslots) {
                    aslot = 0;
                    aphase ^= 1u;
                }
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
    if (warp == 0) h2t::tmem_dealloc(tmem, tf_tmem_cols(NP));
}

}  // namespace h2s
