// h2_mf.cuh -- matrix-free block rows: coupling and dense entries evaluated in the product.
//
// The coupling block S_ts[nu][mu] = kappa(xi^t_nu, xi^s_mu) (Chebyshev points of the two
// clusters, Sec. 2.1) and the dense block D_ts[i][j] = kappa(x_i, x_j) (Sec. 2) are never
// stored: the stream hands out the same block rows as the stored path (Alg 4 and the dense
// product), and each consumer thread evaluates the entries it needs in FP32 and accumulates
// them at once -- per entry one kernel evaluation instead of four bytes from HBM. The
// producer bulk-copies, per block, the column cluster's point coordinates (float4 per
// point) and its input segment, and at each row start the row cluster's coordinates.
//
// Thread layout (as the narrow accumulator): 16 output lanes x 8 column groups; lane l owns
// outputs 4l .. 4l+3 and group g the columns g, g+8, ...; the groups are summed in a fixed
// order at the end of the row, so the result is deterministic.
#pragma once

#include "../../include/h2.h"
#include "h2_stream.cuh"

namespace h2s {

struct MfArgs {
    const float4 *node_pts;  // [node][k]: Chebyshev points of every cluster (x, y, z, 0)
    const float4 *leaf_pts;  // [leaf][mp]: the points of every leaf in tree order
    int k;
    int p, lp;               // points per dimension of the Chebyshev grids, log2(p) (or -1)
    int dim;                 // coordinates per point
    float a, neg_inv_a, neg_b;  // kernel parameters: a, -1/a, -b
    int deg;
};

// kappa in FP32 through CUDA's fast intrinsics. DIM = 2 serves points of one or two
// coordinates (the unused ones are zero: nothing to a distance, a factor 1 to a product),
// DIM = 3 points of three.
template <int KIND, int DIM>
__device__ __forceinline__ float mf_kernel(const float (&x)[3], const float4 &y, const MfArgs &a)
{
    if constexpr (KIND == H2_K_POLY) {
        float g = (1.f + x[0] * y.x) * (1.f + x[1] * y.y);
        if constexpr (DIM == 3) g *= 1.f + x[2] * y.z;
        float v = 1.f;
        for (int e = 0; e < a.deg; ++e) v *= g;
        return v;
    } else {
        const float dx = x[0] - y.x, dy = x[1] - y.y;
        float r2 = dx * dx + dy * dy;
        if constexpr (DIM == 3) {
            const float dz = x[2] - y.z;
            r2 += dz * dz;
        }
        if constexpr (KIND == H2_K_GAUSS) {
            return __expf(r2 * a.neg_inv_a);
        } else if constexpr (KIND == H2_K_EXP) {
            const float r = r2 > 0.f ? r2 * rsqrtf(r2) : 0.f;
            return __expf(r * a.neg_inv_a);
        } else {  // H2_K_IMQ
            return __powf(r2 + a.a, a.neg_b);
        }
    }
}

// One-dimensional factor of a separable kernel: kappa(x, y) = prod_d f(x_d, y_d) for the
// Gaussian (f = exp(-(x_d - y_d)^2 / a)) and the product kernel (f = (1 + x_d y_d)^deg).
template <int KIND>
__device__ __forceinline__ float mf_factor(float x, float y, const MfArgs &a)
{
    if constexpr (KIND == H2_K_GAUSS) {
        const float d = x - y;
        return __expf(d * d * a.neg_inv_a);
    } else {
        const float g = 1.f + x * y;
        float v = 1.f;
        for (int e = 0; e < a.deg; ++e) v *= g;
        return v;
    }
}

__device__ __forceinline__ float coord(const float4 &p, int d) { return d == 0 ? p.x : (d == 1 ? p.y : p.z); }

// Shared-memory bytes of one stage's vector region: input segment, column coordinates, row
// coordinates.
__host__ __device__ inline uint32_t mf_seg_bytes(int kx, int mp, int nvmax)
{
    return uint32_t((kx > mp ? kx : mp) * nvmax * 4);
}
__host__ __device__ inline uint32_t mf_coord_bytes(int k, int mp) { return uint32_t((k > mp ? k : mp) * 16); }

template <int KIND, int DIM, int NVMAX>
__global__ void __launch_bounds__(kThreads, 4)
    k_stream_mf(Op<float> op, Vec<float> vec, MfArgs ma, Pipe pp, const StreamDesc *__restrict__ desc,
                const int64_t *__restrict__ chunks, int64_t nchunks, int ticket_index)
{
    static_assert(NVMAX <= 4, "the matrix-free stream runs passes of at most four vectors");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem<float> s = carve<float, NVMAX>(smem_raw, pp, 0, op.kx, true);
    init_pipe(s, pp);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int kx = op.kx, mp = op.mp, nv = vec.nv, vs = vec.vs;
    const uint32_t seg = mf_seg_bytes(kx, mp, NVMAX), cb = mf_coord_bytes(ma.k, mp);
    Ring ring(pp.ns);

    if (warp == 4) {
        if (lane == 0) {
            int *ticket = vec.tickets + ticket_index;
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
            uint32_t dphase = 0;
            bool ok = true;
            if (tA < nchunks) fetch_desc(0, recA);
            while (ok && tA < nchunks) {
                const int64_t recB = tB < nchunks ? chunks[tB] : 0;
                const int64_t tC = atomicAdd(ticket, 1);
                ok = h2p::mbar_wait(&s.dbar[slot], dphase >> slot & 1u, s.abort_flag, vec.err);
                dphase ^= 1u << slot;
                const int cnt = int(recA & 0xffff);
                const int pre = cnt - 1 < 4 ? cnt - 1 : 4;
                bool row_start = true;  // chunks hold whole rows
                for (int i = 0; ok && i < cnt; ++i) {
                    if (i == pre && tB < nchunks) fetch_desc(slot ^ 1, recB);
                    const StreamDesc d = s.dbuf[slot * kChunkDesc + i];
                    ok = h2p::mbar_wait(&s.empty[ring.stage], ring.phase ^ 1u, s.abort_flag, vec.err);
                    if (!ok) break;
                    s.desc[ring.stage] = d;
                    unsigned char *xs = s.xs + size_t(ring.stage) * pp.x_bytes;
                    uint32_t bytes = 0;
                    const void *xsrc = nullptr, *csrc = nullptr, *rsrc = nullptr;
                    uint32_t xb = 0, cbytes = 0, rbytes = 0;
                    if (!(d.flags & kZero)) {
                        const bool dense = d.flags & kDense;
                        xsrc = dense ? static_cast<const void *>(vec.xt + int64_t(d.x_node) * mp * vs)
                                     : static_cast<const void *>(vec.xh + int64_t(d.x_node) * kx * vs);
                        xb = uint32_t((dense ? mp : kx) * nv * 4);
                        csrc = dense ? static_cast<const void *>(ma.leaf_pts + int64_t(d.x_node) * mp)
                                     : static_cast<const void *>(ma.node_pts + int64_t(d.x_node) * ma.k);
                        cbytes = uint32_t(d.cols) * 16u;
                        if (row_start) {
                            rsrc = dense ? static_cast<const void *>(ma.leaf_pts + int64_t(d.out_node) * mp)
                                         : static_cast<const void *>(ma.node_pts + int64_t(d.out_node) * ma.k);
                            rbytes = uint32_t(d.rows) * 16u;
                        }
                        bytes = xb + cbytes + rbytes;
                    }
                    h2p::mbar_arrive_expect_tx(&s.full[ring.stage], bytes);
                    if (xb) h2p::bulk_g2s(xs, xsrc, xb, &s.full[ring.stage]);
                    if (cbytes) h2p::bulk_g2s(xs + seg, csrc, cbytes, &s.full[ring.stage]);
                    if (rbytes) h2p::bulk_g2s(xs + seg + cb, rsrc, rbytes, &s.full[ring.stage]);
                    if (bytes) {
                        ring.issued |= 1u << ring.stage;
                        ring.parity = (ring.parity & ~(1u << ring.stage)) | (ring.phase << ring.stage);
                    }
                    row_start = (d.flags & kLast) != 0;
                    ring.next();
                }
                slot ^= 1;
                tA = tB;
                recA = recB;
                tB = tC;
            }
            if (ok && h2p::mbar_wait(&s.empty[ring.stage], ring.phase ^ 1u, s.abort_flag, vec.err)) {
                s.desc[ring.stage].flags = kEnd;
                h2p::mbar_arrive(&s.full[ring.stage]);
            }
            drain_on_abort(s, ring);
        }
        return;
    }

    const int tid = threadIdx.x;
    Acc<float, NVMAX> acc;
    float tc[4][3];  // row coordinates of this thread's four outputs
    // Separable kernels on Chebyshev tensor grids: a coupling block is the Kronecker product
    // S = F_{dim-1} x ... x F_0 of p x p factor tables, F_d[a][b] = f(xi^t_{d,a}, xi^s_{d,b}),
    // so a block needs dim p^2 evaluations instead of k^2. With 4 | p a thread's four outputs
    // share their higher digits, and with p | G (G column groups) all of a thread's columns
    // share their digit 0: entry (nu, mu) = A_e B(mu) with A_e = F_0[nu_0(e)][mu_0] fixed
    // per block and B(mu) = prod_{d>=1} F_d[nu_d][mu_d].
    constexpr bool kSeparable = KIND == H2_K_GAUSS || KIND == H2_K_POLY;
    __shared__ float row1d[3][8];   // the row cluster's grid coordinates per dimension
    __shared__ float fac[2][3][64]; // factor tables, double-buffered by block parity
    int fbuf = 0;
    bool sep_row = false;
    int nu0[4] = {0, 0, 0, 0}, nuhi[3] = {0, 0, 0};
    bool fresh = true;
    for (;;) {
        if (!h2p::mbar_wait(&s.full[ring.stage], ring.phase, s.abort_flag, vec.err)) return;
        const StreamDesc d = s.desc[ring.stage];
        if (d.flags & kEnd) break;
        const bool dense = d.flags & kDense;
        const int xld = dense ? mp : kx;
        const unsigned char *xs = s.xs + size_t(ring.stage) * pp.x_bytes;
        const float *xv = reinterpret_cast<const float *>(xs);
        const float4 *cc = reinterpret_cast<const float4 *>(xs + seg);
        if (fresh) {
            acc.setup(d.rows, d.ld, tid);  // ld is a multiple of 4: four outputs per lane
            acc.zero();
            sep_row = false;
            if (!(d.flags & kZero)) {
                const float4 *rc = reinterpret_cast<const float4 *>(xs + seg + cb);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float4 p = rc[acc.o0 + e < d.rows ? acc.o0 + e : 0];
                    tc[e][0] = p.x;
                    tc[e][1] = p.y;
                    tc[e][2] = p.z;
                }
                if constexpr (kSeparable) {
                    const int P = ma.p;
                    sep_row = !dense && ma.dim == DIM && ma.lp >= 2 && (acc.G % P) == 0 && P <= 8;
                    if (sep_row) {
                        if (tid < (DIM << ma.lp)) {
                            const int dd = tid >> ma.lp, aa = tid & (P - 1);
                            row1d[dd][aa] = coord(rc[aa << (ma.lp * dd)], dd);
                        }
#pragma unroll
                        for (int e = 0; e < 4; ++e) nu0[e] = (acc.o0 + e) & (P - 1);
#pragma unroll
                        for (int dd = 1; dd < 3; ++dd) nuhi[dd] = (acc.o0 >> (ma.lp * dd)) & (P - 1);
                        h2p::consumer_sync(kConsumers);
                    }
                }
            }
            fresh = false;
        }
        if (!(d.flags & kZero)) {
            bool done = false;
            if constexpr (kSeparable) {
                if (sep_row) {
                    const int P = ma.p, lp = ma.lp;
                    for (int e = tid; e < (DIM << (2 * lp)); e += kConsumers) {  // P is a power of two here
                        const int dd = e >> (2 * lp), aa = (e >> lp) & (P - 1), bb = e & (P - 1);
                        fac[fbuf][dd][(aa << lp) + bb] = mf_factor<KIND>(row1d[dd][aa], coord(cc[bb << (lp * dd)], dd), ma);
                    }
                    h2p::consumer_sync(kConsumers);
                    if (acc.o0 < d.rows) {
                        const int mu0 = acc.g & (P - 1);
                        float A[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) A[e] = fac[fbuf][0][(nu0[e] << lp) + mu0];
#pragma unroll 2
                        for (int j = acc.g; j < d.cols; j += acc.G) {
                            float B = fac[fbuf][1][(nuhi[1] << lp) + ((j >> lp) & (P - 1))];
                            if constexpr (DIM == 3) B *= fac[fbuf][2][(nuhi[2] << lp) + ((j >> (2 * lp)) & (P - 1))];
#pragma unroll
                            for (int v = 0; v < NVMAX; ++v) {
                                if (v >= nv) break;
                                const float t = B * xv[v * xld + j];
#pragma unroll
                                for (int e = 0; e < 4; ++e) acc.a[v][e] += A[e] * t;
                            }
                        }
                    }
                    fbuf ^= 1;
                    done = true;
                }
            }
            if (!done && acc.o0 < d.rows) {
#pragma unroll 2
                for (int j = acc.g; j < d.cols; j += acc.G) {
                    const float4 c = cc[j];
                    float xj[NVMAX];
#pragma unroll
                    for (int v = 0; v < NVMAX; ++v) xj[v] = v < nv ? xv[v * xld + j] : 0.f;
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float kv = mf_kernel<KIND, DIM>(tc[e], c, ma);
#pragma unroll
                        for (int v = 0; v < NVMAX; ++v) acc.a[v][e] += kv * xj[v];
                    }
                }
            }
        }
        release(&s.empty[ring.stage], lane);
        ring.next();
        if (d.flags & kLast) {
            if (acc.reduce(d.rows, nv, s.red)) {
                float *out = dense ? vec.yd + int64_t(d.out_node) * mp * vs : vec.yh + int64_t(d.out_node) * kx * vs;
                acc.store(out, xld, nv, d.rows);
            }
            h2p::consumer_sync(kConsumers);
            fresh = true;
        }
    }
}

// Coordinates for the matrix-free stream: every cluster's Chebyshev points (multi-index
// nu = j0 + p j1 + p^2 j2, Sec. 2.1) and every leaf's points, as float4 with zeros beyond dim.
__global__ void k_mf_node_points(const double *__restrict__ cheb, int64_t nodes, int dim, int p, int k,
                                        float4 *__restrict__ out)
{
    const int64_t total = nodes * k;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t t = e / k;
        int nu = int(e % k);
        float c[3] = {0.f, 0.f, 0.f};
        for (int d = 0; d < dim; ++d) {
            c[d] = float(cheb[(t * dim + d) * p + nu % p]);
            nu /= p;
        }
        out[e] = make_float4(c[0], c[1], c[2], 0.f);
    }
}

__global__ void k_mf_leaf_points(const double *__restrict__ pts_tree, const int32_t *__restrict__ leaf_lo,
                                        int64_t nleaves, int dim, int mp, float4 *__restrict__ out)
{
    const int64_t total = nleaves * mp;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
        const int64_t l = e / mp;
        const int i = int(e % mp);
        const int r0 = leaf_lo[l], R = leaf_lo[l + 1] - r0;
        float c[3] = {0.f, 0.f, 0.f};
        if (i < R)
            for (int d = 0; d < dim; ++d) c[d] = float(pts_tree[(int64_t(r0) + i) * dim + d]);
        out[e] = make_float4(c[0], c[1], c[2], 0.f);
    }
}

}  // namespace h2s
