// h2_batch.cuh -- one persistent launch over the block rows of many operators.
//
// A batch of products of uneven operators is a set of independent instances of Sec. 3's
// three phases. The coupling rows of every level and the dense rows of every operator
// (Alg 4 and the dense product) are merged into one descriptor list -- each descriptor
// carries its operator's index -- handed out in chunks of whole rows by an atomic ticket,
// like the single-operator stream (k_stream). A CTA reads the operator's table entry for
// each descriptor: its block values, its coefficient and leaf vector trees, their strides
// and its number of vectors.
#pragma once

#include "h2_stream.cuh"

namespace h2s {

template <typename T>
struct BatchOp {
    const unsigned char *vals;  // the operator's block values
    const T *xh, *xt;           // input trees: [node][v][kx], [leaf][v][mp]
    T *yh, *yd;                 // output trees, same layouts
    int kx, mp;
    int vs;                     // vectors per node in the trees
    int nv;                     // vectors of this product
};

// Operator index of a merged descriptor (the descriptor's spare 32-bit field).
__host__ __device__ inline int batch_op(const StreamDesc &d) { return d.pad1; }

template <typename T, int NVMAX>
__global__ void __launch_bounds__(kThreads, 1)
    k_stream_batch(const BatchOp<T> *__restrict__ ops, Pipe pp, const StreamDesc *__restrict__ desc,
                   const int64_t *__restrict__ chunks, int64_t nchunks, int *ticket, int *err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // the widest operator's strides size the vector slots (the same carve for every CTA)
    Smem<T> s = carve<T, NVMAX>(smem_raw, pp, 0, 0, true);
    init_pipe(s, pp);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const uint32_t es = sizeof(T);
    Ring ring(pp.ns);

    if (warp == 4) {
        if (lane == 0) {
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
                ok = h2p::mbar_wait(&s.dbar[slot], dphase >> slot & 1u, s.abort_flag, err);
                dphase ^= 1u << slot;
                const int cnt = int(recA & 0xffff);
                const int pre = cnt - 1 < 4 ? cnt - 1 : 4;
                for (int i = 0; ok && i < cnt; ++i) {
                    if (i == pre && tB < nchunks) fetch_desc(slot ^ 1, recB);
                    const StreamDesc d = s.dbuf[slot * kChunkDesc + i];
                    if (d.flags & kZero) {
                        ok = produce(s, pp, ring, nullptr, 0, nullptr, 0, nullptr, 0, &d, err);
                    } else {
                        const BatchOp<T> &o = ops[batch_op(d)];
                        const bool dense = d.flags & kDense;
                        const uint32_t tb = (uint32_t(d.ld) * d.cols * es + 15u) & ~15u;
                        const T *x = dense ? o.xt + int64_t(d.x_node) * o.mp * o.vs : o.xh + int64_t(d.x_node) * o.kx * o.vs;
                        const uint32_t xb = uint32_t(dense ? o.mp : o.kx) * o.nv * es;
                        ok = produce(s, pp, ring, o.vals + d.src, tb, x, xb, nullptr, 0, &d, err);
                    }
                }
                slot ^= 1;
                tA = tB;
                recA = recB;
                tB = tC;
            }
            if (ok && h2p::mbar_wait(&s.empty[ring.stage], ring.phase ^ 1u, s.abort_flag, err)) {
                s.desc[ring.stage].flags = kEnd;
                h2p::mbar_arrive(&s.full[ring.stage]);
            }
            drain_on_abort(s, ring);
        }
        return;
    }

    const int tid = threadIdx.x;
    AccStreamOf<T, NVMAX> acc;
    bool fresh = true;
    for (;;) {
        if (!h2p::mbar_wait(&s.full[ring.stage], ring.phase, s.abort_flag, err)) return;
        const StreamDesc d = s.desc[ring.stage];
        if (d.flags & kEnd) break;
        const BatchOp<T> &o = ops[batch_op(d)];
        const bool dense = d.flags & kDense;
        const int xld = dense ? o.mp : o.kx;
        if (fresh) {
            acc.setup(d.rows, d.ld, tid);
            acc.zero();
            fresh = false;
        }
        if (!(d.flags & kZero))
            acc.gemv(stage_tile(s, pp, ring.stage), d.ld, d.rows, d.cols, stage_x(s, pp, ring.stage), xld, o.nv);
        release(&s.empty[ring.stage], lane);
        ring.next();
        if (d.flags & kLast) {
            if (acc.reduce(d.rows, o.nv, s.red)) {
                T *out = dense ? o.yd + int64_t(d.out_node) * o.mp * o.vs : o.yh + int64_t(d.out_node) * o.kx * o.vs;
                acc.store(out, xld, o.nv, d.rows);
            }
            h2p::consumer_sync(kConsumers);
            fresh = true;
        }
    }
}

// ------------------------------------------------------------------ merged sweeps
//
// The members' up- and downsweeps run as merged launches too: one launch per sweep step and
// accumulator width over a task table (one SweepTask per member, its items numbered after
// the previous member's), so a batch takes a few launches per width instead of a dozen per
// member. The subtree steps are k_up_batch / k_down_batch (h2_stream.cuh); the gathers and
// the row-major staging of wide passes are below, one item per leaf or per 32-point tile.

// Members' gathers: xt[leaf][v][i] = X[v n + perm[..]] (narrow passes, as k_gather) or from
// the row-major staging copy (wide passes, as k_gather_rows). Resets each member's tickets.
template <typename T>
__global__ void k_gather_batch(const SweepTask<T> *__restrict__ tasks, int ntasks, int64_t total, int rows)
{
    __shared__ T buf[64 * 33];
    for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
        const SweepTask<T> &t = tasks[sweep_task_of(tasks, ntasks, g)];
        const Op<T> &op = t.op;
        const Vec<T> &vec = t.vec;
        const int64_t leaf = g - t.first;
        if (leaf == 0 && threadIdx.x < kTickets) vec.tickets[threadIdx.x] = 0;
        const int r0 = op.leaf_lo[leaf], R = op.leaf_lo[leaf + 1] - r0;
        if (!rows) {
            for (int e = threadIdx.x; e < R * vec.nv; e += blockDim.x) {
                const int i = e % R, v = e / R;
                vec.xt[(leaf * vec.vs + v) * op.mp + i] = vec.X[int64_t(v) * op.n + op.perm[r0 + i]];
            }
        } else {
            for (int e = threadIdx.x; e < R * vec.nv; e += blockDim.x) {
                const int i = e / vec.nv, v = e % vec.nv;
                buf[i * 33 + v] = vec.xr[int64_t(op.perm[r0 + i]) * vec.ldr + v];
            }
            __syncthreads();
            for (int e = threadIdx.x; e < R * vec.nv; e += blockDim.x) {
                const int v = e / R, i = e % R;
                vec.xt[(leaf * vec.vs + v) * op.mp + i] = buf[i * 33 + v];
            }
            __syncthreads();
        }
    }
}

// Members' row-major staging of X (as k_rows_in; nv <= 32): one 32-point tile per item.
// Block 32 x 8.
template <typename T>
__global__ void k_rows_in_batch(const SweepTask<T> *__restrict__ tasks, int ntasks, int64_t total)
{
    __shared__ T tt[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
        const SweepTask<T> &t = tasks[sweep_task_of(tasks, ntasks, g)];
        const int64_t n = t.op.n, u0 = (g - t.first) * 32;
        const int nv = t.vec.nv, ldr = t.vec.ldr;
        for (int j = ty; j < 32; j += 8) {
            const int64_t u = u0 + tx;
            if (u < n && j < nv) tt[j][tx] = t.vec.X[int64_t(j) * n + u];
        }
        __syncthreads();
        for (int j = ty; j < 32; j += 8) {
            const int64_t u = u0 + j;
            if (u < n && tx < nv) t.vec.xr[u * ldr + tx] = tt[tx][j];
        }
        __syncthreads();
    }
}

// Members' epilogue of wide passes (as k_rows_out): Y[v n + u] = alpha yr[u ldr + v] + beta
// Y[v n + u], Y not read when beta = 0. Block 32 x 8.
template <typename T>
__global__ void k_rows_out_batch(const SweepTask<T> *__restrict__ tasks, int ntasks, int64_t total)
{
    __shared__ T tt[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
        const SweepTask<T> &t = tasks[sweep_task_of(tasks, ntasks, g)];
        const int64_t n = t.op.n, u0 = (g - t.first) * 32;
        const int nv = t.vec.nv, ldr = t.vec.ldr;
        const T alpha = t.vec.alpha, beta = t.vec.beta;
        for (int j = ty; j < 32; j += 8) {
            const int64_t u = u0 + j;
            if (u < n && tx < nv) tt[j][tx] = t.vec.yr[u * ldr + tx];
        }
        __syncthreads();
        for (int j = ty; j < 32; j += 8) {
            const int64_t u = u0 + tx;
            if (u < n && j < nv) {
                T *dst = t.vec.Y + int64_t(j) * n + u;
                const T y = tt[tx][j];
                *dst = (beta == T(0)) ? alpha * y : alpha * y + beta * *dst;
            }
        }
        __syncthreads();
    }
}

}  // namespace h2s
