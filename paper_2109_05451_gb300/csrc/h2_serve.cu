// h2_serve.cu -- serving loop of CG solves on resident H^2 operators with continuous batching.
//
// Requests (operator, b, sigma2, tol, maxit) queue in FIFO order and are admitted as soon as
// a solve slot and enough slot memory are free ("admission by footprint"). Every admitted
// solve advances on its own CUDA stream with its own product workspace and fork/join
// context, so solves admitted while others run overlap them on the device. The solve is
// unpreconditioned CG from x0 = 0 with the kernels and the order of operations of
// h2_cg_solve (h2_cgk.cuh): step lengths and the stopping test are evaluated on the device,
// so the scheduler never blocks on a solve -- it keeps up to kAhead iterations enqueued per
// slot and reads each iteration's state (flag, count, scalars) from pinned memory once the
// iteration's event has completed. Iterations enqueued after the device set the converged
// flag leave x untouched. The result of a request therefore does not depend on the other
// requests in flight, and equals h2_cg_solve's result bitwise.
//
// Refined requests (h2_server_submit_refined) run the same CG iterations as the inner solver
// of a mixed-precision iterative refinement: when an inner solve stops, one outer step
// (x_o += d, r = b - (A64 + sigma2 I) x_o with the FP64 operator) is enqueued, and the
// scheduler either finishes the request (FP64 residual below tol) or restarts the inner CG on
// r, with the same captured iteration graph.
//
// One scheduler thread per server drives all slots; the public calls only touch the
// request queue and the result list under a mutex.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "h2_cgk.cuh"
#include "h2_internal.h"
#include "h2_nvtx.h"

// device side of the server (a named namespace: nvcc's host stubs of kernels whose types
// live in an unnamed namespace clash with the unnamed namespace of h2_cgk.cuh)
namespace h2srv {

// Device state of one solve, copied to the host after every iteration.
struct Head {
    int flag;        // 0 running, 1 converged, 2 breakdown
    int iters;       // iterations applied
    double scal[8];  // see h2_cgk.cuh: [0] r.r [1] p.Ap [2] r.r new [3] b.b [4] true residual^2
                     // refined solves: [3] the inner right-hand side's r.r, [5] b.b
};

// x += d (the outer update of a refined solve)
__global__ void k_axpy(double *__restrict__ x, const double *__restrict__ d, int64_t n)
{
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        x[i] += d[i];
}

// Restart of a refined solve's inner CG on the outer residual r (already in r and p):
// r.r of the new right-hand side is both the inner r.r and its reference, the flag clears.
__global__ void k_restart(Head *h)
{
    h->scal[3] = h->scal[0];
    h->flag = 0;
}

// flag = 1 before the first iteration when b = 0 (x = 0 is the solution) or the initial
// residual already meets the tolerance (the tests of h2_cg_solve, in the same order).
__global__ void k_init(Head *h, double tol)
{
    const double bb = h->scal[3], rr = h->scal[0];
    if (bb == 0.0 || sqrt(rr / bb) < tol) h->flag = 1;
}

}  // namespace h2srv

namespace {

using namespace h2cg;
using h2srv::Head;
using Clock = std::chrono::steady_clock;

constexpr int kRing = 4;      // iteration snapshots per slot (> kAhead)
constexpr int kAhead = 2;     // iterations enqueued ahead of the host's look at their state
constexpr size_t kAl = 256;   // alignment of every region of slot memory
constexpr int kGraphMinIters = 8;  // requests allowing fewer iterations are launched eagerly

size_t al(size_t b) { return (b + kAl - 1) / kAl * kAl; }

// First-fit allocator over one device allocation; free ranges coalesce on release.
class Arena {
  public:
    int init(size_t bytes)
    {
        cap_ = al(bytes);
        if (cudaMalloc(&base_, cap_) != cudaSuccess) {
            cudaGetLastError();
            base_ = nullptr;
            return H2_ENOMEM;
        }
        free_[0] = cap_;
        return H2_OK;
    }
    void destroy()
    {
        if (base_) cudaFree(base_);
        base_ = nullptr;
        free_.clear();
    }
    size_t capacity() const { return cap_; }
    char *alloc(size_t bytes)
    {
        bytes = al(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const size_t off = it->first, sz = it->second;
            free_.erase(it);
            if (sz > bytes) free_[off + bytes] = sz - bytes;
            return base_ + off;
        }
        return nullptr;
    }
    void release(char *p, size_t bytes)
    {
        bytes = al(bytes);
        const size_t off = size_t(p - base_);
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && off + bytes == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }

  private:
    char *base_ = nullptr;
    size_t cap_ = 0;
    std::map<size_t, size_t> free_;  // offset -> bytes
};

struct Request {
    int64_t id = 0;
    h2_handle op = nullptr;
    h2_handle op64 = nullptr;  // refined solves: FP64 copy of the operator for the outer residuals
    double inner_tol = 0;      // refined solves: relative tolerance of each inner CG
    double sigma2 = 0, tol = 0;
    int maxit = 0;
    const double *b = nullptr;
    double *x = nullptr;
    int64_t n = 0;
    bool fp64 = false;
    size_t bytes = 0;
    double t_submit = 0;
};

struct Slot {
    bool busy = false, finishing = false;
    bool cancel = false;  // stop after the iterations already enqueued
    Request req;
    double t_admit = 0;
    int enq = 0, done = 0;
    int enq_cap = 0;  // iterations may be enqueued while enq < enq_cap
    cudaStream_t st = nullptr;
    h2_exec ex;
    cudaEvent_t ev[kRing] = {};
    cudaEvent_t ev_fin = nullptr;
    cudaGraphExec_t iter = nullptr;  // the captured iteration of the admitted request
    Head *ring = nullptr;     // pinned, kRing + 1 (the last: after the true residual)
    double *stage = nullptr;  // pinned, max_points doubles (b in, x out)
    // device regions, carved from the arena per request
    char *mem = nullptr;
    Head *head = nullptr;
    double *partial = nullptr, *b = nullptr, *x = nullptr, *r = nullptr, *p = nullptr, *Ap = nullptr;
    float *pf = nullptr, *Apf = nullptr;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    // refined solves: outer iterate, FP64 product workspace, the pending outer step
    double *xo = nullptr;
    void *ws64 = nullptr;
    size_t ws64_bytes = 0;
    bool outer_pending = false;
    cudaEvent_t ev_outer = nullptr;
};

size_t request_bytes(h2_handle h, bool fp64, int64_t n, h2_handle h64 = nullptr)
{
    const size_t nd = al(size_t(n) * 8), nf = al(size_t(n) * 4);
    return al(sizeof(Head)) + al(kDotBlocks * sizeof(double)) + 5 * nd + (fp64 ? 0 : 2 * nf) +
           al(h2_workspace_bytes(h, 1)) + (h64 ? nd + al(h2_workspace_bytes(h64, 1)) : 0);
}

int status_of(cudaError_t e) { return e == cudaSuccess ? H2_OK : (e == cudaErrorMemoryAllocation ? H2_ENOMEM : H2_ECUDA); }

}  // namespace

struct h2_server {
    int device = 0;
    int64_t max_points = 0;
    Arena arena;
    std::vector<Slot> slots;
    Head *ring_all = nullptr;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request> queue;
    std::vector<h2_request_result> results;
    std::vector<int64_t> inflight;  // ids admitted and not yet completed
    std::vector<int64_t> cancels;   // cancel requests for ids in flight
    int64_t next_id = 1;
    int64_t outstanding = 0;  // queued + in flight
    std::atomic<bool> stop{false};
    std::thread th;
    Clock::time_point t0;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

    // out = (A + sigma2 I) v on the slot's stream
    int apply(Slot &s, const double *v, double *out)
    {
        const Request &q = s.req;
        const int64_t n = q.n;
        int rc;
        if (q.fp64) {
            rc = h2_matvec_exec(q.op, v, out, 1, 1.0, 0.0, s.ws, s.ws_bytes, s.st, &s.ex);
            if (rc != H2_OK) return rc;
            k_shift<double><<<grid_for(n), kThreads, 0, s.st>>>(out, v, q.sigma2, out, n);
        } else {
            k_to_float<<<grid_for(n), kThreads, 0, s.st>>>(v, s.pf, n);
            rc = h2_matvec_exec(q.op, s.pf, s.Apf, 1, 1.0, 0.0, s.ws, s.ws_bytes, s.st, &s.ex);
            if (rc != H2_OK) return rc;
            k_shift<float><<<grid_for(n), kThreads, 0, s.st>>>(s.Apf, v, q.sigma2, out, n);
        }
        return status_of(cudaGetLastError());
    }

    // out = (A64 + sigma2 I) v with the refinement operator (FP64)
    int apply64(Slot &s, const double *v, double *out)
    {
        const Request &q = s.req;
        const int rc = h2_matvec_exec(q.op64, v, out, 1, 1.0, 0.0, s.ws64, s.ws64_bytes, s.st, &s.ex);
        if (rc != H2_OK) return rc;
        k_shift<double><<<grid_for(q.n), kThreads, 0, s.st>>>(out, v, q.sigma2, out, q.n);
        return status_of(cudaGetLastError());
    }

    // the stopping tolerance of the CG iterations: the request's, or a refined solve's inner one
    static double cg_tol(const Request &q) { return q.op64 ? q.inner_tol : q.tol; }

    int admit(Slot &s, const Request &q, char *mem)
    {
        h2n::Range range("h2_server: admit");
        s.busy = true;
        s.finishing = false;
        s.cancel = false;
        s.req = q;
        s.enq = s.done = 0;
        s.enq_cap = q.maxit;
        s.outer_pending = false;
        s.t_admit = now();
        s.mem = mem;
        const size_t nd = al(size_t(q.n) * 8), nf = al(size_t(q.n) * 4);
        char *m = mem;
        s.head = reinterpret_cast<Head *>(m);
        m += al(sizeof(Head));
        s.partial = reinterpret_cast<double *>(m);
        m += al(kDotBlocks * sizeof(double));
        double **vec[5] = {&s.b, &s.x, &s.r, &s.p, &s.Ap};
        for (double **v : vec) {
            *v = reinterpret_cast<double *>(m);
            m += nd;
        }
        s.pf = s.Apf = nullptr;
        if (!q.fp64) {
            s.pf = reinterpret_cast<float *>(m);
            m += nf;
            s.Apf = reinterpret_cast<float *>(m);
            m += nf;
        }
        s.ws = m;
        s.ws_bytes = h2_workspace_bytes(q.op, 1);
        m += al(s.ws_bytes);
        s.xo = nullptr;
        s.ws64 = nullptr;
        s.ws64_bytes = 0;
        if (q.op64) {
            s.xo = reinterpret_cast<double *>(m);
            m += nd;
            s.ws64 = m;
            s.ws64_bytes = h2_workspace_bytes(q.op64, 1);
        }
        const size_t bytes = size_t(q.n) * 8;
        std::memcpy(s.stage, q.b, bytes);
        cudaMemcpyAsync(s.b, s.stage, bytes, cudaMemcpyHostToDevice, s.st);
        cudaMemsetAsync(s.head, 0, sizeof(Head), s.st);
        cudaMemsetAsync(s.x, 0, bytes, s.st);
        // x0 = 0: r = b - (A + sigma2 I) 0 = b, p = r
        cudaMemcpyAsync(s.r, s.b, bytes, cudaMemcpyDeviceToDevice, s.st);
        cudaMemcpyAsync(s.p, s.b, bytes, cudaMemcpyDeviceToDevice, s.st);
        dot(s.r, s.r, q.n, s.partial, s.head->scal + 0, s.st);
        dot(s.b, s.b, q.n, s.partial, s.head->scal + 3, s.st);
        if (q.op64) {  // refined: x0 = 0 is the outer iterate, the inner CG starts on r = b
            cudaMemsetAsync(s.xo, 0, bytes, s.st);
            k_copy_scalar<<<1, 1, 0, s.st>>>(s.head->scal, 5, 3);
        }
        h2srv::k_init<<<1, 1, 0, s.st>>>(s.head, cg_tol(q));
        const int rc = status_of(cudaGetLastError());
        if (rc == H2_OK && q.maxit == 0) return q.op64 ? outer_step(s) : finish(s);
        return rc;
    }

    // One CG iteration's device work (product, inner products, updates, stopping test).
    int iteration_body(Slot &s)
    {
        const Request &q = s.req;
        const int64_t n = q.n;
        double *scal = s.head->scal;
        int rc = apply(s, s.p, s.Ap);
        if (rc != H2_OK) return rc;
        dot(s.p, s.Ap, n, s.partial, scal + 1, s.st);
        k_update_xr_if<<<grid_for(n), kThreads, 0, s.st>>>(s.x, s.r, s.p, s.Ap, scal, &s.head->flag, n);
        dot(s.r, s.r, n, s.partial, scal + 2, s.st);
        k_check<<<1, 1, 0, s.st>>>(scal, &s.head->flag, &s.head->iters, cg_tol(q));
        k_update_p_if<<<grid_for(n), kThreads, 0, s.st>>>(s.p, s.r, scal, &s.head->flag, n);
        k_roll_if<<<1, 1, 0, s.st>>>(scal, &s.head->flag);
        return status_of(cudaGetLastError());
    }

    // The iteration as a CUDA graph (its arguments are fixed for the request), captured after
    // one eager iteration has set up every kernel it launches; replaying it replaces about two
    // dozen launches per iteration. Without a graph the iteration is launched eagerly.
    void capture_iteration(Slot &s)
    {
        if (s.iter || s.req.maxit < kGraphMinIters) return;
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(s.st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        const int rc = iteration_body(s);
        const cudaError_t e = cudaStreamEndCapture(s.st, &g);
        if (rc == H2_OK && e == cudaSuccess && g && cudaGraphInstantiate(&s.iter, g, 0) != cudaSuccess) s.iter = nullptr;
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
    }

    int enqueue_iteration(Slot &s)
    {
        h2n::Range range("h2_server: CG iteration");
        int rc;
        if (s.iter) {
            rc = status_of(cudaGraphLaunch(s.iter, s.st));
        } else {
            rc = iteration_body(s);
            if (rc == H2_OK && s.enq == 0) capture_iteration(s);
        }
        if (rc != H2_OK) return rc;
        const int i = s.enq % kRing;
        cudaMemcpyAsync(&s.ring[i], s.head, sizeof(Head), cudaMemcpyDeviceToHost, s.st);
        cudaEventRecord(s.ev[i], s.st);
        ++s.enq;
        return status_of(cudaGetLastError());
    }

    // Refined solve, after an inner CG: x_o += d, d = 0, r = p = b - (A64 + sigma2 I) x_o in
    // FP64, its r.r (also the next inner solve's initial r.r); the state goes to the host.
    int outer_step(Slot &s)
    {
        h2n::Range range("h2_server: refinement step");
        const Request &q = s.req;
        const size_t bytes = size_t(q.n) * 8;
        h2srv::k_axpy<<<grid_for(q.n), kThreads, 0, s.st>>>(s.xo, s.x, q.n);
        cudaMemsetAsync(s.x, 0, bytes, s.st);
        int rc = apply64(s, s.xo, s.Ap);
        if (rc != H2_OK) return rc;
        k_residual<<<grid_for(q.n), kThreads, 0, s.st>>>(s.b, s.Ap, s.r, s.p, q.n);
        dot(s.r, s.r, q.n, s.partial, s.head->scal + 4, s.st);
        k_copy_scalar<<<1, 1, 0, s.st>>>(s.head->scal, 0, 4);
        cudaMemcpyAsync(&s.ring[kRing], s.head, sizeof(Head), cudaMemcpyDeviceToHost, s.st);
        cudaEventRecord(s.ev_outer, s.st);
        s.outer_pending = true;
        s.done = s.enq;  // iterations enqueued after the inner convergence changed nothing
        return status_of(cudaGetLastError());
    }

    // Refined solve, done: the outer iterate to the host (its FP64 residual is in ring[kRing]).
    int finish_refined(Slot &s)
    {
        h2n::Range range("h2_server: finish");
        s.finishing = true;
        cudaMemcpyAsync(s.stage, s.xo, size_t(s.req.n) * 8, cudaMemcpyDeviceToHost, s.st);
        cudaEventRecord(s.ev_fin, s.st);
        return status_of(cudaGetLastError());
    }

    // true residual with one more product, then x and the final state to the host
    int finish(Slot &s)
    {
        h2n::Range range("h2_server: finish");
        s.finishing = true;
        int rc = apply(s, s.x, s.Ap);
        if (rc != H2_OK) return rc;
        k_residual<<<grid_for(s.req.n), kThreads, 0, s.st>>>(s.b, s.Ap, s.r, nullptr, s.req.n);
        dot(s.r, s.r, s.req.n, s.partial, s.head->scal + 4, s.st);
        cudaMemcpyAsync(&s.ring[kRing], s.head, sizeof(Head), cudaMemcpyDeviceToHost, s.st);
        cudaMemcpyAsync(s.stage, s.x, size_t(s.req.n) * 8, cudaMemcpyDeviceToHost, s.st);
        cudaEventRecord(s.ev_fin, s.st);
        return status_of(cudaGetLastError());
    }

    void complete(Slot &s, int rc)
    {
        const Head &h = s.ring[kRing];
        h2_request_result r{};
        r.request_id = s.req.id;
        r.iters = rc == H2_OK ? h.iters : 0;
        const double bb = s.req.op64 ? h.scal[5] : h.scal[3];
        r.true_relres = (rc == H2_OK && bb > 0.0) ? std::sqrt(h.scal[4] / bb) : 0.0;
        const bool ok = s.req.op64 ? (bb == 0.0 || r.true_relres < s.req.tol) : h.flag == 1;
        r.status = rc != H2_OK ? rc : s.cancel ? H2_ECANCELED : (ok ? H2_OK : H2_ENOTCONV);
        if (rc == H2_OK) std::memcpy(s.req.x, s.stage, size_t(s.req.n) * 8);
        r.t_submit = s.req.t_submit;
        r.t_admit = s.t_admit;
        r.t_done = now();
        if (rc != H2_OK) cudaStreamSynchronize(s.st);  // nothing of this request may still run
        if (s.iter) {
            cudaGraphExecDestroy(s.iter);
            s.iter = nullptr;
        }
        arena.release(s.mem, s.req.bytes);
        s.busy = false;
        s.mem = nullptr;
        std::lock_guard<std::mutex> lk(mu);
        results.push_back(r);
        inflight.erase(std::remove(inflight.begin(), inflight.end(), r.request_id), inflight.end());
        --outstanding;
        cv.notify_all();
    }

    // one pass over the slots; true if anything moved
    bool step()
    {
        bool moved = false;
        {  // admissions, strict FIFO
            std::unique_lock<std::mutex> lk(mu);
            while (!queue.empty()) {
                Slot *free_slot = nullptr;
                for (Slot &s : slots)
                    if (!s.busy) {
                        free_slot = &s;
                        break;
                    }
                if (!free_slot) break;
                char *mem = arena.alloc(queue.front().bytes);
                if (!mem) break;
                const Request q = queue.front();
                queue.pop_front();
                inflight.push_back(q.id);
                lk.unlock();
                const int rc = admit(*free_slot, q, mem);
                if (rc != H2_OK) complete(*free_slot, rc);
                moved = true;
                lk.lock();
            }
        }
        std::vector<int64_t> cancel_now;
        {
            std::lock_guard<std::mutex> lk(mu);
            cancel_now.swap(cancels);
        }
        for (Slot &s : slots)
            if (s.busy && !s.finishing &&
                std::find(cancel_now.begin(), cancel_now.end(), s.req.id) != cancel_now.end())
                s.cancel = true;
        for (Slot &s : slots) {
            if (!s.busy) continue;
            if (s.finishing) {
                const cudaError_t e = cudaEventQuery(s.ev_fin);
                if (e == cudaErrorNotReady) continue;
                complete(s, status_of(e));
                moved = true;
                continue;
            }
            if (s.outer_pending) {  // refined solve: the FP64 residual of the new outer iterate
                const cudaError_t e = cudaEventQuery(s.ev_outer);
                if (e == cudaErrorNotReady) continue;
                moved = true;
                s.outer_pending = false;
                if (e != cudaSuccess) {
                    complete(s, status_of(e));
                    continue;
                }
                const Head h = s.ring[kRing];
                const double bb = h.scal[5];
                const bool conv = bb == 0.0 || std::sqrt(h.scal[4] / bb) < s.req.tol;
                if (conv || h.flag == 2 || h.iters >= s.req.maxit || s.cancel) {
                    const int rc = finish_refined(s);
                    if (rc != H2_OK) complete(s, rc);
                    continue;
                }
                h2srv::k_restart<<<1, 1, 0, s.st>>>(s.head);  // next inner CG on the outer residual
                s.enq_cap = s.enq + (s.req.maxit - h.iters);
                const int rc = status_of(cudaGetLastError());
                if (rc != H2_OK) {
                    complete(s, rc);
                    continue;
                }
            }
            while (s.done < s.enq) {
                const cudaError_t e = cudaEventQuery(s.ev[s.done % kRing]);
                if (e == cudaErrorNotReady) break;
                moved = true;
                if (e != cudaSuccess) {
                    complete(s, status_of(e));
                    break;
                }
                const Head h = s.ring[s.done % kRing];
                ++s.done;
                if (h.flag != 0 || h.iters >= s.req.maxit) {
                    const int rc = s.req.op64 ? outer_step(s) : finish(s);
                    if (rc != H2_OK) complete(s, rc);
                    break;
                }
            }
            if (!s.busy || s.finishing || s.outer_pending) continue;
            if (s.cancel) {  // no new iterations; finish once the enqueued ones are done
                if (s.done == s.enq) {
                    const int rc = s.req.op64 ? outer_step(s) : finish(s);
                    if (rc != H2_OK) complete(s, rc);
                    moved = true;
                }
                continue;
            }
            while (s.enq - s.done < kAhead && s.enq < s.enq_cap) {
                const int rc = enqueue_iteration(s);
                moved = true;
                if (rc != H2_OK) {
                    complete(s, rc);
                    break;
                }
            }
        }
        return moved;
    }

    void run()
    {
        cudaSetDevice(device);
        for (;;) {
            const bool moved = step();
            bool busy = false;
            for (const Slot &s : slots) busy = busy || s.busy;
            if (stop.load() && !busy) break;
            if (!moved) std::this_thread::sleep_for(std::chrono::microseconds(busy ? 10 : 50));
        }
    }
};

extern "C" {

size_t h2_server_request_bytes(h2_handle h)
{
    if (!h) return 0;
    h2_info info;
    if (h2_get_info(h, &info) != H2_OK || info.uploaded_prec < 0) return 0;
    return request_bytes(h, info.uploaded_prec == H2_FP64, info.n);
}

int h2_server_create(size_t slot_memory_bytes, int max_slots, int64_t max_points, h2_server_t *out)
{
    if (!out || max_slots < 1 || max_points < 1 || slot_memory_bytes == 0) return H2_EINVAL;
    *out = nullptr;
    h2_server *s = new (std::nothrow) h2_server;
    if (!s) return H2_ENOMEM;
    s->t0 = Clock::now();
    s->max_points = max_points;
    cudaGetDevice(&s->device);
    int rc = s->arena.init(slot_memory_bytes);
    s->slots.resize(size_t(max_slots));
    if (rc == H2_OK)
        rc = status_of(cudaMallocHost(reinterpret_cast<void **>(&s->ring_all), sizeof(Head) * (kRing + 1) * max_slots));
    for (int i = 0; rc == H2_OK && i < max_slots; ++i) {
        Slot &sl = s->slots[size_t(i)];
        sl.ring = s->ring_all + size_t(i) * (kRing + 1);
        rc = status_of(cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking));
        if (rc == H2_OK) rc = h2_exec_create(&sl.ex);
        for (int j = 0; rc == H2_OK && j < kRing; ++j)
            rc = status_of(cudaEventCreateWithFlags(&sl.ev[j], cudaEventDisableTiming));
        if (rc == H2_OK) rc = status_of(cudaEventCreateWithFlags(&sl.ev_fin, cudaEventDisableTiming));
        if (rc == H2_OK) rc = status_of(cudaEventCreateWithFlags(&sl.ev_outer, cudaEventDisableTiming));
        if (rc == H2_OK)
            rc = status_of(cudaMallocHost(reinterpret_cast<void **>(&sl.stage), size_t(max_points) * sizeof(double)));
    }
    if (rc != H2_OK) {
        h2_server_destroy(s);
        return rc;
    }
    s->th = std::thread([s] { s->run(); });
    *out = s;
    return H2_OK;
}

int h2_server_submit(h2_server_t s, h2_handle op, double sigma2, const double *b, double *x, double tol, int maxit,
                     int64_t *request_id)
{
    if (request_id) *request_id = 0;
    if (!s || !op || !b || !x || maxit < 0 || !(tol >= 0) || !(sigma2 >= 0)) return H2_EINVAL;
    h2_info info;
    if (h2_get_info(op, &info) != H2_OK) return H2_EINVAL;
    if (info.uploaded_prec < 0) return H2_ESTATE;
    if (info.n > s->max_points) return H2_EINVAL;
    Request q;
    q.op = op;
    q.sigma2 = sigma2;
    q.tol = tol;
    q.maxit = maxit;
    q.b = b;
    q.x = x;
    q.n = info.n;
    q.fp64 = info.uploaded_prec == H2_FP64;
    q.bytes = request_bytes(op, q.fp64, q.n);
    if (al(q.bytes) > s->arena.capacity()) return H2_ENOMEM;
    q.t_submit = s->now();
    std::lock_guard<std::mutex> lk(s->mu);
    q.id = s->next_id++;
    s->queue.push_back(q);
    ++s->outstanding;
    if (request_id) *request_id = q.id;
    return H2_OK;
}

int h2_server_submit_refined(h2_server_t s, h2_handle op, h2_handle op64, double sigma2, const double *b, double *x,
                             double tol, double inner_tol, int maxit, int64_t *request_id)
{
    if (request_id) *request_id = 0;
    if (!s || !op || !op64 || !b || !x || maxit < 0 || !(tol >= 0) || !(sigma2 >= 0) ||
        !(inner_tol > 0 && inner_tol < 1))
        return H2_EINVAL;
    h2_info info, info64;
    if (h2_get_info(op, &info) != H2_OK || h2_get_info(op64, &info64) != H2_OK) return H2_EINVAL;
    if (info.uploaded_prec < 0 || info64.uploaded_prec != H2_FP64) return H2_ESTATE;
    if (info.n != info64.n || info.n > s->max_points) return H2_EINVAL;
    Request q;
    q.op = op;
    q.op64 = op64;
    q.inner_tol = inner_tol;
    q.sigma2 = sigma2;
    q.tol = tol;
    q.maxit = maxit;
    q.b = b;
    q.x = x;
    q.n = info.n;
    q.fp64 = info.uploaded_prec == H2_FP64;
    q.bytes = request_bytes(op, q.fp64, q.n, op64);
    if (al(q.bytes) > s->arena.capacity()) return H2_ENOMEM;
    q.t_submit = s->now();
    std::lock_guard<std::mutex> lk(s->mu);
    q.id = s->next_id++;
    s->queue.push_back(q);
    ++s->outstanding;
    if (request_id) *request_id = q.id;
    return H2_OK;
}

size_t h2_server_request_bytes_refined(h2_handle op, h2_handle op64)
{
    if (!op || !op64) return 0;
    h2_info info, info64;
    if (h2_get_info(op, &info) != H2_OK || info.uploaded_prec < 0) return 0;
    if (h2_get_info(op64, &info64) != H2_OK || info64.uploaded_prec != H2_FP64 || info64.n != info.n) return 0;
    return request_bytes(op, info.uploaded_prec == H2_FP64, info.n, op64);
}

int h2_server_poll(h2_server_t s, h2_request_result *results, int max_results, int *n_results)
{
    if (n_results) *n_results = 0;
    if (!s || max_results < 0 || (max_results > 0 && !results)) return H2_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    const int n = int(std::min<size_t>(size_t(max_results), s->results.size()));
    for (int i = 0; i < n; ++i) results[i] = s->results[size_t(i)];
    s->results.erase(s->results.begin(), s->results.begin() + n);
    if (n_results) *n_results = n;
    return H2_OK;
}

int h2_server_wait(h2_server_t s, double timeout_s)
{
    if (!s || !(timeout_s >= 0)) return H2_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    const bool ok = s->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), [s] { return s->outstanding == 0; });
    return ok ? H2_OK : H2_ETIMEOUT;
}

int h2_server_cancel(h2_server_t s, int64_t request_id)
{
    if (!s) return H2_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
        if (it->id != request_id) continue;
        h2_request_result r{};
        r.request_id = request_id;
        r.status = H2_ECANCELED;
        r.t_submit = it->t_submit;
        r.t_done = s->now();
        s->queue.erase(it);
        s->results.push_back(r);
        --s->outstanding;
        s->cv.notify_all();
        return H2_OK;
    }
    if (std::find(s->inflight.begin(), s->inflight.end(), request_id) == s->inflight.end()) return H2_EINVAL;
    s->cancels.push_back(request_id);
    return H2_OK;
}

int h2_server_destroy(h2_server_t s)
{
    if (!s) return H2_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->outstanding -= int64_t(s->queue.size());  // queued requests are dropped unstarted
        s->queue.clear();
    }
    s->stop.store(true);
    if (s->th.joinable()) s->th.join();
    for (Slot &sl : s->slots) {
        if (sl.st) cudaStreamSynchronize(sl.st);
        for (cudaEvent_t e : sl.ev)
            if (e) cudaEventDestroy(e);
        if (sl.ev_fin) cudaEventDestroy(sl.ev_fin);
        if (sl.ev_outer) cudaEventDestroy(sl.ev_outer);
        h2_exec_destroy(&sl.ex);
        if (sl.st) cudaStreamDestroy(sl.st);
        if (sl.stage) cudaFreeHost(sl.stage);
    }
    if (s->ring_all) cudaFreeHost(s->ring_all);
    s->arena.destroy();
    delete s;
    return H2_OK;
}

}  // extern "C"
