#!/usr/bin/env python3
"""Benchmark: H^2 matrix-vector product on GB300 at the paper's precision (FP64).

Workload (default): N = 2^20 points on a 1024 x 1024 grid in [0,1]^2, Gaussian kernel
exp(-r^2/0.01), leaf size 64, 8 x 8 Chebyshev grid (rank 64), eta = 0.7, nv = 1,
x ~ N(0,1). A step is one full product Y = A_H2 X (upsweep, all-level coupling
product, dense near field, downsweep, epilogue) in FP64, the precision of every product
in the paper's experiments (Sec. 6). The headline metric is the algorithmic HBM throughput
of the product: the operator entries it must stream (coupling blocks, dense blocks, leaf
bases twice, transfers twice) plus X read and Y written, divided by the device time of one
product. Gflop/s counts 2 flops per entry per vector. The FP64 product is bound by the FP64
fused multiply-add rate of the part, which the bench measures first (h2_measure_peak); its
roofline object compares the dominant kernel against that measured rate. The same product
in FP32 (HBM-bound) is reported beside it under "fp32", with its own roofline and e2e.

Timing: W warm-up products, then K timed products with the L2 flushed (a 512 MB write)
before each one, outside the events; CUDA events on the launching stream; barrier and
synchronize on both sides; max over ranks. Several GPUs run independent replicas
(no collective on the data path): the value is the sum over ranks.

``--impl reference`` times the FP64 CPU oracle on a bounded sample of the same workload
family instead (rank 0 only), one oracle process per host core.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic_inputs as si  # noqa: E402

METRIC = "H2 matvec GB/s (nv=1, FP64, 2D Gaussian grid N=2^20, rank 64)"
# FP32 CUDA-core rate from unit counts at the maximum SM clock; only used where no measured
# rate is at hand (CPU-side tests of the roofline arithmetic)
FFMA_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def entry_counts(info, nv=1):
    """Matrix entries a product streams, and the vector elements it reads / writes."""
    mat = info.coupling_entries + info.dense_entries + 2 * info.basis_entries + 2 * info.transfer_entries
    vec = 2 * info.n * nv
    return mat, vec


def oracle_entry_counts(h):
    lvl, t, s, dt, ds = h.blocks()
    lo, hi = h.ranges()
    k = h.rank
    dense = int(np.sum((hi[dt] - lo[dt]) * (hi[ds] - lo[ds])))
    return len(t) * k * k + dense + 2 * h.n * k + 2 * (h.nnodes - 1) * k * k


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # raw samples go to a scratch file; the JSON line carries their summary
        self.path = os.path.join(tempfile.gettempdir(), f"h2_bench_clocks_{os.getpid()}_gpu{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={CLOCK_FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


def max_over_ranks(x: float, dist, device) -> float:
    """The largest value of x over the ranks (x itself without a process group)."""
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    if dist is not None and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gbs(world: int, bytes_per_rank_step: float, ms_per_step: float) -> float:
    """Whole-job throughput of independent replicas: every rank moves bytes_per_rank_step
    per step, and the job's step takes the slowest rank's time."""
    return world * bytes_per_rank_step / (ms_per_step * 1e-3) / 1e9


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def kernel_traffic(grid: int, prec: str = "fp32"):
    """DRAM bytes per launch of the streaming kernel from the committed ncu capture, or
    None when the capture was of another workload or the kernel source changed since."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"k_stream_traffic_grid1024_{prec}.json")
    if grid != 1024 or not os.path.exists(path):
        return None
    rec = json.load(open(path))
    h = hashlib.sha256()
    for f in rec["source_files"]:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    if h.hexdigest()[:16] != rec["source_sha256_16"]:
        return None
    return rec["traffic_bytes_per_launch"]


def measure_device_peaks(h2, gpu: int):
    """Arithmetic rates of this GPU, measured by h2_measure_peak (register-resident chains of
    one instruction kind on every SM, CUDA-event timed, nothing else running): the FP64 and
    FP32 fused multiply-add rates and the special-function 2^x rate as bursts (fastest of five
    30 ms launches), and the FP64 rate that bounds the headline product also sustained
    (fastest of five 400 ms launches), with the SM clocks sampled meanwhile. No clock or power
    setting is touched."""
    with ClockSampler(gpu) as clk:
        dfma, _ = h2.h2_measure_peak("dfma", 30.0)
        ffma, _ = h2.h2_measure_peak("ffma", 30.0)
        ex2, _ = h2.h2_measure_peak("ex2", 30.0)
        dfma_s, _ = h2.h2_measure_peak("dfma", 400.0)
    return {"dfma_tflops": dfma / 1e12, "dfma_tflops_sustained": dfma_s / 1e12, "ffma_tflops": ffma / 1e12,
            "ex2_per_s": ex2, "clocks": clk.summary(),
            "how": "h2_measure_peak: per thread 4 FMA accumulators with rotating multiplicands or 8 FMA chains "
                   "(the faster form; 8 ex2 chains), 32 warps per SM on every SM, fastest of 5 launches of ~30 ms "
                   "(burst) or ~400 ms (sustained) per form, CUDA events"}


def bottom_stream_entries(info):
    """Coupling entries of the levels the main streaming kernel takes (the lowest
    min(depth, 4) + 1 levels; the upper levels run on the side stream) and dense entries."""
    lb = info.depth - min(info.depth, 4)
    blocks = sum(int(info.coupling_per_level[l]) for l in range(lb, info.depth + 1))
    return blocks * info.rank * info.rank, int(info.dense_entries)


def stream_roofline(kernel, nbytes, flops, ms, alu_peak_tflops, alu_kind, peak_hbm, hbm_kind, traffic=None):
    """Roofline of one streaming launch: its algorithmic bytes at the measured copy bandwidth or
    its flops at the measured arithmetic rate, whichever takes longer, against its measured
    duration. achieved / peak in the bound's own unit; frac = achieved / peak."""
    t_hbm = nbytes / (peak_hbm * 1e9)
    t_alu = flops / (alu_peak_tflops * 1e12)
    sec = ms * 1e-3
    if t_alu > t_hbm:
        r = {"kernel": kernel, "bound": "alu", "achieved": flops / sec / 1e12, "peak": alu_peak_tflops,
             "unit": "TFLOP/s", "peak_kind": alu_kind}
    else:
        r = {"kernel": kernel, "bound": "hbm", "achieved": nbytes / sec / 1e9, "peak": peak_hbm, "unit": "GB/s",
             "peak_kind": hbm_kind}
    r["frac"] = r["achieved"] / r["peak"]
    r["traffic"] = traffic
    r.update({"algorithmic_bytes": int(nbytes), "algorithmic_flops": int(flops), "ms": ms,
              "bound_ms": 1e3 * max(t_hbm, t_alu), "hbm_GB/s": nbytes / sec / 1e9,
              "hbm_frac": nbytes / sec / 1e9 / peak_hbm})
    return r


def _oracle_sample(side: int):
    import oracle
    w = si.grid_gauss(side)
    pts = w.make_points()
    h = oracle.OracleH2(pts, w.kernel, w.leaf_size, w.cheb_order, w.eta, assemble=True)
    x = w.make_x(len(pts))
    return h, x, 8 * (oracle_entry_counts(h) + 2 * len(pts)), 2 * oracle_entry_counts(h)


def _oracle_worker(side, reps, barrier, queue):
    """One oracle process of the all-cores baseline: build the sample, wait for the others,
    time `reps` products back to back."""
    try:
        h, x, nbytes, flops = _oracle_sample(side)
        h.matvec(x)  # warm-up
        barrier.wait()
        t0 = time.perf_counter()
        for _ in range(reps):
            h.matvec(x)
        queue.put((time.perf_counter() - t0, reps, nbytes, flops, None))
    except Exception as exc:  # reported to the parent, which fails loudly
        try:
            barrier.abort()
        except Exception:
            pass
        queue.put((0.0, 0, 0, 0, f"{type(exc).__name__}: {exc}"))


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_all_cores(side: int = 256, reps: int = 5, workers: int = 0):
    """The oracle on every host core: `workers` independent processes (spawned, so that no
    CUDA state is inherited), each running its own products of the sample; the aggregate is
    the bytes of all products over the slowest process's time. The oracle itself is unchanged
    (one thread per product)."""
    import multiprocessing as mp
    workers = workers or host_cores()
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(workers)
    queue = ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(side, reps, barrier, queue)) for _ in range(workers)]
    for p in procs:
        p.start()
    res = [queue.get(timeout=900) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    errs = [r[4] for r in res if r[4]]
    if errs:
        raise RuntimeError(f"oracle worker failed: {errs[0]}")
    t = max(r[0] for r in res)
    nbytes = sum(r[1] * r[2] for r in res)
    flops = sum(r[1] * r[3] for r in res)
    return {"value": nbytes / t / 1e9, "unit": "GB/s", "cores": workers, "gflops": flops / t / 1e9,
            "wall_s": t, "products": sum(r[1] for r in res)}


def cpu_baseline(steps: int = 0, all_cores: bool = True):
    """The oracle (plain FP64 C, one thread per product) on a bounded sample: the same
    workload family at N = 2^16 (256 x 256 grid, same kernel, rank, leaf size and eta),
    blocks stored; one process on one core, and one process per host core."""
    h, x, nbytes, flops = _oracle_sample(256)
    h.matvec(x)  # warm-up
    nrep = steps if steps > 0 else 5
    times = []
    for _ in range(nrep):
        t0 = time.perf_counter()
        h.matvec(x)
        times.append(time.perf_counter() - t0)
    t = statistics.mean(times)
    one = {"value": nbytes / t / 1e9, "unit": "GB/s", "cores": 1, "ms_per_product": t * 1e3,
           "gflops": flops / t / 1e9}
    out = {"value": one["value"], "unit": "GB/s", "cores": 1, "cores_available": host_cores(), "kind": "oracle",
           "sample": f"256x256 grid (N=65536) of the same kernel/rank/leaf/eta, FP64 blocks stored, "
                     f"{nrep} products, mean {t * 1e3:.0f} ms", "ms_per_product": t * 1e3, "one_core": one}
    if all_cores:
        allc = oracle_all_cores(256, nrep)
        out.update({"value": allc["value"], "cores": allc["cores"],
                    "sample": f"256x256 grid (N=65536) of the same kernel/rank/leaf/eta, FP64 blocks stored; "
                              f"{allc['cores']} oracle processes, {nrep} products each, aggregate over "
                              f"{allc['wall_s']:.1f} s (one core: {t * 1e3:.0f} ms per product)",
                    "all_cores": allc})
    return out


def multi_rhs(h2, torch, steps, warmup, peak_hbm, peak_kind, n_points=None, with_fp64=True,
              ffma_peak=FFMA_PEAK_TFLOPS, dfma_peak=None, alu_kind="measured (h2_measure_peak, {} FMA chains)"):
    """The multi-vector workload: N = 2^21 uniform random points in [0,1]^3, exp(-r/0.2),
    leaf 64, 4 x 4 x 4 Chebyshev grid (rank 64), eta 0.7, 32 vectors, in split-BF16 on the
    tensor cores, in FP32 on the tensor cores (3xTF32; the default for FP32 passes of more
    than 8 vectors) and in FP32 on the CUDA cores (FMA), and in FP64. Its ~113 GB of stored blocks exceed L2 by far, so no flush is
    needed between products. Bytes and flops are algorithmic: every stored entry once per
    product (bases and transfers twice), X read and Y written; 2 flops per entry per vector."""
    w = si.CLOUD3D_EXP if not n_points or n_points == 2 ** 21 else si.cloud3d(n_points)
    pts = w.make_points()
    op = h2.H2Operator(pts, w.kernel, w.leaf_size, w.cheb_order, w.eta)
    info = op.info
    n, nv = op.n, w.nv
    mat_entries, vec_elems = entry_counts(info, nv)
    bytes_step = 4 * (mat_entries + vec_elems)
    flops = 2 * mat_entries * nv
    Xh = np.ascontiguousarray(w.make_x(n).T).astype(np.float32)
    out = {"workload": w.name, "n": n, "nv": nv, "rank": info.rank, "leaf": info.leaf_size, "eta": w.eta,
           "kernel": "exp(-r/0.2)", "depth": info.depth, "coupling_blocks": info.n_coupling,
           "dense_blocks": info.n_dense, "bytes_per_step": bytes_step, "flops_per_step": flops,
           "l2": f"inputs larger than L2 ({4 * mat_entries / 1e9:.1f} GB of blocks per product), no flush"}
    stream = torch.cuda.current_stream()
    results = {}
    precs = ("bf16x2", "fp32", "fp32_cuda_cores", "fp64") if with_fp64 else ("bf16x2", "fp32", "fp32_cuda_cores")
    for prec in precs:
        t0 = time.perf_counter()
        if prec != "fp32_cuda_cores":  # the CUDA-core FP32 pass reuses the FP32 upload
            op.upload(prec)
        upload_s = time.perf_counter() - t0
        if prec.startswith("fp32"):
            h2.h2_set_fp32_tensor(op.handle, prec == "fp32")
        X = torch.from_numpy(Xh).cuda().t()
        if prec == "fp64":
            X = X.double()
        Y = op.new_vectors(nv, fill=0.0)
        if prec == "fp64":  # DFMA-bound (about 2 s per product): one warm-up, two timed
            steps, warmup = 2, 1
        for _ in range(warmup):
            op.matvec(X, Y)
        h2.h2_get_timing(op.handle)
        h2.h2_set_timing(op.handle, True)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in evs:
            a.record(stream)
            op.matvec(X, Y)
            b.record(stream)
        torch.cuda.synchronize()
        h2.h2_set_timing(op.handle, False)
        ms = [a.elapsed_time(b) for a, b in evs]
        phase_ms, phase_launches, prods = h2.h2_get_timing(op.handle)
        phase_ms = phase_ms / max(prods, 1)
        ms_step = float(np.mean(ms))
        gbs = bytes_step / (ms_step * 1e-3) / 1e9
        # the block stream (phase 1): every coupling and dense entry once, one read of each
        # node's and leaf's input segment, one write of each output segment
        seg = 4 * nv * ((info.n_nodes + 1) * info.rank + n)
        blk_bytes = 4 * (info.coupling_entries + info.dense_entries) + 2 * seg
        blk_gbs = blk_bytes / (float(phase_ms[1]) * 1e-3) / 1e9
        blk_tflops = 2 * (info.coupling_entries + info.dense_entries) * nv / (float(phase_ms[1]) * 1e-3) / 1e12
        if prec == "bf16x2":
            roof = {"kernel": "k_stream_tc (split-BF16 tcgen05, 128x64x16 MMAs, FP32 accumulation in TMEM)",
                    "bound": "hbm", "achieved": blk_gbs, "peak": peak_hbm, "unit": "GB/s",
                    "frac": blk_gbs / peak_hbm, "peak_kind": peak_kind, "algorithmic_bytes": blk_bytes}
        elif prec == "fp32":
            roof = {"kernel": "k_stream_tf32 (3xTF32 tcgen05, A = [S_hi; S_lo] in TMEM, 128x64x8 MMAs, FP32 "
                              "accumulation in TMEM)",
                    "bound": "hbm", "achieved": blk_gbs, "peak": peak_hbm, "unit": "GB/s",
                    "frac": blk_gbs / peak_hbm, "peak_kind": peak_kind, "algorithmic_bytes": blk_bytes,
                    "block_tflops": blk_tflops}
        else:
            # 16 flop per byte at 32 vectors: the FP32 stream is bound by the CUDA-core FMA rate
            roof = {"kernel": "k_stream (FP32, register-blocked wide accumulator)", "bound": "alu",
                    "achieved": blk_tflops, "peak": ffma_peak, "unit": "TFLOP/s",
                    "frac": blk_tflops / ffma_peak, "peak_kind": alu_kind.format("FP32"),
                    "hbm_GB/s": blk_gbs}
        if prec == "fp64":
            # 8 flop per FP64 byte at 32 vectors: bound by the FP64 FMA rate
            roof = {"kernel": "k_stream (FP64, register-blocked wide accumulator)", "bound": "alu",
                    "achieved": blk_tflops, "peak": dfma_peak, "unit": "TFLOP/s",
                    "frac": blk_tflops / dfma_peak if dfma_peak else None,
                    "peak_kind": alu_kind.format("FP64")}
            gbs = 8 * (mat_entries + vec_elems) / (ms_step * 1e-3) / 1e9
        out[prec] = {"ms_per_step": ms_step, "ms_median": float(np.median(ms)), "GB/s": gbs,
                     "gflops": flops / (ms_step * 1e-3) / 1e9, "frac_of_hbm": gbs / peak_hbm,
                     "steps": steps, "upload_s": upload_s,
                     "phases_ms": dict(zip(h2.PHASES, [float(v) for v in phase_ms])), "roofline": roof}
        results[prec] = Y.t().contiguous().cpu().double().numpy()
        del X, Y
    if "fp64" in results:
        ref = results["fp64"]
        nref = float(np.linalg.norm(ref))
        for prec in ("bf16x2", "fp32", "fp32_cuda_cores"):
            out[prec]["relerr_vs_fp64"] = float(np.linalg.norm(results[prec] - ref)) / nref
    op.close()
    return out


def serve_benchmark(h2, torch, requests_per_rate=32, maxit=100, rates=(0.5, 0.8, 1.0, 1.2), slots=8,
                    sigma2=1e-2, label=None, refined=False):
    """CG serving loop (h2_server_*): solves of (K + sigma2 I) x = b with tol 1e-6 on resident
    operators of uniform random points in [0,1]^2 (N = 2^14, 2^16, 2^18, 2^20), kernel
    (r^2 + 1e-4)^(-1.5), leaf 64, 8 x 8 Chebyshev grid (rank 64), eta 0.7, FP32 products and
    FP64 Krylov state; b ~ N(0,1); sizes drawn uniformly; Poisson arrivals at the given
    fractions of the one-at-a-time capacity. CG is capped at maxit iterations.

    sigma2 = 1e-2 is the literal shift: the system is SPD but its condition number is 1.3e4 at
    N = 2^12 and 2.7e6 at 2^14 (dense eigenvalues of the oracle's operator), so tol 1e-6 lies far
    beyond any serving budget without a preconditioner and the converged fraction and the achieved
    true residuals are reported beside the latencies. sigma2 = 1e4 is the same 1e-2 taken relative
    to the kernel's diagonal value kappa(0) = 1e6 (a unit-diagonal kernel plus 1e-2 I); there the
    solves converge, and p50 / p99 are reported over converged solves. refined: every request is a
    mixed-precision refinement (inner CG on the FP32 operator to 1e-3, outer FP64 residuals on an
    FP64 upload of the same operator), so tol holds for the FP64 residual."""
    sizes = [2 ** 14, 2 ** 16, 2 ** 18, 2 ** 20]
    tol = 1e-6
    ops = {n: h2.H2Operator(si.uniform_cloud(n, 2, 50 + i), ("imq", 1e-4, 1.5, 0), 64, 8, 0.7).upload("fp32")
           for i, n in enumerate(sizes)}
    ops64 = {}
    if refined:
        ops64 = {n: h2.H2Operator(si.uniform_cloud(n, 2, 50 + i), ("imq", 1e-4, 1.5, 0), 64, 8, 0.7).upload("fp64")
                 for i, n in enumerate(sizes)}
        big = max(h2.H2Server.request_bytes_refined(ops[n], ops64[n]) for n in sizes)
    else:
        big = max(h2.H2Server.request_bytes(o) for o in ops.values())

    def submit(server, n, b):
        if refined:
            return server.submit(ops[n], b, tol, maxit, sigma2, op64=ops64[n], inner_tol=1e-3)
        return server.submit(ops[n], b, tol, maxit, sigma2)
    server = h2.H2Server(slots * big, slots, max(sizes))
    try:
        def rhs(n, seed):
            return si.gaussian_vectors(n, 1, seed)[:, 0].copy()

        # warm-up and one-at-a-time capacity (each size alone, sizes uniform)
        alone, alone_iters, alone_res = {}, {}, {}
        for rep in range(2):
            for n, op in ops.items():
                submit(server, n, rhs(n, 7))
                server.wait()
                (r,) = server.poll()
                alone[n] = r["t_done"] - r["t_submit"]
                alone_iters[n] = r["iters"]
                alone_res[n] = r["true_relres"]
        capacity = 1.0 / float(np.mean(list(alone.values())))
        rng = np.random.default_rng(2026)
        per_rate = []
        for f in rates:
            lam = f * capacity
            gaps = rng.exponential(1.0 / lam, requests_per_rate)
            pick = rng.integers(0, len(sizes), requests_per_rate)
            bs = [rhs(sizes[k], 1000 + j) for j, k in enumerate(pick)]
            t0 = time.perf_counter()
            t = 0.0
            for j in range(requests_per_rate):
                t += gaps[j]
                delay = t0 + t - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                submit(server, sizes[pick[j]], bs[j])
            server.wait(600.0)
            res = server.poll(requests_per_rate + 8)
            lat = np.array([r["t_done"] - r["t_submit"] for r in res])
            wait_q = np.array([r["t_admit"] - r["t_submit"] for r in res])
            span = max(r["t_done"] for r in res) - min(r["t_submit"] for r in res)
            conv = np.array([r["status"] == h2.H2_OK for r in res])
            entry = {
                "offered_fraction": f, "offered_solves_per_s": lam, "requests": len(res),
                "solves_per_s": len(res) / span, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                "p99_ms": 1e3 * float(np.percentile(lat, 99)), "mean_queue_ms": 1e3 * float(wait_q.mean()),
                "mean_iters": float(np.mean([r["iters"] for r in res])),
                "converged_fraction": float(conv.mean()),
                "median_true_relres": float(np.median([r["true_relres"] for r in res])),
                "max_true_relres": float(np.max([r["true_relres"] for r in res]))}
            if conv.any():
                entry["converged_p50_ms"] = 1e3 * float(np.percentile(lat[conv], 50))
                entry["converged_p99_ms"] = 1e3 * float(np.percentile(lat[conv], 99))
                entry["converged_max_true_relres"] = float(np.max([r["true_relres"] for r, c in zip(res, conv) if c]))
            per_rate.append(entry)
        return {"workload": label or f"imq_cloud2d {{2^14,2^16,2^18,2^20}}, (r^2+1e-4)^-1.5, rank 64, "
                                     f"sigma2 {sigma2:g}, tol 1e-6",
                "sigma2": sigma2, "maxit": maxit, "slots": slots,
                "precision": ("mixed-precision refinement: inner CG with fp32 products to 1e-3, fp64 outer residuals"
                              if refined else "fp32 products, fp64 Krylov state"),
                "alone_ms": {str(n): 1e3 * v for n, v in alone.items()},
                "alone_iters": {str(n): v for n, v in alone_iters.items()},
                "alone_true_relres": {str(n): v for n, v in alone_res.items()},
                "capacity_solves_per_s": capacity, "rates": per_rate}
    finally:
        server.close()
        for op in list(ops.values()) + list(ops64.values()):
            op.close()


def matrix_free(h2, torch, op, x_host, flush, stream, steps, warmup, stored_ms, Y_stored, ex2_peak):
    """The same product with the coupling and dense entries evaluated in FP32 inside the
    stream (H2_FP32_MF: no blocks stored; bases and transfers as in FP32). The reported rate is
    evaluations per second over the block stream's time, against the measured special-function
    rate (2^x results per second, h2_measure_peak): one special-function operation per entry
    for the exponential kernels' generic path (the separable Gaussian path forms its entries
    from tables with multiplies, so for it this is a rate, not a bound). The L2 is flushed
    before every timed product, as for the stored path."""
    info = op.info
    evals = info.coupling_entries + info.dense_entries
    ref = Y_stored.double().cpu().numpy()
    op.upload("fp32mf")
    X = torch.from_numpy(x_host).to(device="cuda", dtype=torch.float32)
    Y = torch.empty_like(X)
    for _ in range(warmup):
        op.matvec(X, Y)
    h2.h2_get_timing(op.handle)
    h2.h2_set_timing(op.handle, True)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in evs:
        flush.zero_()
        a.record(stream)
        op.matvec(X, Y)
        b.record(stream)
    torch.cuda.synchronize()
    h2.h2_set_timing(op.handle, False)
    phase_ms, _, prods = h2.h2_get_timing(op.handle)
    phase_ms = phase_ms / max(prods, 1)
    ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    got = Y.double().cpu().numpy()
    sfu_peak = ex2_peak
    stream_rate = evals / (float(phase_ms[1]) * 1e-3)
    out = {"ms_per_step": ms, "speedup_vs_stored": stored_ms / ms, "evaluations_per_step": evals,
           "evaluations_per_s": evals / (ms * 1e-3), "device_bytes": h2.h2_get_info(op.handle).device_bytes,
           "phases_ms": dict(zip(h2.PHASES, [float(v) for v in phase_ms])),
           "relerr_vs_stored_fp32": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
           "roofline": {"kernel": "k_stream_mf (FP32 evaluation of coupling and dense entries)", "bound": "alu",
                        "achieved": stream_rate, "peak": sfu_peak, "unit": "evaluations/s",
                        "frac": stream_rate / sfu_peak,
                        "peak_kind": "measured (h2_measure_peak, ex2 chains)"}}
    op.upload("fp32")
    return out


FP64_PEAK_TFLOPS = 1.25  # nominal FP64 rate of the part; only used where no measured rate is at hand


def compress_oracle_sample(h2, torch):
    """The oracle's recompression (numpy FP64, one Python thread driving LAPACK on small
    matrices) timed on a bounded sample -- the 2D compression set at 128 x 128 points
    (N = 2^14) -- beside the GPU's on the same sample."""
    import time
    import oracle
    import oracle.compress as oc
    w = dataclasses.replace(si.COMPRESS_2D, points="grid2d:128")
    pts = w.make_points()
    orc = oracle.OracleH2(pts, w.kernel, w.leaf_size, w.cheb_order, w.eta)
    t0 = time.perf_counter()
    c = oc.CompressedH2(orc, si.COMPRESS_TAU)
    cpu_s = time.perf_counter() - t0
    op = h2.H2Operator(pts, w.kernel, w.leaf_size, w.cheb_order, w.eta)
    op.compress(si.COMPRESS_TAU).close()
    g = op.compress(si.COMPRESS_TAU)
    gpu_ms = float(sum(g.compress_info.ms))
    same = g.level_ranks == c.ranks
    g.close()
    op.close()
    return {"kind": "oracle", "sample": "2D compression set at 128 x 128 points (N = 2^14), tau = 1e-3",
            "cores": 1, "oracle_s": cpu_s, "gpu_ms": gpu_ms, "ranks_equal": same}


def compress_benchmark(h2, torch, steps=3, sets=("2d", "3d"), grid2d=1024, dfma_peak=None):
    """Algebraic recompression (Sec. 5) of the compression sets of Sec. 6 (synthetic_inputs
    COMPRESS_2D at N = 2^20, COMPRESS_3D at N = 2^18) to tau = 1e-3 on the GPU in FP64. Per
    set: device time of each step (CUDA events inside h2_compress, mean over `steps` calls
    after one warm-up call), the whole call's wall time (with the copies of the operator to
    and from the device), operation counts and rate against the FP64 peak (the path is bound
    by FP64 arithmetic), level ranks, low-rank memory before and after, and the relative
    error of the compressed FP64 product against the original's on one Gaussian vector."""
    import time
    out = {}
    chosen = {"2d": si.COMPRESS_2D if grid2d == 1024 else dataclasses.replace(
        si.COMPRESS_2D, name=f"compress_grid2d_exp_{grid2d}", points=f"grid2d:{grid2d}"), "3d": si.COMPRESS_3D}
    for w in (chosen[k] for k in sets):
        pts = w.make_points()
        op = h2.H2Operator(pts, w.kernel, w.leaf_size, w.cheb_order, w.eta)
        g = op.compress(si.COMPRESS_TAU)  # warm-up (kernel attributes, allocator)
        g.close()
        ms = np.zeros(4)
        wall = []
        for _ in range(steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g = op.compress(si.COMPRESS_TAU)
            wall.append(time.perf_counter() - t0)
            ms += np.array(list(g.compress_info.ms))
            info = g.compress_info
            if _ + 1 < steps:
                g.close()
        ms /= steps
        flops = np.array(list(info.flops))
        x = si.gaussian_vectors(len(pts), 1, 1)
        X = torch.from_numpy(x[:, 0]).cuda()
        op.upload("fp64")
        g.upload("fp64")
        y0 = op.matvec(X).cpu().numpy()
        y1 = g.matvec(X).cpu().numpy()
        # what the compression buys: the FP32 product (nv = 1, L2 flushed) of both operators
        prod = {}
        X32 = X.float()
        flush = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device="cuda")
        for name, o in (("uncompressed", op), ("compressed", g)):
            o.upload("fp32")
            Y32 = torch.empty_like(X32)
            for _ in range(3):
                o.matvec(X32, Y32)
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(10)]
            h2.h2_get_timing(o.handle)
            h2.h2_set_timing(o.handle, True)
            for a, b in evs:
                flush.zero_()
                a.record()
                o.matvec(X32, Y32)
                b.record()
            torch.cuda.synchronize()
            h2.h2_set_timing(o.handle, False)
            phase_ms, _, nprod = h2.h2_get_timing(o.handle)
            prod[name] = float(np.mean([a.elapsed_time(b) for a, b in evs]))
            oinfo = h2.h2_get_info(o.handle)
            prod[name + "_device_GB"] = oinfo.device_bytes / 1e9
            mat, vec = entry_counts(oinfo, 1)
            prod[name + "_GB/s"] = 4 * (mat + vec) / (prod[name] * 1e-3) / 1e9
            prod[name + "_phases_ms"] = dict(zip(h2.PHASES, [float(v) / max(nprod, 1) for v in phase_ms]))
        prod["speedup"] = prod["uncompressed"] / prod["compressed"]
        del flush
        total_ms = float(ms.sum())
        gflops = float(flops.sum()) / (total_ms * 1e-3) / 1e9
        out[w.name] = {
            "n": len(pts), "kernel": w.kernel[0], "rank_in": info.rank_in, "leaf": w.leaf_size, "eta": w.eta,
            "tau": info.tau, "depth": info.depth, "level_ranks": list(info.level_rank)[:info.depth + 1],
            "rank_out": info.rank_out,
            "ms": {"orthogonalize": ms[0], "downsweep": ms[1], "truncate": ms[2], "project": ms[3], "total": total_ms},
            "wall_s": float(np.mean(wall)),
            "gflop": {"orthogonalize": flops[0] / 1e9, "downsweep": flops[1] / 1e9, "truncate": flops[2] / 1e9,
                      "project": flops[3] / 1e9},
            "gflops": gflops, "jacobi_sweeps": int(info.jacobi_sweeps),
            "lowrank_GB_in": info.lowrank_bytes_in / 1e9, "lowrank_GB_out": info.lowrank_bytes_out / 1e9,
            "lowrank_reduction": info.lowrank_bytes_in / max(info.lowrank_bytes_out, 1),
            "relerr_vs_uncompressed": float(np.linalg.norm(y1 - y0) / np.linalg.norm(y0)),
            "product_fp32_ms": prod,
            "error_bound_rel": float(2 * np.sqrt(info.dropped_energy) * np.linalg.norm(x) / np.linalg.norm(y0)),
            "roofline": {"kernel": "h2_compress (FP64 QR / Jacobi SVD / small products, CUDA cores)", "bound": "alu",
                         "achieved": gflops / 1e3, "peak": dfma_peak or FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": gflops / 1e3 / (dfma_peak or FP64_PEAK_TFLOPS),
                         "peak_kind": "measured (h2_measure_peak, FP64 FMA chains)" if dfma_peak
                         else "nominal FP64 rate"},
        }
        g.close()
        op.close()
        torch.cuda.empty_cache()
    return out


def batch_roofline(total_bytes, total_flops, ms, ffma_peak=None):
    """The batch's bound: its blocks streamed once at the measured copy bandwidth, or its
    flops at the FP32 FMA rate (measured when given), whichever takes longer; frac = that
    time / the measured one."""
    peak_gbs, kind = measured_peaks()
    fma = ffma_peak or FFMA_PEAK_TFLOPS
    t_hbm = total_bytes / (peak_gbs * 1e9) * 1e3
    t_fma = total_flops / (fma * 1e12) * 1e3
    bound = "hbm" if t_hbm >= t_fma else "alu"
    return {"bound": bound, "bound_ms": max(t_hbm, t_fma), "hbm_ms": t_hbm, "fma_ms": t_fma,
            "achieved": total_bytes / (ms * 1e-3) / 1e9 if bound == "hbm" else total_flops / (ms * 1e-3) / 1e12,
            "peak": peak_gbs if bound == "hbm" else fma, "unit": "GB/s" if bound == "hbm" else "TFLOP/s",
            "frac": max(t_hbm, t_fma) / ms,
            "peak_kind": f"{kind} HBM / {'measured' if ffma_peak else 'derived'} FP32 FMA"}


def batch_benchmark(h2, torch, steps=10, warmup=3, count=64, n_max=2 ** 18, with_fp64=True, ffma_peak=None,
                    plain=False):
    """Batched products of 64 uneven operators (synthetic_inputs.uneven_batch: N log-uniform
    in [2^12, 2^18], even members 2D grids with orders 4-8, odd members 3D clouds with orders
    3-4, exp(-r/l) with l in [0.05, 0.3], leaf 64, eta 0.7, nv in 1..16), FP32, as one
    graph-replayed batch (h2_batch_run, autotuned) against the same products issued one after
    another (h2_matvec) and against the batch with each member's sweeps as its own launches.
    The batch streams more than L2 holds, so no flush is needed. plain: the batched product
    alone, default configuration (for profiler launch lists)."""
    members = si.uneven_batch(count=count, n_max=n_max)
    ops, Xs, Ys = [], [], []
    total_bytes = 0
    total_flops = 0
    for m in members:
        op = h2.H2Operator(m.points, m.kernel, m.leaf_size, m.cheb_order, m.eta).upload("fp32")
        mat, vec = entry_counts(op.info, m.nv)
        total_bytes += 4 * (mat + vec)
        total_flops += 2 * mat * m.nv
        ops.append(op)
        Xs.append(torch.from_numpy(np.ascontiguousarray(m.make_x().T)).float().cuda().t())
        Ys.append(op.new_vectors(m.nv, fill=0.0))
    stream = torch.cuda.current_stream()
    try:
        t0 = time.perf_counter()
        batch = h2.H2Batch(ops, Xs, Ys, autotune=not plain)
        create_s = time.perf_counter() - t0
        desc = batch.describe()

        def timed(fn):
            for _ in range(warmup):
                fn()
            torch.cuda.synchronize()
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for a, b in evs:
                a.record(stream)
                fn()
                b.record(stream)
            torch.cuda.synchronize()
            return [a.elapsed_time(b) for a, b in evs]

        ms_batch = timed(batch.run)
        batch.check()
        batch.run()
        torch.cuda.synchronize()
        y32 = [Y.double().cpu().numpy() for Y in Ys]
        if plain:
            batch.close()
            return {"batched_ms": float(np.median(ms_batch)), "configuration": desc}
        # the earlier schedule: the same batch with every member's sweeps as its own launches
        own = h2.H2Batch(ops, Xs, Ys, member_sweeps=True)
        ms_own = float(np.median(timed(own.run)))
        own.close()
        ms_seq = timed(lambda: [op.matvec(X, Y) for op, X, Y in zip(ops, Xs, Ys)])
        batch.close()
        mb, msq = float(np.median(ms_batch)), float(np.median(ms_seq))
        # the same batch with FP64 members: plain FP64 time and the FP32 results' error against it
        fp64 = None
        if with_fp64:
            for op in ops:
                op.upload("fp64")
            X64 = [X.double() for X in Xs]
            Y64 = [op.new_vectors(Y.shape[1] if Y.dim() > 1 else 1, fill=0.0) for op, Y in zip(ops, Ys)]
            b64 = h2.H2Batch(ops, X64, Y64)
            ms64 = float(np.median(timed(b64.run)))
            b64.run()
            torch.cuda.synchronize()
            num = sum(float(np.sum((a - Y.cpu().numpy()) ** 2)) for a, Y in zip(y32, Y64))
            den = sum(float(np.sum(Y.cpu().numpy() ** 2)) for Y in Y64)
            b64.close()
            fp64 = {"batched_ms": ms64, "batched_GB/s": 2 * total_bytes / (ms64 * 1e-3) / 1e9,
                    "fp32_speedup": ms64 / mb, "fp32_relerr_vs_fp64": float(np.sqrt(num / den))}
        return {"workload": f"uneven_batch: {count} operators, N log-uniform [2^12, {n_max}], 2D grids / 3D "
                            "clouds, exp(-r/l), rank 16-64, nv 1-16, FP32",
                "points": int(sum(len(m.points) for m in members)), "vectors": int(sum(m.nv for m in members)),
                "bytes_per_step": total_bytes, "flops_per_step": total_flops,
                "batched_ms": mb, "batched_GB/s": total_bytes / (mb * 1e-3) / 1e9,
                "batched_gflops": total_flops / (mb * 1e-3) / 1e9,
                "sequential_ms": msq, "sequential_GB/s": total_bytes / (msq * 1e-3) / 1e9,
                "speedup_vs_sequential": msq / mb, "member_sweeps_ms": ms_own,
                "create_s": create_s, "configuration": desc,
                "roofline": batch_roofline(total_bytes, total_flops, mb, ffma_peak),
                "fp64": fp64, "l2": "inputs larger than L2, no flush"}
    finally:
        for op in ops:
            op.close()


def run_reference(args, rank):
    """The reference arm: the FP64 oracle (the reference is a paper; the oracle written from
    it is the comparison program) on every host core, one process per core, each step one
    product per process on the bounded sample; rank 0 only."""
    if rank != 0:
        return
    nrep = max(1, args.steps)
    allc = oracle_all_cores(256, nrep)
    ms_step = 1e3 * allc["wall_s"] / nrep
    sample = (f"256x256 grid (N=65536) of the same kernel/rank/leaf/eta, FP64 blocks stored; {allc['cores']} oracle "
              f"processes, {nrep} products each")
    line = {"impl": "reference", "metric": METRIC, "value": allc["value"], "unit": "GB/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "grid256_gauss (bounded sample of grid1024_gauss)", "n": 65536, "nv": 1,
                       "rank": 64, "leaf": 64, "eta": 0.7},
            "cpu_baseline": {"kind": "oracle", "cores": allc["cores"], "cores_available": host_cores(),
                             "sample": sample, "value": allc["value"], "unit": "GB/s"},
            "e2e": {"value": allc["value"], "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp32", action="store_true", help="skip the FP32 product beside the FP64 headline")
    ap.add_argument("--no-fp64", action="store_true",
                    help="skip the FP64 counterparts of the batch and multi-vector measurements")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-peaks", action="store_true",
                    help="skip the arithmetic-rate measurements and use nominal rates (profiler captures only)")
    ap.add_argument("--no-multi-rhs", action="store_true",
                    help="skip the 32-vector measurement on the 2^21-point 3D cloud")
    ap.add_argument("--cloud-n", type=int, default=2 ** 21,
                    help="points of the 3D cloud of the 32-vector measurement (2^21 = the benchmarked size; "
                         "smaller sizes are for profiler captures)")
    ap.add_argument("--multi-rhs-steps", type=int, default=0, help="timed 32-vector products (0: steps / 20, >= 5)")
    ap.add_argument("--no-multi-rhs-fp64", action="store_true",
                    help="skip the FP64 product of the 32-vector workload (218 GB of blocks at 2^21 points)")
    ap.add_argument("--no-serve", action="store_true", help="skip the CG serving-loop measurement")
    ap.add_argument("--no-matrix-free", action="store_true", help="skip the matrix-free product measurement")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched uneven-operator measurement")
    ap.add_argument("--no-compress", action="store_true", help="skip the algebraic-compression measurement")
    ap.add_argument("--compress-sets", default="2d,3d", help="compression sets to time (2d, 3d)")
    ap.add_argument("--compress-grid", type=int, default=1024, help="grid side of the 2D compression set")
    ap.add_argument("--compress-steps", type=int, default=3, help="timed compressions per set")
    ap.add_argument("--batch-count", type=int, default=64, help="operators of the batched measurement")
    ap.add_argument("--batch-steps", type=int, default=10, help="timed replays of the batched measurement")
    ap.add_argument("--batch-plain", action="store_true",
                    help="time the batched product alone in its default configuration (profiler launch lists)")
    ap.add_argument("--batch-nmax", type=int, default=2 ** 18,
                    help="largest N of the batched measurement (smaller values are for profiler captures)")
    ap.add_argument("--serve-maxit", type=int, default=100, help="CG iteration cap of each served solve")
    ap.add_argument("--serve-requests", type=int, default=48, help="requests per arrival rate")
    ap.add_argument("--serve-reg-maxit", type=int, default=3000,
                    help="CG iteration cap of the regularized served mix (sigma2 = 1e-2 x kappa(0))")
    ap.add_argument("--serve-reg-requests", type=int, default=16, help="requests per rate, regularized mix")
    ap.add_argument("--grid", type=int, default=1024,
                    help="grid side of the 2D Gaussian workload (1024 = the benchmarked N = 2^20; smaller "
                         "sides are for profiler captures)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import paper_2109_05451_gb300 as h2

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    w = si.GRID1024_GAUSS if args.grid == 1024 else si.grid_gauss(args.grid)
    pts = w.make_points()
    t0 = time.perf_counter()
    op = h2.H2Operator(pts, w.kernel, w.leaf_size, w.cheb_order, w.eta)
    build_s = time.perf_counter() - t0
    info = op.info
    n = op.n
    x_host = w.make_x(n)[:, 0]
    mat_entries, vec_elems = entry_counts(info)
    flops = 2 * mat_entries
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    peak_hbm, peak_kind = measured_peaks()

    def time_products(prec, steps, warmup):
        t_up = time.perf_counter()
        op.upload(prec)
        upload_s = time.perf_counter() - t_up
        es = 8 if prec == "fp64" else 4
        X = torch.from_numpy(x_host).to(device="cuda", dtype=op.dtype)
        Y = torch.empty_like(X)
        for _ in range(warmup):
            op.matvec(X, Y)
        h2.h2_get_timing(op.handle)  # reset counters
        h2.h2_set_timing(op.handle, True)
        barrier()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in evs:
            flush.zero_()
            a.record(stream)
            op.matvec(X, Y)
            b.record(stream)
        barrier()
        h2.h2_set_timing(op.handle, False)
        step_ms = [a.elapsed_time(b) for a, b in evs]
        phase_ms, phase_launches, prods = h2.h2_get_timing(op.handle)
        return {"prec": prec, "esize": es, "step_ms": step_ms, "phase_ms": phase_ms / max(prods, 1),
                "phase_launches": phase_launches, "products": prods, "upload_s": upload_s, "X": X, "Y": Y}

    if args.no_peaks:
        peaks = {"dfma_tflops": FP64_PEAK_TFLOPS, "dfma_tflops_sustained": FP64_PEAK_TFLOPS,
                 "ffma_tflops": FFMA_PEAK_TFLOPS, "ex2_per_s": 152 * 32 * 2.07e9, "how": "nominal (not measured)"}
    else:
        peaks = measure_device_peaks(h2, local)
    dfma_peak = max(peaks["dfma_tflops"], peaks["dfma_tflops_sustained"])
    ffma_peak = peaks["ffma_tflops"]
    rate_kind = "nominal (not measured)" if args.no_peaks else "measured (h2_measure_peak, {} FMA chains)"
    cpl_entries, dns_entries = bottom_stream_entries(info)
    # the dominant kernel (phase 1, the streaming product of the lower levels' coupling rows
    # and of all dense rows): its blocks, one read of each input segment tree and one write of
    # each output segment; 2 flops per block entry
    seg_elems = 2 * ((info.n_nodes + 1) * info.rank + n)
    stream_flops = 2 * (cpl_entries + dns_entries)

    def e2e(X, Y, es):
        """End to end through the public API: pinned host X -> device, product, Y -> host."""
        dt = torch.float64 if es == 8 else torch.float32
        xh = torch.from_numpy(x_host.astype(np.float64 if es == 8 else np.float32)).pin_memory()
        yh = torch.empty_like(xh).pin_memory()
        for _ in range(3):
            X.copy_(xh, non_blocking=True)
            op.matvec(X, Y)
            yh.copy_(Y, non_blocking=True)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            X.copy_(xh, non_blocking=True)
            op.matvec(X, Y)
            yh.copy_(Y, non_blocking=True)
        e1.record(stream)
        barrier()
        e2e_ms = e0.elapsed_time(e1) / args.steps
        assert X.dtype == dt
        return {"value": job_gbs(world, es * (mat_entries + vec_elems), max_over_ranks(e2e_ms, dist, "cuda")),
                "unit": "GB/s", "h2d_bytes_per_step": es * n, "d2h_bytes_per_step": es * n}

    # ---- headline: FP64
    with ClockSampler(local) as clk:
        res = time_products("fp64", args.steps, max(3, args.warmup))
    clocks = clk.summary()
    ms_local = float(np.sum(res["step_ms"]))
    ms_total = max_over_ranks(ms_local, dist, "cuda")
    ms_step = ms_total / args.steps
    bytes_step = 8 * (mat_entries + vec_elems)
    value = job_gbs(world, bytes_step, ms_step)
    roof64 = stream_roofline("k_stream<double,1> (coupling rows of the lower levels + dense rows, Alg 4 + A_de x)",
                             8 * (cpl_entries + dns_entries + seg_elems), stream_flops, float(res["phase_ms"][1]),
                             dfma_peak, rate_kind.format("FP64"), peak_hbm, peak_kind,
                             kernel_traffic(args.grid, "fp64"))
    e2e64 = e2e(res["X"], res["Y"], 8)
    launches_per_product = int(np.sum(res["phase_launches"])) // max(res["products"], 1)
    Y64 = res["Y"].cpu().numpy()
    del res["X"], res["Y"]

    # ---- the same product in FP32 (HBM-bound)
    fp32 = None
    if not args.no_fp32:
        with ClockSampler(local) as clk32:
            r32 = time_products("fp32", args.steps, max(3, args.warmup))
        ms32 = max_over_ranks(float(np.sum(r32["step_ms"])), dist, "cuda") / args.steps
        b32 = 4 * (mat_entries + vec_elems)
        fp32 = {"value": job_gbs(world, b32, ms32), "unit": "GB/s", "ms_per_step": ms32,
                "ms_median": float(np.median(r32["step_ms"])), "gflops": world * flops / (ms32 * 1e-3) / 1e9,
                "bytes_per_step": b32, "frac_of_hbm": (b32 / (ms32 * 1e-3) / 1e9) / peak_hbm,
                "phases_ms": dict(zip(h2.PHASES, [float(v) for v in r32["phase_ms"]])),
                "roofline": stream_roofline("k_stream<float,1> (coupling rows of the lower levels + dense rows)",
                                            4 * (cpl_entries + dns_entries + seg_elems), stream_flops,
                                            float(r32["phase_ms"][1]), ffma_peak,
                                            rate_kind.format("FP32"), peak_hbm, peak_kind,
                                            kernel_traffic(args.grid, "fp32")),
                "e2e": e2e(r32["X"], r32["Y"], 4), "clocks": clk32.summary(), "upload_s": r32["upload_s"],
                "relerr_vs_fp64": float(np.linalg.norm(r32["Y"].double().cpu().numpy() - Y64) / np.linalg.norm(Y64))}
        res32_Y = r32["Y"]
        del r32["X"]

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cpu = cpu_baseline()
            cpu = {k: cpu[k] for k in ("value", "unit", "cores", "cores_available", "kind", "sample", "one_core",
                                       "all_cores") if k in cpu}
        except Exception as exc:  # the baseline is context; its failure must not hide the GPU line
            cpu = {"value": None, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": f"failed: {exc}"}

    # the metric names the default 2^20-point grid; another --grid names its own size
    metric = METRIC if args.grid == 1024 else METRIC.replace("N=2^20", f"N={n}")
    line = {
        "metric": metric, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n": n, "nv": 1, "rank": info.rank, "leaf": info.leaf_size, "eta": w.eta,
                   "kernel": "exp(-r^2/0.01)", "depth": info.depth, "coupling_blocks": info.n_coupling,
                   "dense_blocks": info.n_dense, "parallelism": f"replicas x{world}",
                   "l2": "flushed (512 MB write) before every timed product"},
        "gflops": world * flops / (ms_step * 1e-3) / 1e9,
        # the paper's protocol (Sec. 6): the mean of the runs left after dropping the fastest
        # and the slowest, here over this rank's timed products
        "ms_trimmed_mean": float(np.mean(sorted(res["step_ms"])[1:-1])) if len(res["step_ms"]) > 2 else ms_step,
        "ms_median": float(np.median(res["step_ms"])),
        "bytes_per_step": bytes_step,
        "flops_per_step": flops,
        "frac_of_hbm": (bytes_step / (ms_step * 1e-3) / 1e9) / peak_hbm,
        # the whole product against its bound: every flop at the measured FP64 FMA rate or
        # every byte at the measured copy bandwidth, whichever takes longer
        "product_bound_ms": 1e3 * max(flops / (dfma_peak * 1e12), bytes_step / (peak_hbm * 1e9)),
        "phases_ms": dict(zip(h2.PHASES, [float(v) for v in res["phase_ms"]])),
        "roofline": roof64,
        "e2e": e2e64,
        "gpu_launches": launches_per_product * args.steps,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "peaks": peaks,
        "build_s": build_s, "upload_s": res["upload_s"],
    }
    line["product_bound_frac"] = line["product_bound_ms"] / ms_step
    if fp32 is not None:
        line["fp32"] = fp32
    if world > 1:
        # replicas: the side measurements below characterise one GPU; at N > 1 the line is the
        # replicated headline product only, so the job holds its GPUs for no longer than that
        args.no_matrix_free = args.no_multi_rhs = args.no_batch = args.no_compress = args.no_serve = True
    if not args.no_matrix_free and fp32 is not None:
        try:
            line["matrix_free"] = matrix_free(h2, torch, op, x_host, flush, stream, max(20, args.steps // 4),
                                              max(3, args.warmup), fp32["ms_per_step"], res32_Y,
                                              peaks["ex2_per_s"])
        except Exception as exc:  # reported, never silently dropped
            line["matrix_free"] = {"error": f"{type(exc).__name__}: {exc}"}
    if not args.no_multi_rhs:
        op.close()
        try:
            mr_steps = args.multi_rhs_steps if args.multi_rhs_steps > 0 else max(5, args.steps // 20)
            line["multi_rhs"] = multi_rhs(h2, torch, mr_steps, 3, peak_hbm, peak_kind, args.cloud_n,
                                          not args.no_multi_rhs_fp64, ffma_peak, dfma_peak, rate_kind)
        except Exception as exc:  # reported, never silently dropped
            line["multi_rhs"] = {"error": f"{type(exc).__name__}: {exc}"}
    if not args.no_batch:
        try:
            line["batch"] = batch_benchmark(h2, torch, steps=args.batch_steps, count=args.batch_count,
                                            n_max=args.batch_nmax, with_fp64=not args.no_fp64, ffma_peak=ffma_peak,
                                            plain=args.batch_plain)
        except Exception as exc:  # reported, never silently dropped
            line["batch"] = {"error": f"{type(exc).__name__}: {exc}"}
    if not args.no_compress:
        try:
            line["compress"] = compress_benchmark(h2, torch, args.compress_steps, tuple(args.compress_sets.split(",")),
                                                  args.compress_grid, None if args.no_peaks else dfma_peak)
            if rank == 0 and world == 1 and not args.no_cpu_baseline:
                line["compress"]["cpu_baseline"] = compress_oracle_sample(h2, torch)
        except Exception as exc:  # reported, never silently dropped
            line["compress"] = {"error": f"{type(exc).__name__}: {exc}"}
    if not args.no_serve:
        try:
            line["serve"] = serve_benchmark(h2, torch, args.serve_requests, args.serve_maxit)
            line["serve_regularized"] = serve_benchmark(
                h2, torch, args.serve_reg_requests, args.serve_reg_maxit, rates=(0.5, 1.0, 1.2), sigma2=1e4,
                label="imq_cloud2d {2^14,2^16,2^18,2^20}, (r^2+1e-4)^-1.5, rank 64, sigma2 1e4 "
                      "(1e-2 x kappa(0)), tol 1e-6 on the FP64 residual", refined=True)
        except Exception as exc:  # reported, never silently dropped
            line["serve"] = {"error": f"{type(exc).__name__}: {exc}"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
