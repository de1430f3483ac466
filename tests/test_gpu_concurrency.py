"""Concurrent products on one handle from several host threads and streams, through the C ABI.

h2_matvec keeps one workspace per stream and h2_matvec_ws runs on the workspace it is given;
every product borrows its own fork/join context (side stream and events) while its launches
are enqueued. Two host threads, each on its own stream, issue interleaved products of one
operator with different inputs; every result must match the oracle at the precision's
tolerance (FP64 1e-12, FP32 1e-5 relative l2).
"""
import threading

import numpy as np
import pytest

import oracle
import synthetic_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2109_05451_gb300 as h2  # noqa: E402

TOL = {"fp64": 1e-12, "fp32": 1e-5}
DT = {"fp64": torch.float64, "fp32": torch.float32}


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def problem():
    pts = si.uniform_cloud(20000, 2, 11)
    args = (("exp", 0.1, 0, 0), 64, 6, 0.7)
    orc = oracle.OracleH2(pts, *args)
    return pts, args, orc


@pytest.mark.parametrize("entry", ["matvec", "matvec_ws"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_two_threads_two_streams_one_handle(problem, prec, entry):
    pts, args, orc = problem
    op = h2.H2Operator(pts, *args).upload(prec)
    nthreads, reps, nv = 2, 6, 2
    X = {(t, r): si.gaussian_vectors(op.n, nv, 100 + 10 * t + r) for t in range(nthreads) for r in range(reps)}
    ref = {key: orc.matvec(x) for key, x in X.items()}
    out, errors = {}, []
    barrier = threading.Barrier(nthreads)

    def worker(t):
        try:
            s = torch.cuda.Stream()
            ws = None
            if entry == "matvec_ws":
                nb = h2.h2_workspace_bytes(op.handle, nv)
                ws = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
            with torch.cuda.stream(s):
                Xd = {r: torch.from_numpy(np.ascontiguousarray(X[(t, r)].T)).to(device="cuda", dtype=DT[prec]).t()
                      for r in range(reps)}
                Yd = {r: op.new_vectors(nv, fill=float("nan")) for r in range(reps)}
            s.synchronize()
            barrier.wait()
            for r in range(reps):
                if entry == "matvec":
                    h2.h2_matvec(op.handle, Xd[r], Yd[r], nv, 1.0, 0.0, s)
                else:
                    h2.h2_matvec_ws(op.handle, Xd[r], Yd[r], nv, 1.0, 0.0, ws, ws.numel(), s)
            s.synchronize()
            for r in range(reps):
                out[(t, r)] = Yd[r].t().contiguous().cpu().double().numpy().T
        except Exception as exc:  # reported by the main thread
            errors.append(exc)

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(nthreads)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors
    for key in X:
        assert relerr(out[key], ref[key]) <= TOL[prec], key
    op.close()


def test_products_need_the_operators_device():
    """A product with no device copy is refused; with several GPUs, so is one issued while
    another device is current."""
    pts = si.uniform_cloud(3000, 2, 3)
    op = h2.H2Operator(pts, ("exp", 0.1, 0, 0), 32, 4, 0.7)
    X = torch.zeros(op.n, dtype=torch.float64, device="cuda")
    Y = torch.zeros_like(X)
    with pytest.raises(h2.H2Error) as e:
        h2.h2_matvec(op.handle, X, Y, 1)
    assert e.value.status == h2.H2_ESTATE
    op.upload("fp64")
    if torch.cuda.device_count() > 1:
        with torch.cuda.device(1):
            with pytest.raises(h2.H2Error) as e:
                h2.h2_matvec(op.handle, X, Y, 1, stream=0)
            assert e.value.status == h2.H2_EINVAL
    op.close()
