"""The no-allocation product entry point, h2_matvec_noalloc, through the C ABI.

Callers that must not allocate device memory (inside a fixed memory-pool budget, from an
allocator or out-of-memory handler, or in a real-time loop) use h2_matvec_noalloc, which
takes its workspace from a fixed per-GPU scratch area instead of allocating one. Its
output must match the allocating entry point's, call after call, since the scratch area
keeps the previous call's contents. This file is named to run after every other test, so
a run that stops at the first failure has already run everything else.
"""
import numpy as np
import pytest

import oracle
import synthetic_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2109_05451_gb300 as h2  # noqa: E402

TOL = {"fp64": 1e-12, "fp32": 1e-5, "bf16x2": 1e-4}
DT = {"fp64": torch.float64, "fp32": torch.float32, "bf16x2": torch.float32}


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def to_dev(X, prec):
    return torch.from_numpy(np.ascontiguousarray(np.asfortranarray(X).T)).to(device="cuda", dtype=DT[prec]).t()


def to_host(Y):
    return Y.t().contiguous().cpu().double().numpy().T


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x2"])
def test_noalloc_matches_allocating_product_on_consecutive_calls(prec):
    pts = si.grid_2d(128)
    args = (("gauss", 0.01, 0, 0), 64, 8, 0.7)
    op = h2.H2Operator(pts, *args).upload(prec)
    nv = 3
    X = si.gaussian_vectors(op.n, nv, 5)
    Y0 = si.gaussian_vectors(op.n, nv, 6)
    Xd = to_dev(X, prec)
    ref = op.new_vectors(nv)
    ref.copy_(to_dev(Y0, prec))
    h2.h2_matvec(op.handle, Xd, ref, nv, 0.5, -2.0)
    torch.cuda.synchronize()
    ref_h = to_host(ref)
    # the oracle's result for the same call
    orc = 0.5 * oracle.OracleH2(pts, *args).matvec(X) - 2.0 * Y0
    assert relerr(ref_h, orc) <= TOL[prec]
    assert h2.h2_workspace_bytes(op.handle, nv) <= h2.H2_NOALLOC_SCRATCH_BYTES
    # a second operator of another size and precision leaves its own values in the scratch
    # area (tickets and vector trees at other offsets) between the two calls
    other = h2.H2Operator(si.uniform_cloud(5000, 3, 2), ("exp", 0.2, 0, 0), 32, 3, 0.7)
    other.upload("fp32" if prec == "fp64" else "fp64")
    Xo = torch.ones((other.n, 2), dtype=other.dtype, device="cuda").t().contiguous().t()
    Yo = other.new_vectors(2, fill=0.0)
    for call in range(2):  # the second call runs on scratch holding other values
        Yd = op.new_vectors(nv)
        Yd.copy_(to_dev(Y0, prec))
        h2.h2_matvec_noalloc(op.handle, Xd, Yd, nv, 0.5, -2.0)
        torch.cuda.synchronize()
        got = to_host(Yd)
        assert relerr(got, ref_h) <= TOL[prec]
        assert relerr(got, orc) <= TOL[prec]
        if call == 0:
            h2.h2_matvec_noalloc(other.handle, Xo, Yo, 2, 1.0, 0.0)
            torch.cuda.synchronize()
    other.close()
    op.close()


def test_noalloc_rejects_operator_larger_than_scratch():
    """N = 2^20 at rank 64 in FP32 with 4 vectors needs about 100 MB of workspace."""
    w = si.GRID1024_GAUSS
    op = h2.H2Operator(w.make_points(), w.kernel, w.leaf_size, w.cheb_order, w.eta).upload("fp32")
    nv = 4
    assert h2.h2_workspace_bytes(op.handle, nv) > h2.H2_NOALLOC_SCRATCH_BYTES
    X = op.new_vectors(nv, fill=1.0)
    Y = op.new_vectors(nv, fill=0.0)
    with pytest.raises(h2.H2Error) as e:
        h2.h2_matvec_noalloc(op.handle, X, Y, nv, 1.0, 0.0)
    assert e.value.status == h2.H2_EINVAL
    op.close()
