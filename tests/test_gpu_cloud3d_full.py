"""GPU parity at the full size of the multi-vector workload: N = 2^21 uniform random points
in [0,1]^3, exp(-r/0.2), leaf 64, 4 x 4 x 4 Chebyshev grid (rank 64), eta 0.7, 32 Gaussian
vectors -- the configuration and launch path that bench.py times.

The oracle's complete FP64 upsweep plus the tree multiply and downsweep along the ancestors
of sampled leaves give their output rows exactly (no blocks are assembled); the GPU rows
must agree to 1e-4 (split-BF16 tensor-core stream) and 1e-5 (FP32) relative l2.
"""
import numpy as np
import pytest

import oracle
import synthetic_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2109_05451_gb300 as h2  # noqa: E402


@pytest.fixture(scope="module")
def cloud3d_full():
    w = si.CLOUD3D_EXP
    pts = w.make_points()
    orc = oracle.OracleH2(pts, w.kernel, w.leaf_size, w.cheb_order, w.eta)
    X = w.make_x(len(pts))
    rng = np.random.default_rng(21)
    first = 2 ** orc.depth
    leaves = np.unique(np.concatenate([[first, first + 1, orc.nnodes], rng.integers(first, orc.nnodes + 1, 5)]))
    rows, ref = orc.matvec_leaves(X, leaves)
    op = h2.H2Operator(pts, w.kernel, w.leaf_size, w.cheb_order, w.eta)
    yield op, X, rows, ref, orc
    op.close()


@pytest.mark.parametrize("prec,tol", [("bf16x2", 1e-4), ("fp32", 1e-5)])
def test_cloud3d_2pow21_32_vectors_sampled_leaves(cloud3d_full, prec, tol):
    op, X, rows, ref, orc = cloud3d_full
    info = h2.h2_get_info(op.handle)
    assert info.depth == orc.depth == 15 and info.rank == 64 and info.n_coupling == len(orc.blocks()[1])
    op.upload(prec)
    Xd = torch.from_numpy(np.ascontiguousarray(X.T)).to(device="cuda", dtype=torch.float32).t()
    Yd = op.new_vectors(X.shape[1], fill=float("nan"))
    op.matvec(Xd, Yd)
    torch.cuda.synchronize()
    got = Yd[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    del Xd, Yd
    assert np.all(np.isfinite(got))
    err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    assert err <= tol, err
