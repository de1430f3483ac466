"""GPU parity: libh2's CUDA product against the FP64 CPU oracle, through the C ABI.

Tolerances (relative l2 over the compared entries): 1e-12 for FP64, 1e-5 for FP32.
Small cases compare every output entry; the full-size 2^20 grid compares the output
rows of sampled leaves that the oracle computes exactly (its upsweep is complete and
its tree multiply / downsweep follow each sampled leaf's ancestors).
"""
import numpy as np
import pytest

import oracle
import synthetic_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2109_05451_gb300 as h2  # noqa: E402

TOL = {"fp64": 1e-12, "fp32": 1e-5, "fp32mf": 1e-5}
DT = {"fp64": torch.float64, "fp32": torch.float32, "fp32mf": torch.float32}


def relerr(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def to_dev(X, prec):
    X = np.asfortranarray(X)
    return torch.from_numpy(np.ascontiguousarray(X.T)).to(device="cuda", dtype=DT[prec]).t()


def to_host(Y):
    return Y.t().contiguous().cpu().double().numpy().T


def gpu_matvec(op, X, prec, alpha=1.0, beta=0.0, Y0=None):
    Xd = to_dev(X, prec)
    Yd = to_dev(Y0, prec) if Y0 is not None else op.new_vectors(X.shape[1], fill=float("nan"))
    op.matvec(Xd, Yd, alpha=alpha, beta=beta)
    torch.cuda.synchronize()
    return to_host(Yd)


CASES = {
    "grid64_exp": lambda: (si.grid_2d(64), ("exp", 0.1, 0, 0), 64, 4, 0.9),
    "grid37_gauss_k25": lambda: (si.grid_2d(37), ("gauss", 0.01, 0, 0), 32, 5, 0.7),
    "cloud3d_k64": lambda: (si.uniform_cloud(6000, 3, 0), ("exp", 0.2, 0, 0), 64, 4, 0.7),
    "cloud3d_k27_ragged": lambda: (si.uniform_cloud(3001, 3, 5), ("exp", 0.2, 0, 0), 40, 3, 0.7),
    "cloud1d_imq": lambda: (si.uniform_cloud(999, 1, 4), ("imq", 1e-4, 1.5, 0), 16, 6, 1.0),
    "poly_exact": lambda: (si.uniform_cloud(2000, 2, 6), ("poly", 0, 0, 3), 32, 4, 0.7),
    "tiny_single_leaf": lambda: (si.uniform_cloud(7, 2, 1), ("exp", 0.1, 0, 0), 64, 4, 0.9),
    "all_dense": lambda: (si.grid_2d(20), ("exp", 0.1, 0, 0), 16, 4, 1e-9),
}


@pytest.fixture(scope="module")
def built():
    cache = {}

    def get(name):
        if name not in cache:
            pts, ker, m, p, eta = CASES[name]()
            cache[name] = (pts, ker, oracle.OracleH2(pts, ker, m, p, eta), h2.H2Operator(pts, ker, m, p, eta))
        return cache[name]
    return get


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_matvec_matches_oracle(built, name, prec):
    pts, ker, orc, op = built(name)
    op.upload(prec)
    X = si.gaussian_vectors(len(pts), 1, 1)
    ref = orc.matvec(X)
    got = gpu_matvec(op, X, prec)
    assert np.all(np.isfinite(got))
    assert relerr(got, ref) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_alpha_beta_and_nan_output(built, prec):
    pts, ker, orc, op = built("cloud3d_k64")
    op.upload(prec)
    X = si.gaussian_vectors(len(pts), 2, 1)
    Y0 = si.gaussian_vectors(len(pts), 2, 2)
    assert relerr(gpu_matvec(op, X, prec, 0.75, -1.25, Y0), orc.matvec(X, 0.75, -1.25, Y0)) <= TOL[prec]
    # beta = 0: Y (NaN here) is not read
    got = gpu_matvec(op, X, prec, 2.0, 0.0)
    assert np.all(np.isfinite(got)) and relerr(got, orc.matvec(X, 2.0)) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_multi_rhs_columns_and_repeatability(built, prec):
    pts, ker, orc, op = built("grid37_gauss_k25")
    op.upload(prec)
    X = si.gaussian_vectors(len(pts), 5, 3)
    Y = gpu_matvec(op, X, prec)
    assert relerr(Y, orc.matvec(X)) <= TOL[prec]
    for v in (0, 3):
        Yv = gpu_matvec(op, X[:, v:v + 1], prec)
        assert relerr(Yv[:, 0], Y[:, v]) <= 10 * np.finfo(np.float32 if prec == "fp32" else np.float64).eps
    assert np.array_equal(gpu_matvec(op, X, prec), Y)  # bitwise repeatable (no atomics)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("nv", [5, 8, 13, 32, 37])
@pytest.mark.parametrize("name", sorted(CASES))
def test_wide_passes_match_oracle(built, name, nv, prec):
    """More than 4 vectors: one pass of up to 32 vectors on the wide kernels (37 = 32 + a
    4-vector tail), every tile read once per pass."""
    pts, ker, orc, op = built(name)
    op.upload(prec)
    X = si.gaussian_vectors(len(pts), nv, 11)
    Y0 = si.gaussian_vectors(len(pts), nv, 12)
    got = gpu_matvec(op, X, prec, 0.5, 2.0, Y0)
    assert np.all(np.isfinite(got))
    assert relerr(got, orc.matvec(X, 0.5, 2.0, Y0)) <= TOL[prec]


def test_wide_fallback_for_large_leaves():
    """Leaves of more than 64 points keep the 4-vector chunks for any vector count."""
    pts = si.uniform_cloud(3000, 2, 9)
    ker = ("exp", 0.2, 0, 0)
    orc = oracle.OracleH2(pts, ker, 100, 4, 0.7)
    op = h2.H2Operator(pts, ker, 100, 4, 0.7).upload("fp32")
    X = si.gaussian_vectors(len(pts), 9, 13)
    assert relerr(gpu_matvec(op, X, "fp32"), orc.matvec(X)) <= TOL["fp32"]
    op.close()


@pytest.mark.parametrize("nv", [1, 3, 6])
@pytest.mark.parametrize("name", sorted(CASES))
def test_matrix_free_matches_oracle(built, name, nv):
    """Coupling and dense entries evaluated in FP32 inside the product (no blocks stored):
    the same structure, so the oracle's product is the reference (1e-5)."""
    pts, ker, orc, op = built(name)
    op.upload("fp32mf")
    assert h2.h2_get_info(op.handle).uploaded_prec == h2.H2_FP32_MF
    X = si.gaussian_vectors(len(pts), nv, 21)
    Y0 = si.gaussian_vectors(len(pts), nv, 22)
    got = gpu_matvec(op, X, "fp32mf", 1.25, -0.5, Y0)
    assert np.all(np.isfinite(got))
    assert relerr(got, orc.matvec(X, 1.25, -0.5, Y0)) <= TOL["fp32mf"]


def test_workspace_entry_point(built):
    pts, ker, orc, op = built("grid64_exp")
    op.upload("fp64")
    nv = 2
    X = si.gaussian_vectors(len(pts), nv, 7)
    Xd = to_dev(X, "fp64")
    Yd = op.new_vectors(nv, fill=0.0)
    nbytes = h2.h2_workspace_bytes(op.handle, nv)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    with pytest.raises(h2.H2Error):
        h2.h2_matvec_ws(op.handle, Xd, Yd, nv, 1.0, 0.0, ws, nbytes - 1)
    h2.h2_matvec_ws(op.handle, Xd, Yd, nv, 1.0, 0.0, ws, nbytes)
    torch.cuda.synchronize()
    assert relerr(to_host(Yd), orc.matvec(X)) <= TOL["fp64"]


@pytest.fixture(scope="module")
def grid1024():
    w = si.GRID1024_GAUSS
    pts = w.make_points()
    orc = oracle.OracleH2(pts, w.kernel, w.leaf_size, w.cheb_order, w.eta)
    op = h2.H2Operator(pts, w.kernel, w.leaf_size, w.cheb_order, w.eta)
    X = w.make_x(len(pts))
    rng = np.random.default_rng(123)
    first = 2 ** orc.depth
    leaves = np.unique(np.concatenate([[first, first + 1, orc.nnodes],
                                       rng.integers(first, orc.nnodes + 1, 29)]))
    rows, ref = orc.matvec_leaves(X, leaves)
    return w, op, X, rows, ref, orc


@pytest.mark.parametrize("prec", ["fp32", "fp64", "fp32mf"])
def test_full_size_grid1024_sampled_leaves(grid1024, prec):
    """N = 2^20 Gaussian grid, rank 64, eta 0.7, nv = 1 -- the benchmarked workload."""
    w, op, X, rows, ref, orc = grid1024
    info = h2.h2_get_info(op.handle)
    assert info.depth == orc.depth == 14 and info.rank == 64
    lvl, _, _, dt, _ = orc.blocks()
    assert info.n_coupling == len(lvl) == 483456 and info.n_dense == len(dt) == 145924
    assert [info.coupling_per_level[l] for l in range(15)] == np.bincount(lvl, minlength=15).tolist()
    op.upload(prec)
    got = gpu_matvec(op, X, prec)
    assert np.all(np.isfinite(got))
    assert relerr(got[rows], ref) <= TOL[prec]
    op.upload("fp32")  # leave the cheaper copy resident for later tests


# ---------------------------------------------------------------- split-BF16 tensor-core path

@pytest.mark.parametrize("nv", [1, 7, 32])
@pytest.mark.parametrize("name", sorted(CASES))
def test_bf16x2_tensor_path_matches_oracle(built, name, nv):
    """Blocks as bf16 hi + lo, three MMA terms, FP32 accumulation in tensor memory (<= 1e-4)."""
    pts, ker, orc, op = built(name)
    op.upload("bf16x2")
    X = si.gaussian_vectors(len(pts), nv, 2)
    got = gpu_matvec(op, X, "fp32")
    assert np.all(np.isfinite(got))
    assert relerr(got, orc.matvec(X)) <= 1e-4


def test_bf16x2_alpha_beta_and_repeatability(built):
    pts, ker, orc, op = built("cloud3d_k64")
    op.upload("bf16x2")
    X = si.gaussian_vectors(len(pts), 20, 3)
    Y0 = si.gaussian_vectors(len(pts), 20, 4)
    got = gpu_matvec(op, X, "fp32", 1.5, -0.5, Y0)
    assert relerr(got, orc.matvec(X, 1.5, -0.5, Y0)) <= 1e-4
    assert np.array_equal(gpu_matvec(op, X, "fp32", 1.5, -0.5, Y0), got)


@pytest.fixture(scope="module")
def cloud3d_medium():
    """The 3D multi-RHS workload's distribution at N = 2^17 (uniform cloud, exp(-r/0.2),
    leaf 64, tri-cubic rank 64, eta 0.7, 32 vectors)."""
    w = si.cloud3d(2 ** 17)
    pts = w.make_points()
    orc = oracle.OracleH2(pts, w.kernel, w.leaf_size, w.cheb_order, w.eta)
    op = h2.H2Operator(pts, w.kernel, w.leaf_size, w.cheb_order, w.eta)
    X = w.make_x(len(pts))
    rng = np.random.default_rng(5)
    first = 2 ** orc.depth
    leaves = np.unique(np.concatenate([[first, orc.nnodes], rng.integers(first, orc.nnodes + 1, 14)]))
    rows, ref = orc.matvec_leaves(X, leaves)
    return op, X, rows, ref


@pytest.mark.parametrize("prec,tol", [("bf16x2", 1e-4), ("fp32", 1e-5)])
def test_cloud3d_multi_rhs_sampled_leaves(cloud3d_medium, prec, tol):
    op, X, rows, ref = cloud3d_medium
    op.upload(prec)
    got = gpu_matvec(op, X, "fp32")
    assert np.all(np.isfinite(got))
    assert relerr(got[rows], ref) <= tol


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32mf"])
def test_loaded_operator_gives_the_same_product(built, prec, tmp_path):
    pts, ker, orc, op = built("cloud3d_k27_ragged")
    path = str(tmp_path / "op.h2")
    op.save(path)
    g = h2.H2Operator.load(path).upload(prec)
    try:
        op.upload(prec)
        X = si.gaussian_vectors(len(pts), 3, 8)
        Y = gpu_matvec(op, X, prec)
        assert np.array_equal(gpu_matvec(g, X, prec), Y)
        assert relerr(Y, orc.matvec(X)) <= TOL[prec]
    finally:
        g.close()


@pytest.mark.parametrize("nv", [9, 16, 32])
@pytest.mark.parametrize("name", ["cloud3d_k64", "grid37_gauss_k25", "cloud3d_k27_ragged", "all_dense"])
def test_fp32_tensor_and_cuda_core_passes_agree(built, name, nv):
    """FP32 passes of more than 8 vectors: the 3xTF32 tensor-core stream (default) and the
    CUDA-core FMA stream each meet the FP32 tolerance against the oracle; the two differ by
    FP32 rounding only."""
    pts, ker, orc, op = built(name)
    op.upload("fp32")
    X = si.gaussian_vectors(len(pts), nv, 31)
    Y0 = si.gaussian_vectors(len(pts), nv, 32)
    ref = orc.matvec(X, 0.75, 0.5, Y0)
    h2.h2_set_fp32_tensor(op.handle, False)
    try:
        cuda_cores = gpu_matvec(op, X, "fp32", 0.75, 0.5, Y0)
    finally:
        h2.h2_set_fp32_tensor(op.handle, True)
    tensor = gpu_matvec(op, X, "fp32", 0.75, 0.5, Y0)
    assert np.all(np.isfinite(tensor))
    assert relerr(cuda_cores, ref) <= TOL["fp32"]
    assert relerr(tensor, ref) <= TOL["fp32"]
    assert relerr(tensor, cuda_cores) <= TOL["fp32"]
    assert np.array_equal(gpu_matvec(op, X, "fp32", 0.75, 0.5, Y0), tensor)  # no atomics on data


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_small_ranks_stream_dense_rows_apart(built, prec):
    """Rank 16 with 64-point leaves: the dense tiles are 4x the coupling tiles, so the lower
    levels' coupling rows and the dense rows run as two streams (the coupling rows with
    several CTAs per SM); the product still matches the oracle, at 1 and at 4 vectors."""
    pts, ker, orc, op = built("grid64_exp")
    op.upload(prec)
    for nv in (1, 4):
        X = si.gaussian_vectors(len(pts), nv, 41)
        h2.h2_get_timing(op.handle)
        got = gpu_matvec(op, X, prec)
        _, launches, products = h2.h2_get_timing(op.handle)
        assert products == 1 and launches[1] == 2  # coupling stream + dense stream
        assert relerr(got, orc.matvec(X)) <= TOL[prec]
    # rank 64 with 64-point leaves: one stream for both
    pts64, _, orc64, op64 = built("cloud3d_k64")
    op64.upload(prec)
    h2.h2_get_timing(op64.handle)
    gpu_matvec(op64, si.gaussian_vectors(len(pts64), 1, 42), prec)
    _, launches, _ = h2.h2_get_timing(op64.handle)
    assert launches[1] == 1


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("dim,order,leaf", [(2, 3, 128), (3, 3, 100)])
def test_small_rank_warp_kernels_with_large_leaves(prec, dim, order, leaf):
    """Ranks of at most 32 sweep the tree with one warp per node and stream the coupling rows
    with one warp per chunk of rows at one vector; leaves of more than 64 points take their
    rows beyond 64 in a second round. Each column against the oracle with alpha and beta, and
    the 2-vector product (the staged kernels) against the oracle too."""
    pts = si.uniform_cloud(9000 if dim == 2 else 6000, dim, 7 + dim)
    ker = ("exp", 0.1 if dim == 2 else 0.2, 0, 0)
    orc = oracle.OracleH2(pts, ker, leaf, order, 0.8)
    op = h2.H2Operator(pts, ker, leaf, order, 0.8).upload(prec)
    try:
        assert op.info.rank == order ** dim and op.info.rank <= 32
        X = si.gaussian_vectors(len(pts), 2, 21)
        Y0 = si.gaussian_vectors(len(pts), 2, 22)
        for v in range(2):
            got = gpu_matvec(op, X[:, v:v + 1], prec, 0.75, -1.25, Y0[:, v:v + 1])
            assert np.all(np.isfinite(got))
            assert relerr(got, orc.matvec(X[:, v:v + 1], 0.75, -1.25, Y0[:, v:v + 1])) <= TOL[prec]
        got = gpu_matvec(op, X[:, :1], prec, 2.0, 0.0)  # beta = 0: the NaN output is not read
        assert np.all(np.isfinite(got)) and relerr(got, orc.matvec(X[:, :1], 2.0)) <= TOL[prec]
        both = gpu_matvec(op, X, prec, 0.75, -1.25, Y0)
        assert relerr(both, orc.matvec(X, 0.75, -1.25, Y0)) <= TOL[prec]
        assert np.array_equal(gpu_matvec(op, X[:, :1], prec, 2.0, 0.0), got)  # deterministic
    finally:
        op.close()
