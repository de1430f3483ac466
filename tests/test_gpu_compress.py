"""GPU recompression (Sec. 5, h2_compress) against the oracle's recompression.

Parity: the level ranks are equal, the low-rank norm agrees to 1e-12 and the energy of the
dropped singular values to 1e-6, and the compressed operator's products agree with the
oracle's compressed products to max(1e-10, 1e3 eps / tau) for tau >= 1e-7 (FP64 upload:
there the GPU's downsweep accumulates Gram matrices where the oracle follows the paper's QR
factorizations, which resolves a node's singular values to about eps sigma_1^2 / sigma),
1e-9 below it (both sides take QR updates) and 1e-5 with an FP32 upload, relative l2. Random point sets are used for the element-wise parity
(no exactly repeated singular values, so the kept subspaces are unique); grids and the
full-size 2D workload are checked through properties that hold at any size: the error
bound of the dropped singular values, orthonormal compressed bases, and the ranks.
"""
import numpy as np
import pytest

import oracle
import oracle.compress as oc
import synthetic_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2109_05451_gb300 as h2  # noqa: E402

CLOUDS = {
    "cloud3d_exp_k27": lambda: (si.uniform_cloud(3000, 3, 2), ("exp", 0.2, 0, 0), 32, 3, 0.95),
    "cloud3d_exp_k64": lambda: (si.uniform_cloud(6000, 3, 0), ("exp", 0.2, 0, 0), 64, 4, 0.95),
    "cloud2d_imq_k36_ragged": lambda: (si.uniform_cloud(3001, 2, 9), ("imq", 1e-4, 1.5, 0), 40, 6, 0.7),
    "cloud2d_exp_k36_deficient": lambda: (si.uniform_cloud(2000, 2, 3), ("exp", 0.1, 0, 0), 24, 6, 0.9),
    "cloud1d_gauss_k8": lambda: (si.uniform_cloud(999, 1, 4), ("gauss", 0.01, 0, 0), 16, 8, 1.0),
}
# The downsweep works with Gram matrices (B^T B of each stacked block row), so a node's singular
# values are resolved to about eps * sigma_1^2 / sigma: the kept directions near the cut
# tau * sigma_1 carry relative errors of order eps / tau against the oracle's QR path.
EPS = 2.220446049250313e-16


def tol(prec, tau):
    if prec == "fp32":
        return 1e-5
    return max(1e-10, 1e3 * EPS / tau) if tau >= 1e-7 else 1e-9  # Gram route / QR route
DT = {"fp64": torch.float64, "fp32": torch.float32}


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def gpu_matvec(op, X, prec):
    Xd = torch.from_numpy(np.ascontiguousarray(X.T)).to(device="cuda", dtype=DT[prec]).t()
    Yd = op.new_vectors(X.shape[1], fill=float("nan"))
    op.matvec(Xd, Yd)
    torch.cuda.synchronize()
    return Yd.t().contiguous().cpu().double().numpy().T


@pytest.fixture(scope="module")
def built():
    cache = {}

    def get(name, tau):
        if name not in cache:
            pts, ker, m, p, eta = CLOUDS[name]()
            cache[name] = (pts, oracle.OracleH2(pts, ker, m, p, eta), h2.H2Operator(pts, ker, m, p, eta))
        pts, orc, op = cache[name]
        key = (name, tau)
        if key not in cache:
            cache[key] = (oc.CompressedH2(orc, tau), op.compress(tau))
        return (pts, orc, op) + cache[key]
    return get


@pytest.mark.parametrize("tau", [1e-3, 1e-6, 1e-8])
@pytest.mark.parametrize("name", sorted(CLOUDS))
def test_ranks_norm_and_dropped_energy_match_the_oracle(built, name, tau):
    pts, orc, op, c, g = built(name, tau)
    info = g.compress_info
    assert g.level_ranks == c.ranks
    assert list(info.level_rank)[:c.q + 1] == c.ranks
    assert info.rank_out == max(1, max(c.ranks)) and info.rank_in == c.k and info.depth == c.q
    assert abs(info.norm_lowrank - c.norm_lr) <= 1e-12 * c.norm_lr
    dropped = sum(float(np.sum(d ** 2)) for d in c.dropped.values())
    assert abs(info.dropped_energy - dropped) <= 1e-6 * dropped + 1e-13 * c.norm_lr ** 2
    before, after = c.lowrank_bytes()
    assert (info.lowrank_bytes_in, info.lowrank_bytes_out) == (before, after)
    assert all(ms >= 0 for ms in info.ms) and info.jacobi_sweeps > 0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("tau", [1e-3, 1e-6, 1e-8])
@pytest.mark.parametrize("name", sorted(CLOUDS))
def test_compressed_products_match_the_oracle(built, name, tau, prec):
    pts, orc, op, c, g = built(name, tau)
    g.upload(prec)
    X = si.gaussian_vectors(len(pts), 3, 11)
    assert rel(gpu_matvec(g, X, prec), c.matvec(X)) <= tol(prec, tau)


@pytest.mark.parametrize("name", ["cloud3d_exp_k27", "cloud2d_exp_k36_deficient"])
def test_tau_zero_keeps_the_operator(built, name):
    pts, orc, op, c, g = built(name, 0.0)
    g.upload("fp64")
    X = si.gaussian_vectors(len(pts), 2, 5)
    assert rel(gpu_matvec(g, X, "fp64"), orc.matvec(X)) <= 1e-11


def test_polynomial_kernel_reaches_its_separation_rank():
    pts = si.uniform_cloud(1600, 2, 6)
    ker = ("poly", 0, 0, 2)
    op = h2.H2Operator(pts, ker, 32, 4, 0.7)
    g = op.compress(1e-10)  # the QR route: the tenth singular value is zero, the ninth small
    ranks = g.level_ranks
    l0 = next(l for l, r in enumerate(ranks) if r > 0)
    assert ranks[l0:] == [9] * (len(ranks) - l0) and g.compress_info.rank_out == 9
    g.upload("fp64")
    X = si.gaussian_vectors(len(pts), 2, 5)
    assert rel(gpu_matvec(g, X, "fp64"), oracle.dense_kx(pts, ker, X)) <= 1e-10


def test_compressed_operator_save_load_and_recompression(built, tmp_path):
    pts, orc, op, c, g = built("cloud3d_exp_k27", 1e-6)
    path = str(tmp_path / "c.h2")
    g.save(path)
    g2 = h2.H2Operator.load(path)
    assert g2.level_ranks == g.level_ranks
    U1, E1 = h2.h2_get_bases(g.handle)
    U2, E2 = h2.h2_get_bases(g2.handle)
    assert np.array_equal(U1, U2) and np.array_equal(E1, E2)
    g.upload("fp64")
    g2.upload("fp64")
    X = si.gaussian_vectors(len(pts), 2, 7)
    assert np.array_equal(gpu_matvec(g, X, "fp64"), gpu_matvec(g2, X, "fp64"))
    # compressing the compressed operator again with a coarser tolerance: ranks fall and
    # the error against the original stays under both compressions' bounds
    g3 = g2.compress(1e-3)
    assert all(a <= b for a, b in zip(g3.level_ranks, g.level_ranks))
    g3.upload("fp64")
    x = si.gaussian_vectors(len(pts), 1, 9)
    err = np.linalg.norm(gpu_matvec(g3, x, "fp64") - orc.matvec(x))
    bound = 2 * (np.sqrt(g.compress_info.dropped_energy) + np.sqrt(g3.compress_info.dropped_energy))
    assert err <= bound * np.linalg.norm(x) * (1 + 1e-9)
    for o in (g2, g3):
        o.close()


def test_bf16_and_matrix_free_uploads_of_a_compressed_operator_are_refused(built):
    pts, orc, op, c, g = built("cloud3d_exp_k27", 1e-3)
    for prec in ("bf16x2", "fp32mf"):
        with pytest.raises(h2.H2Error):
            g.upload(prec)


@pytest.fixture(scope="module")
def grid_workload():
    """The paper's 2D compression set at N = 2^14: a grid, exp(-r/0.1), m 64, 6 x 6
    Chebyshev points (k 36), eta 0.9, tau 1e-3."""
    pts = si.grid_2d(128)
    ker = ("exp", 0.1, 0, 0)
    orc = oracle.OracleH2(pts, ker, 64, 6, 0.9)
    op = h2.H2Operator(pts, ker, 64, 6, 0.9)
    return pts, orc, op, oc.CompressedH2(orc, 1e-3), op.compress(1e-3)


def test_grid_2d_workload_ranks_error_bound_and_orthonormal_bases(grid_workload):
    pts, orc, op, c, g = grid_workload
    info = g.compress_info
    assert g.level_ranks == c.ranks
    g.upload("fp64")
    X = si.gaussian_vectors(len(pts), 1, 3)
    Y = gpu_matvec(g, X, "fp64")
    err = np.linalg.norm(Y - orc.matvec(X))
    assert err <= 2 * np.sqrt(info.dropped_energy) * np.linalg.norm(X) * (1 + 1e-9)
    assert err / np.linalg.norm(orc.matvec(X)) <= 1e-2  # relative accuracy of the order of tau
    assert rel(Y, c.matvec(X)) <= 1e-6  # same ranks; kept subspaces may differ only at repeated singular values
    U, E = h2.h2_get_bases(g.handle)
    lo, hi = orc.ranges()
    first = 2 ** c.q
    kc, r = info.rank_out, c.ranks
    for t in (first, first + 77, c.nnodes):
        Ut = U[lo[t]:hi[t], :r[c.q]]
        assert np.allclose(Ut.T @ Ut, np.eye(r[c.q]), atol=1e-12)
    for t in (1, 2, 5, first // 2, first - 1):
        l = int(t).bit_length() - 1
        if l + 1 > c.q or r[l] == 0:
            continue
        stack = np.vstack([E[2 * t][:r[l + 1], :r[l]], E[2 * t + 1][:r[l + 1], :r[l]]])
        assert np.allclose(stack.T @ stack, np.eye(r[l]), atol=1e-12)
    assert info.lowrank_bytes_out < info.lowrank_bytes_in / 2


def test_full_size_2d_workload_error_bound_on_sampled_leaves():
    """The paper's 2D compression set at N = 2^20 (1024 x 1024 grid, exp(-r/0.1), m 64,
    k 36, eta 0.9, tau 1e-3), as the benchmark compresses it: the compressed FP64 product on
    the rows of sampled leaves (the oracle computes the original operator's rows exactly)
    stays within the bound of the dropped singular values."""
    pts = si.grid_2d(1024)
    ker = ("exp", 0.1, 0, 0)
    op = h2.H2Operator(pts, ker, 64, 6, 0.9)
    g = op.compress(1e-3)
    info = g.compress_info
    assert info.depth == 14 and info.rank_in == 36 and 1 <= info.rank_out <= 36
    assert info.lowrank_bytes_out < info.lowrank_bytes_in / 2
    orc = oracle.OracleH2(pts, ker, 64, 6, 0.9)
    x = si.gaussian_vectors(len(pts), 1, 1)
    first = 2 ** orc.depth
    leaves = np.array([first, first + 5000, orc.nnodes])
    rows, ref = orc.matvec_leaves(x, leaves)
    g.upload("fp64")
    y = gpu_matvec(g, x, "fp64")
    err = np.linalg.norm(y[rows] - ref)
    assert err <= 2 * np.sqrt(info.dropped_energy) * np.linalg.norm(x) * (1 + 1e-9)
    assert err / np.linalg.norm(ref) <= 1e-2
    assert np.all(np.isfinite(y))


@pytest.mark.parametrize("pts,m,eta", [
    (si.uniform_cloud(7, 2, 1), 64, 0.9),      # one leaf: no tree above it, no coupling block
    (si.grid_2d(20), 16, 1e-9),                # nothing admissible: every block dense
])
def test_degenerate_partitions(pts, m, eta):
    ker = ("exp", 0.1, 0, 0)
    orc = oracle.OracleH2(pts, ker, m, 4, eta)
    op = h2.H2Operator(pts, ker, m, 4, eta)
    g = op.compress(1e-3)
    info = g.compress_info
    assert info.norm_lowrank == 0.0 and info.rank_out == 1 and max(g.level_ranks) == 0
    g.upload("fp64")
    X = si.gaussian_vectors(len(pts), 2, 4)
    assert rel(gpu_matvec(g, X, "fp64"), orc.matvec(X)) <= 1e-13


def test_coarse_tolerance_matches_the_oracle(built):
    pts, orc, op, c, g = built("cloud3d_exp_k27", 0.5)
    assert g.level_ranks == c.ranks and max(c.ranks) <= 3
    g.upload("fp64")
    X = si.gaussian_vectors(len(pts), 2, 6)
    assert rel(gpu_matvec(g, X, "fp64"), c.matvec(X)) <= tol("fp64", 0.5)
