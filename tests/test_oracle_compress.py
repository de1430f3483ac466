"""Pins of the oracle's recompression (Sec. 5), each against something other than the
compression code itself: the explicit (densely assembled) low-rank part of the original
operator, orthonormality, the separation rank of polynomial kernels, the SVD truncation
property and the bound of the dropped singular values."""
import numpy as np
import pytest

import oracle
import oracle.compress as oc
import synthetic_inputs as si

CASES = {
    # 2D grid, rank 36 above 16-point leaves: every leaf basis is rank-deficient
    "grid32_exp_k36_deficient": lambda: (si.grid_2d(32), ("exp", 0.1, 0, 0), 16, 6, 0.9),
    "grid32_exp_k16": lambda: (si.grid_2d(32), ("exp", 0.1, 0, 0), 16, 4, 0.9),
    "cloud3d_exp_k27": lambda: (si.uniform_cloud(1500, 3, 2), ("exp", 0.2, 0, 0), 32, 3, 0.95),
    "cloud2d_imq_ragged": lambda: (si.uniform_cloud(1100, 2, 9), ("imq", 1e-4, 1.5, 0), 24, 5, 0.7),
}


@pytest.fixture(scope="module")
def built():
    cache = {}

    def get(name, tau):
        key = (name, tau)
        if name not in cache:
            pts, ker, m, p, eta = CASES[name]()
            orc = oracle.OracleH2(pts, ker, m, p, eta)
            cache[name] = (orc, oc.lowrank_part(orc))
        orc, alr = cache[name]
        if key not in cache:
            cache[key] = oc.CompressedH2(orc, tau)
        return orc, alr, cache[key]
    return get


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def nodes_sample(c):
    first = c.first
    out = {1, 2, 3, min(7, c.nnodes), first, first + 1, c.nnodes, (first + c.nnodes) // 2}
    return sorted(t for t in out if 1 <= t <= c.nnodes)


@pytest.mark.parametrize("name", sorted(CASES))
def test_orthogonalized_operator_equals_the_original(built, name):
    orc, alr, c = built(name, 1e-3)
    assert rel(c.assemble_lowrank("orthogonal"), alr) <= 1e-12
    for t in nodes_sample(c):
        B = c.nested_basis(t, orthogonal_only=True)
        G = B.T @ B
        d = np.round(np.diag(G))
        assert np.all((d == 0) | (d == 1))
        assert np.max(np.abs(G - np.diag(d))) <= 1e-12
        assert int(d.sum()) <= min(B.shape)
        if t >= c.first:
            assert int(d.sum()) == min(c.hi[t] - c.lo[t], c.k)


@pytest.mark.parametrize("name", sorted(CASES))
def test_downsweep_factors_reproduce_each_block_rows_gram_matrix(built, name):
    orc, alr, c = built(name, 1e-3)
    # the leaves' factors hold the whole low-rank part
    assert abs(c.norm_lr - np.linalg.norm(alr)) <= 1e-12 * np.linalg.norm(alr)
    lo, hi = c.lo, c.hi
    for i in nodes_sample(c):
        # A_i: rows of node i, the blocks of node i's row and of its ancestors' rows
        cols = np.zeros(orc.n, dtype=bool)
        t = i
        while t >= 1:
            for b in c.rows.get(t, []):
                s = int(c.blk_s[b])
                cols[lo[s]:hi[s]] = True
            t //= 2
        Ai = alr[lo[i]:hi[i]] * cols
        B = c.nested_basis(i, orthogonal_only=True)
        got = B @ c.Rh[i].T @ c.Rh[i] @ B.T
        ref = Ai @ Ai.T
        scale = max(np.linalg.norm(ref), 1e-300)
        assert np.linalg.norm(got - ref) <= 1e-11 * scale or np.linalg.norm(ref) == 0 == np.linalg.norm(got)
        assert abs(np.linalg.norm(c.Rh[i]) - np.linalg.norm(Ai)) <= 1e-12 * max(np.linalg.norm(alr), 1.0)


@pytest.mark.parametrize("name", sorted(CASES))
def test_tau_zero_reproduces_the_operator(built, name):
    orc, alr, c = built(name, 0.0)
    assert rel(c.assemble_lowrank(), alr) <= 1e-11
    X = si.gaussian_vectors(orc.n, 2, 3)
    assert rel(c.matvec(X), orc.matvec(X)) <= 1e-12


def test_polynomial_kernel_compresses_to_its_separation_rank():
    # prod_d (1 + x_d y_d)^2 in 2D: every far-field block row has rank (2+1)^2 = 9 < k = 16
    pts = si.uniform_cloud(1600, 2, 6)
    ker = ("poly", 0, 0, 2)
    orc = oracle.OracleH2(pts, ker, 32, 4, 0.7)
    c = oc.CompressedH2(orc, 1e-10)
    l0 = int(min(c.blk_level))  # levels above the first coupling block have nothing to represent
    assert c.ranks[:l0] == [0] * l0 and c.ranks[l0:] == [9] * (c.q + 1 - l0)
    X = si.gaussian_vectors(orc.n, 2, 5)
    assert rel(c.matvec(X), oracle.dense_kx(pts, ker, X)) <= 1e-10
    before, after = c.lowrank_bytes()
    assert after < before * (9 / 16) ** 2 * 1.2


@pytest.mark.parametrize("name", sorted(CASES))
def test_leaf_truncation_residual_stays_under_the_relative_cut(built, name):
    orc, alr, c = built(name, 1e-3)
    for t in range(c.first, c.nnodes + 1):
        M = c.Q[t] @ c.Rh[t].T
        res = M - c.U[t] @ (c.U[t].T @ M)
        assert np.linalg.norm(res, 2) <= 1e-3 * np.linalg.norm(M, 2) * (1 + 1e-9) + 1e-13 * c.norm_lr


@pytest.mark.parametrize("name", sorted(CASES))
def test_error_under_the_dropped_singular_value_bound_and_falling_with_tau(built, name):
    errs = []
    for tau in (1e-2, 1e-4, 1e-6):
        orc, alr, c = built(name, tau)
        err = np.linalg.norm(c.assemble_lowrank() - alr)
        bound = 2.0 * np.sqrt(sum(float(np.sum(d ** 2)) for d in c.dropped.values()))
        assert err <= bound * (1 + 1e-8) + 1e-12 * np.linalg.norm(alr)
        # every dropped singular value is under tau times its node's largest
        assert all(len(d) == 0 or d[0] <= tau * c.sigma[t][0] * (1 + 1e-12) or d[0] <= 1e-13 * c.norm_lr
                   for t, d in c.dropped.items())
        errs.append(err)
        for t in nodes_sample(c):  # compressed bases stay orthonormal
            B = c.nested_basis(t)
            G = B.T @ B
            d = np.round(np.diag(G))
            assert G.size == 0 or np.max(np.abs(G - np.diag(d))) <= 1e-11
    assert errs[0] > errs[1] > errs[2]


def test_ranks_are_uniform_per_level_and_shrink_the_operator(built):
    orc, alr, c = built("cloud3d_exp_k27", 1e-3)
    assert all(0 <= r <= c.k for r in c.ranks)
    for l in range(1, c.q + 1):
        for t in range(1 << l, 2 << l):
            assert c.E[t].shape == (c.ranks[l], c.ranks[l - 1])
    for b, l in enumerate(c.blk_level):
        assert c.S[b].shape == (c.ranks[l], c.ranks[l])
    before, after = c.lowrank_bytes()
    assert after < before


@pytest.mark.parametrize("pts,m,eta", [
    (si.uniform_cloud(7, 2, 1), 64, 0.9),      # one leaf: no tree above it, no coupling block
    (si.grid_2d(20), 16, 1e-9),                # nothing admissible: every block dense
])
def test_degenerate_partitions_compress_to_the_same_operator(pts, m, eta):
    orc = oracle.OracleH2(pts, ("exp", 0.1, 0, 0), m, 4, eta)
    c = oc.CompressedH2(orc, 1e-3)
    assert len(c.blk_t) == 0 and max(c.ranks) == 0 and c.norm_lr == 0.0
    X = si.gaussian_vectors(len(pts), 2, 4)
    assert rel(c.matvec(X), orc.matvec(X)) <= 1e-14


def test_coarse_tolerance_keeps_the_bound(built):
    orc, alr, c = built("cloud3d_exp_k27", 0.5)
    err = np.linalg.norm(c.assemble_lowrank() - alr)
    bound = 2.0 * np.sqrt(sum(float(np.sum(d ** 2)) for d in c.dropped.values()))
    assert err <= bound * (1 + 1e-8) and max(c.ranks) <= 3


def test_3d_grid_set_at_a_small_size():
    # the 3D compression set's recipe (grid, exp(-r/0.2), leaf 64, tri-cubic, eta 0.95) at 12^3
    w = si.COMPRESS_3D
    pts = si.grid_3d(12)
    orc = oracle.OracleH2(pts, w.kernel, w.leaf_size, w.cheb_order, w.eta)
    alr = oc.lowrank_part(orc)
    c = oc.CompressedH2(orc, si.COMPRESS_TAU)
    err = np.linalg.norm(c.assemble_lowrank() - alr)
    bound = 2.0 * np.sqrt(sum(float(np.sum(d ** 2)) for d in c.dropped.values()))
    assert err <= bound * (1 + 1e-8) + 1e-12 * np.linalg.norm(alr)
    before, after = c.lowrank_bytes()
    assert max(c.ranks) < c.k and after < before
