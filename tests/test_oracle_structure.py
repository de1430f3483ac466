"""Pins of the oracle's cluster tree, admissibility and block partition (CPU only).

Each check compares the oracle with something other than itself: a value the paper
prints (tests/golden/paper_constants.json), the definition of a partition of the index
square, the admissibility rule of Sec. 6.1 on hand-made boxes, or the invariants of a
complete binary k-d tree with the stated split rule.
"""
import collections
import json
import os

import numpy as np
import pytest

import oracle
import synthetic_inputs as si

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def _build(points, kernel=("exp", 0.1, 0.0, 0), m=64, p=4, eta=0.9):
    return oracle.OracleH2(points, kernel, m, p, eta)


POINT_SETS = {
    "grid64": lambda: si.grid_2d(64),
    "grid37": lambda: si.grid_2d(37),                 # ragged leaves (1369 points)
    "cloud3d": lambda: si.uniform_cloud(3001, 3, 7),  # ragged, 3D
    "cloud1d": lambda: si.uniform_cloud(777, 1, 3),
    "tiny": lambda: si.uniform_cloud(5, 2, 1),        # n <= m: a single leaf
}


# ---------------------------------------------------------------- admissibility rule

def test_admissibility_hand_boxes_equality_is_admissible():
    # 1D unit boxes [0,1] and [2,3]: |C_t - C_s| = 2, (D_t + D_s)/2 = 1.
    assert oracle.admissible([0.0], [1.0], [2.0], [3.0], 0.5)          # 0.5*2 = 1 >= 1
    assert not oracle.admissible([0.0], [1.0], [2.0], [3.0], 0.49)
    # 2D: unit squares with centres 3 apart along x (3-4-5 free): D = sqrt(2) each.
    assert oracle.admissible([0, 0], [1, 1], [3, 0], [4, 1], np.sqrt(2) / 3 * 1.0000001)
    assert not oracle.admissible([0, 0], [1, 1], [3, 0], [4, 1], np.sqrt(2) / 3 * 0.9999999)
    # a box is never admissible with itself unless it is a point
    assert not oracle.admissible([0, 0], [1, 1], [0, 0], [1, 1], 100.0)
    assert oracle.admissible([0.5, 0.5], [0.5, 0.5], [0.5, 0.5], [0.5, 0.5], 0.9)


# ---------------------------------------------------------------- k-d tree invariants

@pytest.mark.parametrize("name", sorted(POINT_SETS))
def test_tree_invariants(name):
    pts = POINT_SETS[name]()
    n, dim = pts.shape
    m = 64 if name != "cloud1d" else 16
    h = _build(pts, m=m)
    q = h.depth
    # depth: smallest q with n <= m 2^q
    assert n <= m * 2 ** q and (q == 0 or n > m * 2 ** (q - 1))
    assert h.nnodes == 2 ** (q + 1) - 1
    perm = h.perm
    assert np.array_equal(np.sort(perm), np.arange(n))
    lo, hi = h.ranges()
    bmin, bmax = h.boxes()
    assert lo[1] == 0 and hi[1] == n
    for t in range(1, h.nnodes + 1):
        sel = pts[perm[lo[t]:hi[t]]]
        assert hi[t] > lo[t]
        assert np.array_equal(bmin[t], sel.min(axis=0)) and np.array_equal(bmax[t], sel.max(axis=0))
        if t < 2 ** q:  # inner node: children split it at floor(n/2)
            c1, c2 = 2 * t, 2 * t + 1
            size = hi[t] - lo[t]
            assert lo[c1] == lo[t] and hi[c1] == lo[c2] == lo[t] + size // 2 and hi[c2] == hi[t]
            ext = bmax[t] - bmin[t]
            d = int(np.argmax(ext))  # first maximum = lowest dimension on ties
            left, right = pts[perm[lo[c1]:hi[c1]], d], pts[perm[lo[c2]:hi[c2]], d]
            assert left.max() <= right.min()
            # equal coordinates are ordered by original index
            if left.max() == right.min():
                v = left.max()
                li = perm[lo[c1]:hi[c1]][left == v]
                ri = perm[lo[c2]:hi[c2]][right == v]
                assert li.max() < ri.min()
    leaves = np.arange(2 ** q, 2 ** (q + 1))
    sizes = hi[leaves] - lo[leaves]
    assert sizes.max() <= m
    assert set(sizes.tolist()) <= {n // 2 ** q, -(-n // 2 ** q)}


# ---------------------------------------------------------------- block partition

@pytest.mark.parametrize("name,eta", [("grid64", 0.9), ("grid37", 0.7), ("cloud3d", 0.7), ("cloud1d", 1.5)])
def test_blocks_tile_index_square_exactly_once(name, eta):
    """Coupling leaves on all levels plus dense leaves form a partition of I x I (Sec. 2.1)."""
    pts = POINT_SETS[name]()
    n = len(pts)
    h = _build(pts, m=64 if name != "cloud1d" else 16, eta=eta)
    lo, hi = h.ranges()
    lvl, t, s, dt, ds = h.blocks()
    cover = np.zeros((n, n), dtype=np.int16)
    for a, b in zip(t, s):
        cover[lo[a]:hi[a], lo[b]:hi[b]] += 1
    for a, b in zip(dt, ds):
        cover[lo[a]:hi[a], lo[b]:hi[b]] += 1
    assert cover.min() == 1 and cover.max() == 1
    # every block pairs two clusters of one level; dense blocks sit on the leaf level
    lev = lambda x: np.floor(np.log2(x)).astype(int)
    assert np.array_equal(lev(t), lvl) and np.array_equal(lev(s), lvl)
    assert np.all(lev(dt) == h.depth) and np.all(lev(ds) == h.depth)


@pytest.mark.parametrize("name,eta", [("grid64", 0.9), ("cloud3d", 0.7)])
def test_blocks_follow_admissibility(name, eta):
    """Coupling leaves are admissible, dense leaves are not, and every block's parent pair
    was inadmissible (it had to be refined) -- Sec. 6.1 condition, dual traversal."""
    pts = POINT_SETS[name]()
    h = _build(pts, eta=eta)
    bmin, bmax = h.boxes()
    lvl, t, s, dt, ds = h.blocks()
    adm = lambda a, b: oracle.admissible(bmin[a], bmax[a], bmin[b], bmax[b], eta)
    for a, b in zip(t, s):
        assert adm(a, b)
        if a > 1:
            assert not adm(a // 2, b // 2)
    for a, b in zip(dt, ds):
        assert not adm(a, b)
        if a > 1:
            assert not adm(a // 2, b // 2)


def test_block_structure_symmetric():
    h = _build(si.grid_2d(64))
    lvl, t, s, dt, ds = h.blocks()
    assert set(zip(t.tolist(), s.tolist())) == set(zip(s.tolist(), t.tolist()))
    assert set(zip(dt.tolist(), ds.tolist())) == set(zip(ds.tolist(), dt.tolist()))


def test_sparsity_constant_matches_paper():
    """Sec. 6.1 prints C_sp = 17 for the 2D grid set with m = 64, eta = 0.9."""
    w = si.GRID64_EXP
    h = oracle.OracleH2(w.make_points(), w.kernel, w.leaf_size, w.cheb_order, w.eta)
    lvl, t, s, dt, ds = h.blocks()
    per_row = collections.Counter(zip(lvl.tolist(), t.tolist()))
    assert max(per_row.values()) == GOLDEN["sparsity_constant_2d"]["value"]
    assert w.leaf_size == GOLDEN["leaf_size"]["value"]


@pytest.mark.parametrize("dim,p,key", [(2, 6, "rank_2d_6x6"), (3, 4, "rank_3d_tricubic")])
def test_rank_is_tensor_grid_size(dim, p, key):
    """Sec. 6.3: a 6x6 grid gives rank 36; tri-cubic interpolation gives rank 64."""
    h = _build(si.uniform_cloud(300, dim, 2), p=p)
    assert h.rank == GOLDEN[key]["value"]
    assert h.leaf_basis(2 ** h.depth).shape[1] == GOLDEN[key]["value"]


def test_tiny_problem_is_a_single_dense_leaf():
    h = _build(POINT_SETS["tiny"]())
    lvl, t, s, dt, ds = h.blocks()
    assert h.depth == 0 and len(t) == 0 and list(dt) == [1] and list(ds) == [1]


def test_no_admissible_blocks_for_tiny_eta():
    h = _build(si.grid_2d(37), eta=1e-9)
    lvl, t, s, dt, ds = h.blocks()
    assert len(t) == 0 and len(dt) == (2 ** h.depth) ** 2
