"""CPU checks of libh2: every declared symbol is exported, argument validation, and the
host build (tree, partition, bases, transfers) agrees with the oracle.

The host build is plain host code (no CUDA call), so these run without a GPU. The tree
and the partition must agree exactly -- the same rules evaluated in the same FP64
operation order -- because the numeric parity on the GPU compares the same structure.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
import paper_2109_05451_gb300 as h2
import synthetic_inputs as si

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "h2.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(h2_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported():
    lib = C.CDLL(h2._build.build())
    names = declared_symbols()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) <= set(h2.SIGNATURES)


def test_status_strings():
    assert h2.h2_status_str(0) == "ok"
    assert "not converged" in h2.h2_status_str(1)


@pytest.mark.parametrize("bad", [
    dict(leaf_size=1), dict(cheb_order=0), dict(eta=-1.0), dict(cheb_order=9),  # 9^2 > 64
])
def test_build_rejects_bad_arguments(bad):
    args = dict(points=si.grid_2d(16), kernel=("exp", 0.1, 0, 0), leaf_size=16, cheb_order=4, eta=0.7)
    args.update(bad)
    with pytest.raises(h2.H2Error) as e:
        h2.h2_build(**args)
    assert e.value.status == h2.H2_EINVAL


def test_build_rejects_non_finite_points():
    pts = si.grid_2d(8)
    pts[3, 1] = np.nan
    with pytest.raises(h2.H2Error):
        h2.h2_build(pts, ("exp", 0.1, 0, 0), 16, 4, 0.7)


def test_device_calls_need_an_upload():
    h = h2.h2_build(si.grid_2d(16), ("exp", 0.1, 0, 0), 16, 4, 0.7)
    try:
        assert h2.h2_workspace_bytes(h, 1) == 0
        rc = h2.load().h2_matvec(h, 1, 1, 1, 1.0, 0.0, None)  # no device copy: refused before any CUDA call
        assert rc == h2.H2_ESTATE
    finally:
        h2.h2_destroy(h)


CASES = {
    "grid64_exp": lambda: (si.grid_2d(64), ("exp", 0.1, 0, 0), 64, 4, 0.9),
    "grid37_gauss": lambda: (si.grid_2d(37), ("gauss", 0.01, 0, 0), 32, 5, 0.7),
    "cloud3d": lambda: (si.uniform_cloud(5000, 3, 0), ("exp", 0.2, 0, 0), 64, 4, 0.7),
    "cloud1d": lambda: (si.uniform_cloud(999, 1, 4), ("imq", 1e-4, 1.5, 0), 16, 6, 1.0),
    "tiny": lambda: (si.uniform_cloud(7, 2, 1), ("exp", 0.1, 0, 0), 64, 4, 0.9),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_host_build_matches_oracle(name):
    pts, ker, m, p, eta = CASES[name]()
    orc = oracle.OracleH2(pts, ker, m, p, eta)
    h = h2.h2_build(pts, ker, m, p, eta)
    try:
        info = h2.h2_get_info(h)
        assert (info.depth, info.rank, info.n_nodes) == (orc.depth, orc.rank, orc.nnodes)
        assert np.array_equal(h2.h2_get_perm(h), orc.perm)
        lvl, t, s, dt, ds = orc.blocks()
        rowptr, col = h2.h2_get_coupling_csr(h)
        rows = np.repeat(np.arange(len(rowptr) - 1), np.diff(rowptr))
        got = sorted(zip(rows.tolist(), col.tolist()))
        assert got == sorted(zip(t.tolist(), s.tolist()))
        drowptr, dcol = h2.h2_get_dense_csr(h)
        first = 2 ** orc.depth
        drows = np.repeat(np.arange(len(drowptr) - 1), np.diff(drowptr)) + first
        assert sorted(zip(drows.tolist(), (dcol + first).tolist())) == sorted(zip(dt.tolist(), ds.tolist()))
        # CSR invariants: columns ascending within each row
        for r in range(len(rowptr) - 1):
            assert np.all(np.diff(col[rowptr[r]:rowptr[r + 1]]) > 0)
        assert info.n_coupling == len(t) and info.n_dense == len(dt)
        for l in range(orc.depth + 1):
            assert info.coupling_per_level[l] == np.sum(lvl == l)
        # bases and transfers to rounding
        U, E = h2.h2_get_bases(h)
        lo, hi = orc.ranges()
        for leaf in sorted({first, first + (first // 3), orc.nnodes}):
            assert np.allclose(U[lo[leaf]:hi[leaf]], orc.leaf_basis(leaf), rtol=0, atol=1e-13)
        for c in sorted({2, 3, orc.nnodes // 2, orc.nnodes} - {0, 1}):
            if c <= orc.nnodes and c >= 2:
                assert np.allclose(E[c], orc.transfer(c), rtol=0, atol=1e-13)
    finally:
        h2.h2_destroy(h)


def test_info_counts_for_grid64():
    """The 2D set of Sec. 6.1 (m = 64, eta = 0.9): C_sp = 17 reported through the ABI."""
    w = si.GRID64_EXP
    h = h2.h2_build(w.make_points(), w.kernel, w.leaf_size, w.cheb_order, w.eta)
    try:
        info = h2.h2_get_info(h)
        assert info.max_coupling_per_row == 17
        assert info.dense_entries == info.n_dense * 64 * 64
        assert info.basis_entries == 4096 * 16 and info.uploaded_prec == -1
    finally:
        h2.h2_destroy(h)


def test_server_calls_reject_bad_arguments_before_cuda():
    lib = h2.load()
    out = C.c_void_p()
    assert lib.h2_server_create(0, 2, 1000, C.byref(out)) == h2.H2_EINVAL
    assert lib.h2_server_create(1 << 20, 0, 1000, C.byref(out)) == h2.H2_EINVAL
    assert lib.h2_server_create(1 << 20, 2, 0, C.byref(out)) == h2.H2_EINVAL
    rid = C.c_int64(0)
    b = np.zeros(4)
    assert lib.h2_server_submit(None, None, 0.0, h2._np_ptr(b), h2._np_ptr(b), 1e-6, 10, C.byref(rid)) == h2.H2_EINVAL
    n = C.c_int(0)
    assert lib.h2_server_poll(None, None, 0, C.byref(n)) == h2.H2_EINVAL
    assert lib.h2_server_wait(None, 1.0) == h2.H2_EINVAL
    assert lib.h2_server_destroy(None) == h2.H2_EINVAL
    h = h2.h2_build(si.grid_2d(16), ("exp", 0.1, 0, 0), 16, 4, 0.7)
    try:
        assert lib.h2_server_request_bytes(h) == 0  # not uploaded
    finally:
        h2.h2_destroy(h)


def test_cancel_and_selftest_reject_bad_arguments_before_cuda():
    lib = h2.load()
    assert lib.h2_server_cancel(None, 1) == h2.H2_EINVAL
    assert lib.h2_selftest_wait_timeout(0) == h2.H2_EINVAL
    assert lib.h2_selftest_wait_timeout(10 ** 12) == h2.H2_EINVAL
    assert h2.h2_status_str(h2.H2_ECANCELED) == "cancelled"


def test_compress_rejects_bad_arguments_before_cuda():
    h = h2.h2_build(si.grid_2d(16), ("exp", 0.1, 0, 0), 16, 4, 0.7)
    try:
        assert h2.h2_get_level_ranks(h) == [16] * (h2.h2_get_info(h).depth + 1)
        for handle, tau in ((0, 1e-3), (h, -1.0), (h, float("nan")), (h, float("inf"))):
            with pytest.raises(h2.H2Error) as e:
                h2.h2_compress(handle, tau, stream=0)
            assert e.value.status == h2.H2_EINVAL
    finally:
        h2.h2_destroy(h)


FULL_SIZE = {
    # the nv = 1 product workload: 2^20-point Gaussian grid, rank 64, eta 0.7
    "grid1024_gauss": lambda: si.GRID1024_GAUSS,
    # the 32-vector workload: 2^21 uniform points in [0,1]^3, tri-cubic rank 64, eta 0.7
    "cloud3d_exp": lambda: si.CLOUD3D_EXP,
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(FULL_SIZE))
def test_full_size_partition_matches_oracle(name):
    """The benchmarked partitions, block by block: the host build's tree and coupling and
    dense lists equal the oracle's (Sec. 6.1 admissibility, same-level pairs), at full size.

    The counts are stated too, so that a change of either side's rule shows as a number:
    2^20 grid 483,456 coupling + 145,924 dense blocks; 2^21 cloud 4,721,738 + 1,948,838."""
    w = FULL_SIZE[name]()
    pts = w.make_points()
    orc = oracle.OracleH2(pts, w.kernel, w.leaf_size, w.cheb_order, w.eta)
    h = h2.h2_build(pts, w.kernel, w.leaf_size, w.cheb_order, w.eta)
    try:
        info = h2.h2_get_info(h)
        assert (info.depth, info.rank, info.n_nodes) == (orc.depth, orc.rank, orc.nnodes)
        assert np.array_equal(h2.h2_get_perm(h), orc.perm)
        lvl, t, s, dt, ds = orc.blocks()
        expect = {"grid1024_gauss": (483456, 145924), "cloud3d_exp": (4721738, 1948838)}[name]
        assert (len(t), len(dt)) == expect == (info.n_coupling, info.n_dense)
        for l in range(orc.depth + 1):
            assert info.coupling_per_level[l] == np.sum(lvl == l)
        rowptr, col = h2.h2_get_coupling_csr(h)
        rows = np.repeat(np.arange(len(rowptr) - 1, dtype=np.int64), np.diff(rowptr))
        o = np.lexsort((s, t))
        g = np.lexsort((col, rows))
        assert np.array_equal(rows[g], t[o]) and np.array_equal(col[g].astype(np.int64), s[o])
        drowptr, dcol = h2.h2_get_dense_csr(h)
        first = 2 ** orc.depth
        drows = np.repeat(np.arange(len(drowptr) - 1, dtype=np.int64), np.diff(drowptr)) + first
        dcol = dcol.astype(np.int64) + first
        o = np.lexsort((ds, dt))
        g = np.lexsort((dcol, drows))
        assert np.array_equal(drows[g], dt[o]) and np.array_equal(dcol[g], ds[o])
    finally:
        h2.h2_destroy(h)
