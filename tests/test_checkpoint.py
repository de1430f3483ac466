"""Checkpoint of the host operator (h2_save / h2_load): a loaded operator is the built one
exactly -- same parameters, tree, partition, bases and transfers bit for bit -- and a damaged
or foreign file is refused on the host before anything reaches a device."""
import numpy as np
import pytest

import paper_2109_05451_gb300 as h2
import synthetic_inputs as si

CASES = {
    "grid37_gauss_k25": lambda: (si.grid_2d(37), ("gauss", 0.01, 0, 0), 32, 5, 0.7),
    "cloud3d_ragged": lambda: (si.uniform_cloud(3001, 3, 5), ("exp", 0.2, 0, 0), 40, 3, 0.7),
    "cloud1d_imq": lambda: (si.uniform_cloud(999, 1, 4), ("imq", 1e-4, 1.5, 0), 16, 6, 1.0),
    "tiny_single_leaf": lambda: (si.uniform_cloud(7, 2, 1), ("exp", 0.1, 0, 0), 64, 4, 0.9),
}

INFO_FIELDS = ["n", "dim", "depth", "rank", "leaf_size", "cheb_order", "eta", "n_nodes", "n_leaves", "n_coupling",
               "n_dense", "max_coupling_per_row", "max_dense_per_row", "coupling_entries", "dense_entries",
               "basis_entries", "transfer_entries"]


def snapshot(h):
    info = h2.h2_get_info(h)
    U, E = h2.h2_get_bases(h)
    return ({f: getattr(info, f) for f in INFO_FIELDS}, list(info.coupling_per_level), h2.h2_get_perm(h),
            h2.h2_get_coupling_csr(h), h2.h2_get_dense_csr(h), U, E)


def same(a, b):
    if isinstance(a, (tuple, list)):
        return len(a) == len(b) and all(same(x, y) for x, y in zip(a, b))
    if isinstance(a, np.ndarray):
        return a.dtype == b.dtype and a.shape == b.shape and a.tobytes() == b.tobytes()
    return a == b


@pytest.mark.parametrize("name", sorted(CASES))
def test_round_trip_is_bitwise(name, tmp_path):
    pts, ker, m, p, eta = CASES[name]()
    h = h2.h2_build(pts, ker, m, p, eta)
    path = str(tmp_path / "op.h2")
    try:
        h2.h2_save(h, path)
        g = h2.h2_load(path)
        try:
            assert same(snapshot(g), snapshot(h))
            # a loaded operator saves to the same bytes
            h2.h2_save(g, str(tmp_path / "again.h2"))
            assert (tmp_path / "again.h2").read_bytes() == (tmp_path / "op.h2").read_bytes()
        finally:
            h2.h2_destroy(g)
    finally:
        h2.h2_destroy(h)


@pytest.fixture(scope="module")
def saved(tmp_path_factory):
    pts, ker, m, p, eta = CASES["grid37_gauss_k25"]()
    h = h2.h2_build(pts, ker, m, p, eta)
    path = tmp_path_factory.mktemp("ckpt") / "op.h2"
    h2.h2_save(h, str(path))
    perm = h2.h2_get_perm(h)
    rowptr, col = h2.h2_get_coupling_csr(h)
    drowptr, dcol = h2.h2_get_dense_csr(h)
    h2.h2_destroy(h)
    return path.read_bytes(), perm, col, dcol


def refused(tmp_path, raw):
    path = tmp_path / "bad.h2"
    path.write_bytes(raw)
    with pytest.raises(h2.H2Error) as e:
        h2.h2_load(str(path))
    assert e.value.status == h2.H2_EINVAL


def patch(raw, old: np.ndarray, new: np.ndarray):
    at = raw.find(old.tobytes())
    assert at > 0 and len(old.tobytes()) == len(new.tobytes())
    return raw[:at] + new.tobytes() + raw[at + len(old.tobytes()):]


def test_truncated_and_foreign_files_are_refused(saved, tmp_path):
    raw = saved[0]
    for cut in (0, 5, 40, len(raw) // 2, len(raw) - 1):
        refused(tmp_path, raw[:cut])
    refused(tmp_path, b"XXXXXXXX" + raw[8:])
    refused(tmp_path, raw[:8] + np.uint32(99).tobytes() + raw[12:])
    with pytest.raises(h2.H2Error):
        h2.h2_load(str(tmp_path / "missing.h2"))


def test_damaged_indices_are_refused(saved, tmp_path):
    raw, perm, col, dcol = saved
    p2 = perm.copy()
    p2[0] = p2[1]                       # not a permutation
    refused(tmp_path, patch(raw, perm, p2))
    c2 = col.copy()
    c2[len(c2) // 2] = 0                # heap index 0 is not a cluster
    refused(tmp_path, patch(raw, col, c2))
    d2 = dcol.copy()
    d2[-1] = 1 << 20                    # leaf index past the last leaf
    refused(tmp_path, patch(raw, dcol, d2))


def test_bad_arguments():
    with pytest.raises(h2.H2Error):
        h2.h2_save(0, "x")
