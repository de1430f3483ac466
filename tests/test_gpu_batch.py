"""GPU tests of batched products of uneven operators (h2_batch_*): one persistent launch per
width class over every member's block rows, the members' sweeps on parallel graph branches,
the whole product captured as a CUDA graph and replayed.

Every member's result must match the oracle (1e-12 FP64, 1e-5 FP32 relative l2) and the
member's own h2_matvec; replays are bitwise repeatable and follow new contents of X and Y;
the autotuner writes its choice to the cache and a later batch reuses it.
"""
import os

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


def to_dev(X, prec):
    return torch.from_numpy(np.ascontiguousarray(np.asfortranarray(X).T)).to(device="cuda", dtype=DT[prec]).t()


def to_host(Y):
    return Y.t().contiguous().cpu().double().numpy().T


@pytest.fixture(scope="module")
def members():
    mem = si.uneven_batch(count=12, n_min=2 ** 10, n_max=2 ** 14, seed=4, nv_max=16)
    out = []
    for m in mem:
        orc = oracle.OracleH2(m.points, m.kernel, m.leaf_size, m.cheb_order, m.eta)
        op = h2.H2Operator(m.points, m.kernel, m.leaf_size, m.cheb_order, m.eta)
        out.append((m, orc, op))
    yield out
    for _, _, op in out:
        op.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_matches_oracle_and_single_products(members, prec):
    ops, Xs, Ys, refs, Xh = [], [], [], [], []
    for m, orc, op in members:
        op.upload(prec)
        X = m.make_x()
        ops.append(op)
        Xh.append(X)
        Xs.append(to_dev(X, prec))
        Ys.append(op.new_vectors(m.nv, fill=float("nan")))
        refs.append(orc.matvec(X))
    b = h2.H2Batch(ops, Xs, Ys)
    try:
        b.run()
        torch.cuda.synchronize()
        b.check()
        for (m, orc, op), Y, ref, X in zip(members, Ys, refs, Xh):
            got = to_host(Y)
            assert np.all(np.isfinite(got)), m.name
            assert relerr(got, ref) <= TOL[prec], m.name
            # the batch streams FP32 blocks on the CUDA cores: compare with the single product
            # on the same path (FP32 passes of more than 8 vectors otherwise take 3xTF32)
            h2.h2_set_fp32_tensor(op.handle, False)
            try:
                single = to_host(op.matvec(to_dev(X, prec)))
            finally:
                h2.h2_set_fp32_tensor(op.handle, True)
            assert relerr(got, single) <= (1e-14 if prec == "fp64" else 1e-6), m.name
        first = [to_host(Y).copy() for Y in Ys]
        b.run()
        torch.cuda.synchronize()
        assert all(np.array_equal(to_host(Y), f) for Y, f in zip(Ys, first))  # bitwise repeatable
        # the graph reads X at every replay: new contents, new result
        for X, (m, _, _) in zip(Xs, members):
            X.mul_(-2.0)
        b.run()
        torch.cuda.synchronize()
        for Y, ref in zip(Ys, refs):
            assert relerr(to_host(Y), -2.0 * ref) <= TOL[prec]
    finally:
        b.close()


def test_batch_alpha_beta(members):
    prec = "fp32"
    ops, Xs, Ys, want = [], [], [], []
    for m, orc, op in members[:6]:
        op.upload(prec)
        X = m.make_x()
        Y0 = si.gaussian_vectors(op.n, m.nv, 77)
        ops.append(op)
        Xs.append(to_dev(X, prec))
        Ys.append(to_dev(Y0, prec))
        want.append(orc.matvec(X, 0.5, -1.5, Y0))
    b = h2.H2Batch(ops, Xs, Ys, alpha=0.5, beta=-1.5)
    try:
        b.run()
        torch.cuda.synchronize()
        for Y, w in zip(Ys, want):
            assert relerr(to_host(Y), w) <= TOL[prec]
    finally:
        b.close()


def test_autotuner_writes_and_reuses_its_cache(members, tmp_path, monkeypatch):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("H2_TUNE_CACHE", str(cache))
    ops, Xs, Ys = [], [], []
    for m, orc, op in members:
        op.upload("fp32")
        ops.append(op)
        Xs.append(to_dev(m.make_x(), "fp32"))
        Ys.append(op.new_vectors(m.nv, fill=0.0))
    b = h2.H2Batch(ops, Xs, Ys, autotune=True)
    d1 = b.describe()
    b.run()
    torch.cuda.synchronize()
    y1 = [to_host(Y).copy() for Y in Ys]
    b.close()
    lines = cache.read_text().strip().splitlines()
    assert lines and all(len(l.split()) == 5 for l in lines)
    assert "(tuned)" in d1
    b2 = h2.H2Batch(ops, Xs, Ys)  # no tuning: the cached choice
    try:
        assert b2.describe().count("(tuned)") == d1.count("(tuned)")
        b2.run()
        torch.cuda.synchronize()
        for Y, y in zip(Ys, y1):
            assert relerr(to_host(Y), y) <= 1e-6
    finally:
        b2.close()
    assert cache.read_text().strip().splitlines() == lines  # nothing re-tuned


def test_batch_rejects_what_it_cannot_run(members):
    (m0, _, op0), (m1, _, op1) = members[0], members[1]
    op0.upload("fp64")
    op1.upload("fp32")
    X0 = to_dev(m0.make_x(), "fp64")
    Y0 = op0.new_vectors(m0.nv)
    X1 = to_dev(m1.make_x(), "fp32")
    Y1 = op1.new_vectors(m1.nv)
    with pytest.raises(h2.H2Error):  # mixed precisions
        h2.H2Batch([op0, op1], [X0, X1], [Y0, Y1])
    op1.upload("bf16x2")
    with pytest.raises(h2.H2Error):  # the tensor-core precision is not batched
        h2.H2Batch([op1], [X1], [op1.new_vectors(m1.nv)])
    op1.upload("fp32")
    Xw = to_dev(si.gaussian_vectors(op1.n, 40, 1), "fp32")
    with pytest.raises(h2.H2Error):  # more than one pass of vectors
        h2.H2Batch([op1], [Xw], [op1.new_vectors(40)])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_merged_sweeps_equal_member_sweeps(members, prec):
    """The merged sweep launches (one per step and width over a table of the members'
    subtrees) run each member's subtrees with the same arithmetic as its own launches: the
    batched results are bitwise equal, and a replay takes a few launches per width."""
    ops, Xs, Ys_a, Ys_b = [], [], [], []
    for m, orc, op in members:
        op.upload(prec)
        ops.append(op)
        Xs.append(to_dev(m.make_x(), prec))
        Ys_a.append(op.new_vectors(m.nv, fill=float("nan")))
        Ys_b.append(op.new_vectors(m.nv, fill=float("nan")))
    merged = h2.H2Batch(ops, Xs, Ys_a)
    own = h2.H2Batch(ops, Xs, Ys_b, member_sweeps=True)
    try:
        desc = merged.describe()
        assert "members with their own sweeps 0" in desc, desc
        assert "sweeps width" in desc and "sweeps width" not in own.describe()
        merged.run()
        own.run()
        torch.cuda.synchronize()
        merged.check()
        own.check()
        for (m, _, _), ya, yb in zip(members, Ys_a, Ys_b):
            assert np.array_equal(to_host(ya), to_host(yb)), m.name
    finally:
        merged.close()
        own.close()
