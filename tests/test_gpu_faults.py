"""Failure detection, exercised without faulting the GPU.

* Device side: every wait of the pipelined kernels gives up after a cycle budget, records the
  failure in a device flag and returns. A self-test waits on a barrier nothing arrives on with
  a short budget, and two warps wait on node flags nothing sets (the small-rank warp sweeps'
  waits): the first gives up and raises the abort word, on which the second, with a fifty
  times longer budget, leaves. The call reports H2_ETIMEOUT and the context keeps working (a
  small-rank product, which runs those warp sweeps, still matches the oracle).
* Host side (the serving loop): a cancelled queued request, a cancelled running request, a
  right-hand side with a NaN, an argument error and a request too large for the slot memory;
  the loop survives all of them and still serves an ordinary request with the same result it
  gives alone.
"""
import time

import numpy as np
import pytest

import oracle
import synthetic_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2109_05451_gb300 as h2  # noqa: E402

SIGMA2 = 0.1


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    assert h2.load().h2_selftest_wait_timeout(2_000_000) == h2.H2_ETIMEOUT
    assert h2.load().h2_selftest_wait_timeout(0) == h2.H2_EINVAL
    assert h2.load().h2_selftest_wait_timeout(10 ** 9) == h2.H2_EINVAL
    pts = si.grid_2d(40)
    ker = ("exp", 0.1, 0, 0)
    orc = oracle.OracleH2(pts, ker, 32, 4, 0.9)
    op = h2.H2Operator(pts, ker, 32, 4, 0.9).upload("fp64")
    X = si.gaussian_vectors(len(pts), 1, 3)
    Y = op.matvec(torch.from_numpy(X[:, 0].copy()).cuda())
    torch.cuda.synchronize()
    ref = orc.matvec(X)[:, 0]
    assert np.linalg.norm(Y.cpu().numpy() - ref) / np.linalg.norm(ref) <= 1e-12
    op.close()


def test_serving_loop_survives_host_side_faults():
    pts = si.uniform_cloud(3000, 2, 3)
    ker = ("exp", 0.1, 0, 0)
    op = h2.H2Operator(pts, ker, 64, 6, 0.7).upload("fp32")
    big = h2.H2Operator(si.grid_2d(160), ker, 64, 6, 0.7).upload("fp64")
    n = op.n

    def rhs(seed):
        return si.gaussian_vectors(n, 1, seed)[:, 0].copy()

    alone = h2.H2Server(4 * h2.H2Server.request_bytes(op), 1, n)
    try:
        rid = alone.submit(op, rhs(5), 1e-5, 400, SIGMA2)
        alone.wait(120)
        (ref,) = alone.poll()
    finally:
        alone.close()
    assert ref["id"] == rid and ref["status"] == h2.H2_OK

    server = h2.H2Server(int(1.5 * h2.H2Server.request_bytes(op)), 1, 200 * 200)
    try:
        with pytest.raises(h2.H2Error) as e:  # can never fit the slot memory
            server.submit(big, si.gaussian_vectors(big.n, 1, 1)[:, 0].copy(), 1e-6, 10, SIGMA2)
        assert e.value.status == h2.H2_ENOMEM
        with pytest.raises(h2.H2Error) as e:  # argument error
            server.submit(op, rhs(1), 1e-6, -1, SIGMA2)
        assert e.value.status == h2.H2_EINVAL
        # tol 0 is never met (the recursive residual of CG keeps shrinking, so any positive
        # tolerance eventually stops it): it runs until cancelled
        long_id = server.submit(op, rhs(1), 0.0, 1_000_000, SIGMA2)
        queued_id = server.submit(op, rhs(2), 1e-6, 100, SIGMA2)       # waits behind it
        assert server.cancel(queued_id) == h2.H2_OK
        b_nan = rhs(3)
        b_nan[17] = np.nan
        nan_id = server.submit(op, b_nan, 1e-6, 50, SIGMA2)
        ok_id = server.submit(op, rhs(5), 1e-5, 400, SIGMA2)
        time.sleep(0.1)
        assert server.cancel(long_id) == h2.H2_OK
        assert server.wait(300) == h2.H2_OK
        res = {r["id"]: r for r in server.poll()}
        assert server.cancel(long_id) == h2.H2_EINVAL  # already completed
    finally:
        server.close()
        op.close()
        big.close()
    assert res[queued_id]["status"] == h2.H2_ECANCELED and res[queued_id]["iters"] == 0
    cancelled = res[long_id]
    assert cancelled["status"] == h2.H2_ECANCELED
    assert 0 < cancelled["iters"] < 1_000_000
    assert np.isfinite(cancelled["true_relres"]) and np.all(np.isfinite(cancelled["x"]))
    assert res[nan_id]["status"] == h2.H2_ENOTCONV and res[nan_id]["iters"] <= 1
    assert res[ok_id]["status"] == h2.H2_OK
    assert res[ok_id]["iters"] == ref["iters"] and np.array_equal(res[ok_id]["x"], ref["x"])
