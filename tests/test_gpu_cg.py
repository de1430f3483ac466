"""h2_cg_solve through the C ABI: CG on (A_H2 + sigma2 I) x = b (Sec. 6.4's Krylov solve,
unpreconditioned), checked with the oracle's FP64 product."""
import numpy as np
import pytest

import oracle
import synthetic_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2109_05451_gb300 as h2  # noqa: E402

SIGMA2 = 0.1


@pytest.fixture(scope="module")
def system():
    w = si.GRID64_EXP  # 64 x 64 grid, exp(-r/0.1), leaf 64, rank 16, eta 0.9
    pts = w.make_points()
    orc = oracle.OracleH2(pts, w.kernel, w.leaf_size, w.cheb_order, w.eta, assemble=True)
    op = h2.H2Operator(pts, w.kernel, w.leaf_size, w.cheb_order, w.eta)
    b = si.gaussian_vectors(len(pts), 1, 11)[:, 0]
    return orc, op, b


def oracle_relres(orc, x, b):
    r = b - (orc.matvec(x)[:, 0] + SIGMA2 * x)
    return float(np.linalg.norm(r) / np.linalg.norm(b))


def solve(op, b, tol, maxit, x0=None):
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd) if x0 is None else torch.from_numpy(x0).cuda()
    status, iters, relres = h2.h2_cg_solve(op.handle, SIGMA2, bd, xd, tol, maxit)
    torch.cuda.synchronize()
    return status, iters, relres, xd.cpu().numpy()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_cg_converges_to_the_oracle_system(system, prec, tol):
    orc, op, b = system
    op.upload(prec)
    status, iters, relres, x = solve(op, b, tol, 5000)
    assert status == h2.H2_OK and 0 < iters < 5000
    assert relres <= tol * 1.5  # true residual reported by the solver (one more product)
    # the same x against the oracle's FP64 operator: the GPU system is the oracle's system
    assert oracle_relres(orc, x, b) <= (5 * tol if prec == "fp64" else 5e-5)


def test_cg_reports_non_convergence(system):
    orc, op, b = system
    op.upload("fp64")
    status, iters, relres, x = solve(op, b, 1e-12, 3)
    assert status == h2.H2_ENOTCONV and iters == 3
    assert relres > 1e-12 and abs(relres - oracle_relres(orc, x, b)) < 1e-10


def test_cg_zero_rhs_and_warm_start(system):
    orc, op, b = system
    op.upload("fp64")
    status, iters, relres, x = solve(op, np.zeros_like(b), 1e-10, 100, x0=np.ones_like(b))
    assert status == h2.H2_OK and iters == 0 and np.all(x == 0.0)
    # warm start from a converged solution: converged at iteration 0
    _, _, _, xs = solve(op, b, 1e-10, 5000)
    status, iters, relres, _ = solve(op, b, 1e-8, 5000, x0=xs)
    assert status == h2.H2_OK and iters == 0 and relres < 1e-8


def test_cg_is_bitwise_repeatable(system):
    orc, op, b = system
    op.upload("fp32")
    r1 = solve(op, b, 1e-5, 5000)
    r2 = solve(op, b, 1e-5, 5000)
    assert r1[1] == r2[1] and np.array_equal(r1[3], r2[3])


def relerr(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def oracle_cg(orc, b, tol, maxit, sigma2=SIGMA2):
    from oracle.cg import cg_solve
    return cg_solve(lambda v: orc.matvec(v.reshape(-1, 1))[:, 0], b, sigma2=sigma2, tol=tol, maxit=maxit)


@pytest.mark.parametrize("steps", [1, 3, 10])
def test_cg_iterates_equal_the_oracle_cg(system, steps):
    """FP64 products: the j-th GPU iterate is the oracle CG's j-th iterate (the same
    Hestenes-Stiefel steps on the same operator), to rounding. Short runs only: CG loses
    orthogonality in finite precision, and a 2e-16 relative perturbation of each product
    already moves the 40th iterate of this system by 1e-5."""
    orc, op, b = system
    op.upload("fp64")
    ref = oracle_cg(orc, b, 0.0, steps)
    status, iters, relres, x = solve(op, b, 0.0, steps)
    assert status == h2.H2_ENOTCONV and iters == ref["iters"] == steps
    assert relerr(x, ref["x"]) <= 1e-12
    assert abs(relres - ref["true_relres"]) <= 1e-12 * max(1.0, ref["true_relres"]) + 1e-14


def test_cg_iteration_count_equals_the_oracle_cg(system):
    orc, op, b = system
    op.upload("fp64")
    ref = oracle_cg(orc, b, 1e-10, 5000)
    status, iters, relres, x = solve(op, b, 1e-10, 5000)
    assert ref["converged"] and status == h2.H2_OK
    # product rounding (GPU and oracle sum in different orders) delays or advances the step at
    # which the recursive residual crosses tol by a few steps out of ~235 here
    assert abs(iters - ref["iters"]) <= max(2, int(0.03 * ref["iters"]))
    assert relerr(x, ref["x"]) <= 1e-8
