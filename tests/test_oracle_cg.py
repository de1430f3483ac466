"""Pins of the oracle's conjugate gradients (the Krylov solve of Sec. 6.4, unpreconditioned)
against properties that the method's mathematics fixes, not against a retyped copy of it:

* finite termination: on an SPD operator with j distinct eigenvalues CG reaches the exact
  solution in j steps (the Krylov space has dimension j);
* the solution of a dense SPD system equals LAPACK's direct solve within tol x cond;
* the A-norm of the error decreases at every step (CG minimises it over a growing space);
* the classical Chebyshev bound 2((sqrt(k)-1)/(sqrt(k)+1))^j on that error for condition k;
* the special cases b = 0 and a warm start at the solution, and breakdown on an
  indefinite operator.
"""
import numpy as np
import pytest

import oracle
import synthetic_inputs as si
from oracle.cg import cg_solve


def diag_op(d):
    return lambda v: d * v


@pytest.mark.parametrize("j", [1, 2, 3, 5, 8])
def test_finite_termination_in_distinct_eigenvalue_count(j):
    rng = np.random.default_rng(j)
    levels = np.linspace(1.0, 4.0, j)
    d = levels[rng.integers(0, j, 200)]
    d[:j] = levels  # every level present
    b = rng.standard_normal(200)
    res = cg_solve(diag_op(d), b, tol=1e-11, maxit=50)
    assert res["converged"] and res["iters"] == j
    assert np.allclose(res["x"], b / d, rtol=1e-10, atol=0)


def test_sigma_shift_is_applied():
    rng = np.random.default_rng(3)
    d = rng.uniform(1.0, 2.0, 64)
    b = rng.standard_normal(64)
    res = cg_solve(diag_op(d), b, sigma2=0.5, tol=1e-13, maxit=200)
    assert res["converged"] and np.allclose(res["x"], b / (d + 0.5), rtol=1e-11, atol=0)
    assert res["true_relres"] < 1e-12


def test_chebyshev_bound_and_monotone_energy_error():
    rng = np.random.default_rng(5)
    kappa = 400.0
    d = np.exp(rng.uniform(0.0, np.log(kappa), 300))
    d[0], d[1] = 1.0, kappa
    b = rng.standard_normal(300)
    xs = b / d

    errs = []
    for steps in range(0, 40):
        res = cg_solve(diag_op(d), b, tol=0.0, maxit=steps)
        e = res["x"] - xs
        errs.append(np.sqrt(e @ (d * e)))
    errs = np.array(errs)
    assert np.all(np.diff(errs) < 0)
    rho = (np.sqrt(kappa) - 1) / (np.sqrt(kappa) + 1)
    bound = 2 * rho ** np.arange(40) * errs[0]
    assert np.all(errs <= bound * (1 + 1e-12))


@pytest.fixture(scope="module")
def h2_system():
    w = si.GRID64_EXP  # 64 x 64 grid, exp(-r/0.1), leaf 64, rank 16, eta 0.9
    pts = w.make_points()
    orc = oracle.OracleH2(pts, w.kernel, w.leaf_size, w.cheb_order, w.eta)
    A = orc.assemble_dense()
    b = si.gaussian_vectors(len(pts), 1, 11)[:, 0]
    return orc, A, b


def test_h2_system_solution_matches_direct_solve(h2_system):
    orc, A, b = h2_system
    sigma2 = 0.1
    M = 0.5 * (A + A.T) + sigma2 * np.eye(len(b))
    ev = np.linalg.eigvalsh(M)
    assert ev[0] > 0  # the shifted H^2 operator of this set is SPD
    cond = ev[-1] / ev[0]
    xs = np.linalg.solve(M, b)
    tol = 1e-10
    res = cg_solve(lambda v: orc.matvec(v.reshape(-1, 1))[:, 0], b, sigma2=sigma2, tol=tol, maxit=5000)
    assert res["converged"] and not res["breakdown"]
    assert res["true_relres"] < 2 * tol
    assert np.linalg.norm(res["x"] - xs) / np.linalg.norm(xs) <= cond * tol
    # the recursive residual tracks the true one
    assert abs(res["relres"][-1] - res["true_relres"]) < 1e-10
    # A-norm error decreases along the iteration
    errs = []
    for steps in (0, 5, 10, 20, 40, 80):
        e = cg_solve(lambda v: M @ v, b, tol=0.0, maxit=steps)["x"] - xs
        errs.append(np.sqrt(e @ (M @ e)))
    assert np.all(np.diff(errs) < 0)


def test_zero_rhs_warm_start_and_breakdown():
    d = np.linspace(1.0, 3.0, 40)
    res = cg_solve(diag_op(d), np.zeros(40), tol=1e-8, maxit=10, x0=np.ones(40))
    assert res["converged"] and res["iters"] == 0 and np.all(res["x"] == 0.0)
    b = np.arange(1.0, 41.0)
    res = cg_solve(diag_op(d), b, tol=1e-8, maxit=10, x0=b / d)
    assert res["converged"] and res["iters"] == 0
    # an indefinite operator: the curvature p.Ap turns non-positive or CG fails to settle
    dn = np.concatenate([np.full(20, -1.0), np.full(20, 1.0)])
    res = cg_solve(diag_op(dn), np.concatenate([np.ones(20), np.zeros(20)]), tol=1e-8, maxit=10)
    assert res["breakdown"] and not res["converged"]
