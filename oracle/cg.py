"""Conjugate gradients for (A_H2 + sigma2 I) x = b -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` and the CPU-baseline leg of ``bench.py`` may import this module. The paper
solves its integral equation with a Krylov method whose operator products are H^2 matvecs
(Sec. 6.4, preconditioned CG on the fractional-diffusion system). The oracle takes the
plain, unpreconditioned method of Hestenes and Stiefel (1952) in FP64 with numpy inner
products, one step at a time in the textbook order:

    r_0 = b - A x_0,  p_0 = r_0
    alpha_j = (r_j . r_j) / (p_j . A p_j)
    x_{j+1} = x_j + alpha_j p_j,   r_{j+1} = r_j - alpha_j A p_j
    stop when ||r_{j+1}|| / ||b|| < tol (the recursively updated residual)
    beta_j = (r_{j+1} . r_{j+1}) / (r_j . r_j),   p_{j+1} = r_{j+1} + beta_j p_j

and reports the true residual ||b - A x|| / ||b|| recomputed with one more product. The
shifted operator is applied as ``apply(v) + sigma2 * v``; ``apply`` is any FP64 product
(the oracle's H^2 matvec in the parity tests). b = 0 gives x = 0 at once.

Pins (``tests/test_oracle_cg.py``): finite termination in exact-arithmetic counts (an
operator with j distinct eigenvalues converges in j steps), the solution of a dense SPD
system against LAPACK's direct solve, the A-norm error decreasing at every step, and the
Chebyshev bound on that error for a known condition number.
"""
from __future__ import annotations

import numpy as np


def cg_solve(apply, b, sigma2: float = 0.0, tol: float = 1e-6, maxit: int = 1000, x0=None):
    """Solve (A + sigma2 I) x = b by CG from x0 (zero by default).

    Returns a dict: ``x``, ``iters`` (products inside the loop), ``converged`` (the
    recursive residual met ``tol``), ``relres`` (recursive ||r||/||b|| after each step,
    the initial one first), ``true_relres`` (recomputed with one more product), and
    ``breakdown`` (a non-finite or non-positive curvature p.Ap, which an operator that
    is not positive definite can produce)."""
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64).reshape(-1)

    def op(v):
        return np.asarray(apply(v), dtype=np.float64).reshape(-1) + sigma2 * v

    bb = float(b @ b)
    if bb == 0.0:
        return {"x": np.zeros(n), "iters": 0, "converged": True, "relres": [0.0],
                "true_relres": 0.0, "breakdown": False}
    r = b - op(x)
    p = r.copy()
    rr = float(r @ r)
    history = [np.sqrt(rr / bb)]
    converged = history[0] < tol
    breakdown = False
    it = 0
    while not converged and it < maxit:
        Ap = op(p)
        pAp = float(p @ Ap)
        if not np.isfinite(pAp) or pAp <= 0.0:
            breakdown = True
            break
        alpha = rr / pAp
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = float(r @ r)
        it += 1
        history.append(np.sqrt(rr_new / bb))
        if history[-1] < tol:
            converged = True
            break
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
    true_res = b - op(x)
    return {"x": x, "iters": it, "converged": converged, "relres": history,
            "true_relres": float(np.sqrt((true_res @ true_res) / bb)), "breakdown": breakdown}
