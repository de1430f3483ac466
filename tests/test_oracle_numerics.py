"""Pins of the oracle's Chebyshev bases, transfers and matvec against mathematics.

None of these compares the oracle with a retyped copy of itself. The references are:
numpy's first-kind Chebyshev points; Lagrange cardinality and polynomial reproduction
(checked with numpy's polynomial evaluation); the nested-basis identity of Sec. 2.1;
exact reproduction of polynomial kernels of degree < p by tensor interpolation;
brute-force dense K x; the special cases where the H^2 form is all dense; and the
algebraic properties of A_H2 (symmetry, linearity, alpha/beta semantics).
"""
import numpy as np
import pytest

import oracle
import synthetic_inputs as si


def relerr(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


# ----------------------------------------------------------------- Chebyshev points

@pytest.mark.parametrize("p", range(1, 11))
def test_cheb_points_are_numpy_first_kind(p):
    ref = np.polynomial.chebyshev.chebpts1(p)
    got = oracle.cheb_points(-1.0, 1.0, p)
    assert np.allclose(np.sort(got), ref, atol=1e-15, rtol=0)
    lo, hi = 0.25, 1.75
    assert np.allclose(np.sort(oracle.cheb_points(lo, hi, p)), lo + (ref + 1) * (hi - lo) / 2, atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 4, 6, 8])
def test_lagrange_cardinal_and_reproduces_polynomials(p):
    xi = oracle.cheb_points(-0.3, 1.1, p)
    for i in range(p):
        for j in range(p):
            assert abs(oracle.lagrange(xi, j, xi[i]) - (1.0 if i == j else 0.0)) < 1e-14
    rng = np.random.default_rng(p)
    coef = rng.standard_normal(p)  # degree p - 1
    for x in np.linspace(-0.3, 1.1, 23):
        interp = sum(oracle.lagrange(xi, j, x) * np.polyval(coef, xi[j]) for j in range(p))
        assert abs(interp - np.polyval(coef, x)) < 1e-12 * (1 + abs(np.polyval(coef, x)))


def test_leaf_basis_partition_of_unity():
    w = si.GRID64_EXP
    h = oracle.OracleH2(w.make_points(), w.kernel, w.leaf_size, w.cheb_order, w.eta)
    for t in (2 ** h.depth, 2 ** h.depth + 17, h.nnodes):
        U = h.leaf_basis(t)
        assert np.allclose(U.sum(axis=1), 1.0, atol=1e-14)


# ------------------------------------------------------------ nested bases (Sec. 2.1)

@pytest.mark.parametrize("dim,p,n", [(2, 4, 4096), (2, 8, 2048), (3, 4, 3000), (1, 6, 900)])
def test_nested_basis_equals_direct_interpolation(dim, p, n):
    """U^{l-1} = diag(U^l_c)[E_c] reproduces the interpolation basis of the parent box
    exactly, because the children's bases reproduce polynomials of degree < p."""
    pts = si.grid_2d(64)[:n] if dim == 2 and n == 4096 else si.uniform_cloud(n, dim, 11)
    h = oracle.OracleH2(pts, ("exp", 0.1, 0, 0), 32, p, 0.9)
    for t in [1, 2, 3, 5, 2 ** (h.depth - 1), 2 ** h.depth - 1]:
        if t >= 2 ** h.depth:
            continue
        Un, Ud = h.nested_basis(t), h.direct_basis(t)
        assert np.max(np.abs(Un - Ud)) < 1e-11 * max(1.0, np.max(np.abs(Ud)))


# ----------------------------------------------------------------- whole operator

@pytest.mark.parametrize("dim,p,deg,n,m", [(2, 4, 3, 1500, 32), (3, 3, 2, 2000, 40), (1, 5, 4, 700, 16),
                                           (2, 8, 7, 3000, 64)])
def test_polynomial_kernel_reproduced_exactly(dim, p, deg, n, m):
    """kappa = prod_d (1 + x_d y_d)^deg with deg <= p-1 is interpolated exactly, so
    A_H2 = K up to rounding (bases, transfers, couplings, permutation all exercised)."""
    pts = si.uniform_cloud(n, dim, 5)
    ker = ("poly", 0.0, 0.0, deg)
    h = oracle.OracleH2(pts, ker, m, p, 0.7)
    lvl, t, s, dt, ds = h.blocks()
    assert len(t) > 0 and h.depth >= 3
    X = si.gaussian_vectors(n, 2, 3)
    assert relerr(h.matvec(X), oracle.dense_kx(pts, ker, X)) < 1e-12


def test_polynomial_kernel_of_too_high_degree_is_not_exact():
    """The exactness test has teeth: degree p is not reproduced."""
    pts = si.uniform_cloud(1500, 2, 5)
    ker = ("poly", 0.0, 0.0, 4)
    h = oracle.OracleH2(pts, ker, 32, 4, 0.7)
    X = si.gaussian_vectors(1500, 1, 3)
    assert relerr(h.matvec(X), oracle.dense_kx(pts, ker, X)) > 1e-9


@pytest.mark.parametrize("n,eta", [(50, 0.9), (1369, 1e-9)])
def test_all_dense_special_cases_equal_brute_force(n, eta):
    """n <= m (one leaf) or eta -> 0 (nothing admissible): A_H2 is K itself."""
    pts = si.grid_2d(37)[:n] if n > 64 else si.uniform_cloud(n, 2, 9)
    ker = ("exp", 0.1, 0, 0)
    h = oracle.OracleH2(pts, ker, 64, 4, eta)
    lvl, t, s, dt, ds = h.blocks()
    assert len(t) == 0
    X = si.gaussian_vectors(n, 3, 4)
    assert relerr(h.matvec(X), oracle.dense_kx(pts, ker, X)) < 1e-14


def test_grid64_error_against_brute_force():
    """Sec. 6.1 accuracy metric |Ax - A_H2 x| / |Ax| (uniform random x, all rows here).
    With the 4x4 Chebyshev grid the interpolation error is a few 1e-3."""
    w = si.GRID64_EXP
    pts = w.make_points()
    h = oracle.OracleH2(pts, w.kernel, w.leaf_size, w.cheb_order, w.eta)
    x = si.uniform_vectors(h.n, 1, 2)
    assert relerr(h.matvec(x), oracle.dense_kx(pts, w.kernel, x)) < 5e-3


def test_error_decreases_geometrically_with_order():
    """Interpolation error falls geometrically with the Chebyshev order p (parity of the
    absolute constant is unpinned: the paper gives no closed-form bound)."""
    pts = si.grid_2d(64)
    ker = ("exp", 0.1, 0, 0)
    x = si.uniform_vectors(len(pts), 1, 2)
    ref = oracle.dense_kx(pts, ker, x)
    errs = [relerr(oracle.OracleH2(pts, ker, 64, p, 0.9).matvec(x), ref) for p in (2, 4, 6, 8)]
    for a, b in zip(errs, errs[1:]):
        assert b < a / 5
    assert errs[-1] < 1e-4


def test_explicit_assembly_matches_tree_product():
    w = si.GRID64_EXP
    h = oracle.OracleH2(w.make_points(), w.kernel, w.leaf_size, w.cheb_order, w.eta, assemble=True)
    A = h.assemble_dense()
    X = si.gaussian_vectors(h.n, 2, 1)
    assert relerr(A @ X, h.matvec(X)) < 1e-13
    assert np.max(np.abs(A - A.T)) < 1e-13 * np.max(np.abs(A))


def test_symmetry_linearity_and_columns():
    pts = si.uniform_cloud(2500, 3, 8)
    h = oracle.OracleH2(pts, ("exp", 0.2, 0, 0), 32, 3, 0.7)
    X = si.gaussian_vectors(h.n, 3, 6)
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    Ax, Ay = h.matvec(x)[:, 0], h.matvec(y)[:, 0]
    assert abs(y @ Ax - x @ Ay) < 1e-13 * np.linalg.norm(Ax) * np.linalg.norm(y)
    assert relerr(h.matvec(2.5 * x - 0.5 * z)[:, 0], 2.5 * Ax - 0.5 * h.matvec(z)[:, 0]) < 1e-14
    AX = h.matvec(X)
    assert relerr(AX[:, 0], Ax) < 1e-15 and relerr(AX[:, 1], Ay) < 1e-15


def test_alpha_beta_semantics():
    w = si.GRID64_EXP
    h = oracle.OracleH2(w.make_points(), w.kernel, w.leaf_size, w.cheb_order, w.eta)
    X = si.gaussian_vectors(h.n, 2, 1)
    Y0 = si.gaussian_vectors(h.n, 2, 2)
    AX = h.matvec(X)
    assert relerr(h.matvec(X, 0.75, -1.25, Y0), 0.75 * AX - 1.25 * Y0) < 1e-15
    nan = np.full((h.n, 2), np.nan, order="F")
    out = h.matvec(X, 2.0, 0.0, nan)
    assert np.all(np.isfinite(out)) and relerr(out, 2.0 * AX) < 1e-15


def test_sampled_leaves_match_full_product():
    pts = si.uniform_cloud(3001, 3, 7)
    h = oracle.OracleH2(pts, ("exp", 0.2, 0, 0), 32, 3, 0.7)
    X = si.gaussian_vectors(h.n, 2, 1)
    Y0 = si.gaussian_vectors(h.n, 2, 2)
    full = h.matvec(X, 1.5, 0.5, Y0)
    leaves = np.array([2 ** h.depth, 2 ** h.depth + 37, h.nnodes])
    rows, vals = h.matvec_leaves(X, leaves, 1.5, 0.5, Y0)
    assert relerr(vals, full[rows]) < 1e-15


def test_collinear_points_use_clamped_boxes():
    """Points on a horizontal line: the y-extent of every box is 0 and is clamped for the
    Chebyshev points; polynomial kernels are still reproduced exactly."""
    n = 600
    pts = np.stack([np.linspace(0, 1, n), np.full(n, 0.5)], axis=1)
    ker = ("poly", 0, 0, 3)
    h = oracle.OracleH2(pts, ker, 16, 4, 0.8)
    X = si.gaussian_vectors(n, 1, 1)
    assert relerr(h.matvec(X), oracle.dense_kx(pts, ker, X)) < 1e-11


@pytest.mark.parametrize("ker,x,y,expect", [
    (("exp", 0.1, 0, 0), [0.0, 0.0], [0.06, 0.08], np.exp(-1.0)),       # r = 0.1 = a
    (("gauss", 0.01, 0, 0), [0.0, 0.0], [0.06, 0.08], np.exp(-1.0)),    # r^2 = 0.01 = a
    (("imq", 1e-4, 1.5, 0), [0.0, 0.0], [0.0, 0.0], 1e6),               # (0 + 1e-4)^(-1.5)
    (("poly", 0, 0, 2), [2.0, 3.0], [0.5, 1.0], 16.0),                  # (1+1)^2 (1+3)^2 / 4
])
def test_kernel_definitions(ker, x, y, expect):
    if ker[0] == "poly":
        expect = (1 + 2.0 * 0.5) ** 2 * (1 + 3.0 * 1.0) ** 2
    assert abs(oracle.kernel_value(ker, x, y) - expect) < 1e-13 * abs(expect)
