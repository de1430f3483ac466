"""FP64 CPU oracle for the H^2 matrix-vector product -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package. It is a ctypes shim over ``h2_oracle.c``, a plain C
implementation written from the paper (arXiv 2109.05451, Sec. 2.1, Sec. 3.1-3.3 with
Alg 1, Alg 4 and Alg 6, Sec. 6.1 and 6.3). It shares no code with the CUDA library.

Parity status of each function (see the pins in ``tests/test_oracle_*.py``):
  * tree, admissibility, partition: pinned (C_sp = 17 of Sec. 6.1, exact tiling of the
    index square, admissibility of every coupling leaf and inadmissibility of every
    refined pair, leaf-size and node-count invariants);
  * Chebyshev points / Lagrange basis: pinned (numpy's first-kind Chebyshev points,
    cardinality at the nodes, polynomial reproduction);
  * transfers: pinned (nested basis = direct interpolation, Sec. 2.1);
  * whole matvec: pinned (exact reproduction of polynomial kernels of degree < p,
    pure-dense special cases equal brute-force K x, interpolation error against
    brute force decreasing geometrically in p, explicit assembly, symmetry, linearity);
  * the absolute interpolation error constant: parity unpinned (the paper gives no
    closed-form bound for it).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "h2_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libh2oracle.so")

KERNELS = {"exp": 0, "gauss": 1, "imq": 2, "poly": 3}

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    P, I64, I, D = C.c_void_p, C.c_int64, C.c_int, C.c_double
    sig = {
        "orc_build": (P, [P, I64, I, I, D, D, I, I, I, D]),
        "orc_free": (None, [P]),
        "orc_assemble": (I, [P]),
        "orc_n": (I64, [P]),
        "orc_depth": (I, [P]),
        "orc_rank": (I, [P]),
        "orc_nnodes": (I64, [P]),
        "orc_ncoupling": (I64, [P]),
        "orc_ndense": (I64, [P]),
        "orc_get_perm": (None, [P, P]),
        "orc_get_ranges": (None, [P, P, P]),
        "orc_get_boxes": (None, [P, P, P]),
        "orc_get_blocks": (None, [P, P, P, P, P, P]),
        "orc_matvec": (I, [P, P, P, I, D, D]),
        "orc_matvec_leaves": (I, [P, P, I, D, D, P, P, I64, P]),
        "orc_leaf_basis": (None, [P, I64, P]),
        "orc_transfer": (None, [P, I64, P]),
        "orc_coupling": (None, [P, I64, I64, P]),
        "orc_dense_block": (None, [P, I64, I64, P]),
        "orc_nested_basis": (None, [P, I64, P]),
        "orc_direct_basis": (None, [P, I64, P]),
        "orc_assemble_h2_dense": (I, [P, P]),
        "orc_dense_kx": (None, [P, I64, I, I, D, D, I, P, I, P]),
        "orc_dense_kx_rows": (None, [P, I64, I, I, D, D, I, P, I, P, I64, P]),
        "orc_kernel_value": (D, [I, D, D, I, P, P, I]),
        "orc_cheb_points": (None, [D, D, I, P]),
        "orc_lagrange": (D, [P, I, I, D]),
        "orc_admissible_boxes": (I, [P, P, P, P, I, D]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _kernel_args(kernel):
    name, a, b, deg = kernel
    return KERNELS[name], float(a), float(b), int(deg)


class OracleH2:
    """The oracle's H^2 operator for one point set and kernel (FP64, host)."""

    def __init__(self, points, kernel, leaf_size: int, cheb_order: int, eta: float,
                 assemble: bool = False):
        lib = _load()
        pts = np.ascontiguousarray(points, dtype=np.float64)
        self.n, self.dim = pts.shape
        self.points = pts
        self.kernel = kernel
        kind, a, b, deg = _kernel_args(kernel)
        self._h = lib.orc_build(_ptr(pts), self.n, self.dim, kind, a, b, deg, int(leaf_size),
                                int(cheb_order), float(eta))
        if not self._h:
            raise ValueError("oracle build rejected its arguments")
        self.leaf_size, self.cheb_order, self.eta = int(leaf_size), int(cheb_order), float(eta)
        self.depth = lib.orc_depth(self._h)
        self.rank = lib.orc_rank(self._h)
        self.nnodes = lib.orc_nnodes(self._h)
        if assemble and lib.orc_assemble(self._h) != 0:
            raise MemoryError("oracle could not store the blocks")

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_free(self._h)
            self._h = None

    # ---- structure
    @property
    def perm(self) -> np.ndarray:
        out = np.empty(self.n, dtype=np.int64)
        _lib.orc_get_perm(self._h, _ptr(out))
        return out

    def ranges(self):
        lo = np.empty(self.nnodes + 1, dtype=np.int64)
        hi = np.empty(self.nnodes + 1, dtype=np.int64)
        _lib.orc_get_ranges(self._h, _ptr(lo), _ptr(hi))
        return lo, hi

    def boxes(self):
        bmin = np.empty((self.nnodes + 1, self.dim))
        bmax = np.empty((self.nnodes + 1, self.dim))
        _lib.orc_get_boxes(self._h, _ptr(bmin), _ptr(bmax))
        return bmin, bmax

    def blocks(self):
        """(levels, t, s) of the coupling blocks and (t, s) of the dense blocks, heap indices."""
        nc, nd = _lib.orc_ncoupling(self._h), _lib.orc_ndense(self._h)
        lvl = np.empty(nc, dtype=np.int32)
        t = np.empty(nc, dtype=np.int64)
        s = np.empty(nc, dtype=np.int64)
        dt = np.empty(nd, dtype=np.int64)
        ds = np.empty(nd, dtype=np.int64)
        _lib.orc_get_blocks(self._h, _ptr(lvl), _ptr(t), _ptr(s), _ptr(dt), _ptr(ds))
        return lvl, t, s, dt, ds

    # ---- pieces
    def leaf_basis(self, t: int) -> np.ndarray:
        lo, hi = self.ranges()
        out = np.empty((hi[t] - lo[t], self.rank))
        _lib.orc_leaf_basis(self._h, int(t), _ptr(out))
        return out

    def transfer(self, c: int) -> np.ndarray:
        out = np.empty((self.rank, self.rank))
        _lib.orc_transfer(self._h, int(c), _ptr(out))
        return out

    def coupling(self, t: int, s: int) -> np.ndarray:
        out = np.empty((self.rank, self.rank))
        _lib.orc_coupling(self._h, int(t), int(s), _ptr(out))
        return out

    def dense_block(self, t: int, s: int) -> np.ndarray:
        lo, hi = self.ranges()
        out = np.empty((hi[t] - lo[t], hi[s] - lo[s]))
        _lib.orc_dense_block(self._h, int(t), int(s), _ptr(out))
        return out

    def nested_basis(self, t: int) -> np.ndarray:
        lo, hi = self.ranges()
        out = np.empty((hi[t] - lo[t], self.rank))
        _lib.orc_nested_basis(self._h, int(t), _ptr(out))
        return out

    def direct_basis(self, t: int) -> np.ndarray:
        lo, hi = self.ranges()
        out = np.empty((hi[t] - lo[t], self.rank))
        _lib.orc_direct_basis(self._h, int(t), _ptr(out))
        return out

    def assemble_dense(self) -> np.ndarray:
        """A_H2 as an explicit n x n matrix (user order). Small n only."""
        A = np.empty((self.n, self.n))
        _lib.orc_assemble_h2_dense(self._h, _ptr(A))
        return A

    # ---- products
    def matvec(self, X, alpha: float = 1.0, beta: float = 0.0, Y=None) -> np.ndarray:
        """alpha * A_H2 X + beta * Y, X and Y (n, nv) in user order."""
        X = np.asfortranarray(np.asarray(X, dtype=np.float64).reshape(self.n, -1))
        nv = X.shape[1]
        out = np.zeros((self.n, nv), order="F") if Y is None else np.array(Y, dtype=np.float64, order="F", copy=True).reshape(self.n, nv, order="F")
        if _lib.orc_matvec(self._h, _ptr(X), _ptr(out), nv, float(alpha), float(beta)) != 0:
            raise MemoryError("oracle matvec failed")
        return out

    def matvec_leaves(self, X, leaves, alpha: float = 1.0, beta: float = 0.0, Y=None):
        """Output rows of the given leaves only: returns (user_rows, values (rows, nv))."""
        X = np.asfortranarray(np.asarray(X, dtype=np.float64).reshape(self.n, -1))
        nv = X.shape[1]
        leaves = np.ascontiguousarray(leaves, dtype=np.int64)
        lo, hi = self.ranges()
        first = 1 << self.depth
        if np.any(leaves < first) or np.any(leaves > self.nnodes):
            raise ValueError("not a leaf")
        nrows = int(np.sum(hi[leaves] - lo[leaves]))
        out = np.empty((nrows, nv))
        Yin = np.zeros((1, 1)) if Y is None else np.asfortranarray(np.asarray(Y, dtype=np.float64).reshape(self.n, nv))
        rc = _lib.orc_matvec_leaves(self._h, _ptr(X), nv, float(alpha), float(beta), _ptr(Yin),
                                    _ptr(leaves), len(leaves), _ptr(out))
        if rc != 0:
            raise MemoryError("oracle matvec_leaves failed")
        perm = self.perm
        rows = np.concatenate([perm[lo[t]:hi[t]] for t in leaves]) if len(leaves) else np.empty(0, np.int64)
        return rows, out


def dense_kx(points, kernel, X) -> np.ndarray:
    """Brute-force K X with K_ij = kappa(x_i, x_j); no H^2 structure."""
    lib = _load()
    pts = np.ascontiguousarray(points, dtype=np.float64)
    n, dim = pts.shape
    X = np.asfortranarray(np.asarray(X, dtype=np.float64).reshape(n, -1))
    Y = np.empty_like(X, order="F")
    kind, a, b, deg = _kernel_args(kernel)
    lib.orc_dense_kx(_ptr(pts), n, dim, kind, a, b, deg, _ptr(X), X.shape[1], _ptr(Y))
    return Y


def dense_kx_rows(points, kernel, X, rows) -> np.ndarray:
    """Rows of the brute-force K X, shape (len(rows), nv)."""
    lib = _load()
    pts = np.ascontiguousarray(points, dtype=np.float64)
    n, dim = pts.shape
    X = np.asfortranarray(np.asarray(X, dtype=np.float64).reshape(n, -1))
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.empty((len(rows), X.shape[1]))
    kind, a, b, deg = _kernel_args(kernel)
    lib.orc_dense_kx_rows(_ptr(pts), n, dim, kind, a, b, deg, _ptr(X), X.shape[1], _ptr(rows),
                          len(rows), _ptr(out))
    return out


def kernel_value(kernel, x, y) -> float:
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    kind, a, b, deg = _kernel_args(kernel)
    return lib.orc_kernel_value(kind, a, b, deg, _ptr(x), _ptr(y), len(x))


def cheb_points(lo: float, hi: float, p: int) -> np.ndarray:
    out = np.empty(p)
    _load().orc_cheb_points(float(lo), float(hi), int(p), _ptr(out))
    return out


def lagrange(xi, j: int, x: float) -> float:
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    return _load().orc_lagrange(_ptr(xi), len(xi), int(j), float(x))


def admissible(tmin, tmax, smin, smax, eta: float) -> bool:
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (tmin, tmax, smin, smax)]
    return bool(_load().orc_admissible_boxes(*[_ptr(a) for a in arrs], len(arrs[0]), float(eta)))
