"""Algebraic recompression of the oracle's H^2 operator (Sec. 5) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this module. FP64 numpy; LAPACK's QR and SVD (``numpy.linalg``) serve as steps, with
no blocking, fusion or reordering. The steps follow Sec. 5 in the paper's order:

  1. Orthogonalization of the basis tree (the pre-processing step at the end of Sec. 5): an
     upsweep of QR factorizations, first of every leaf basis U_t = Q_t R_t, then of every
     sibling pair's reweighted transfers [R_c1 E_c1; R_c2 E_c2] = Q R_t, whose two row
     blocks are the new orthogonal transfers. Every coupling block is re-expressed in the
     orthogonal bases, S_ts <- R_t S_ts R_s^T.
  2. The downsweep for a new basis (Sec. 5.1, Eq. for B_i^q): from the root down, the R factor
     of the QR factorization of the stack [R_{i+} E_i^T; S_{i j1}^T; ...; S_{i jb}^T] -- the
     parent's factor times the transposed transfer first, then the transposed blocks of the
     node's block row in ascending column order.
  3. The truncation upsweep (Sec. 5.2): at a leaf the SVD of the reweighted basis Q_t R_t^T;
     at a parent the SVD of [T_c1 E_c1; T_c2 E_c2] R_t^T. The left singular vectors whose
     singular values pass the cut are the new leaf basis or the two new transfers (its row
     blocks); T_t = U'_t^T Q_t at a leaf and T_t = sum_c E'_c^T T_c E_c at a parent.
  4. Projection (end of Sec. 5): S'_ts = T_t S_ts T_s^T, the block projected on the new
     orthogonal bases (T_t = U'_t^T U_t is the projection of the old basis on the new one).

Readings where the paper leaves a choice open:
  * the threshold is relative to each node: of the reweighted basis of node t, the singular
    values sigma_i > tau * sigma_1(t) are kept, so every block row keeps relative accuracy
    tau in the 2-norm (an absolute cut tau * ||A_lr||_F, with A_lr the low-rank part, drops
    far more as N grows: at N = 2^20 on the 2D set it left a 7 % product error at tau = 1e-3);
    ||A_lr||_F itself is kept as a check, ||A_lr||_F^2 = sum over leaves of ||R_t||_F^2 (a
    leaf's stack holds its whole low-rank block row in orthonormal coordinates);
  * ranks are uniform per level: a level keeps the largest count over its nodes, and nodes
    with fewer singular values above the cut keep their next singular vectors too;
  * a leaf with fewer points than the rank, or a stack with fewer rows than columns, gets
    zero columns in Q (and zero rows in R) so that every factor keeps the k x k shape.

Parity status: pinned by ``tests/test_oracle_compress.py`` -- the orthogonalized operator
equals the original and its bases are orthonormal; the downsweep factors reproduce the Gram
matrix of each node's explicit block row (assembled densely, independent of the QR path);
tau = 0 reproduces the operator; polynomial kernels compress to their exact separation rank;
the leaves' truncation residuals stay under tau times their largest singular value; the
compression error stays under the bound of the dropped singular values and falls with tau.
"""
from __future__ import annotations

import numpy as np


def _pad_cols(M: np.ndarray, cols: int) -> np.ndarray:
    if M.shape[1] >= cols:
        return M[:, :cols]
    return np.hstack([M, np.zeros((M.shape[0], cols - M.shape[1]))])


def _pad_rows(M: np.ndarray, rows: int) -> np.ndarray:
    if M.shape[0] >= rows:
        return M[:rows]
    return np.vstack([M, np.zeros((rows - M.shape[0], M.shape[1]))])


def _qr(M: np.ndarray, k: int):
    """Q (rows x k, orthonormal columns then zero columns) and R (k x k) with M = Q R."""
    Q, R = np.linalg.qr(M, mode="reduced")
    return _pad_cols(Q, k), _pad_rows(R, k)


def _qr_r(M: np.ndarray, k: int) -> np.ndarray:
    return _pad_rows(np.linalg.qr(M, mode="r"), k)


def _svd_left(M: np.ndarray):
    """Left singular vectors and singular values (descending) of M."""
    if M.shape[0] == 0 or M.shape[1] == 0:
        return np.zeros((M.shape[0], 0)), np.zeros(0)
    W, s, _ = np.linalg.svd(M, full_matrices=False)
    return W, s


class CompressedH2:
    """The oracle operator after Sec. 5's compression with relative tolerance tau.

    Attributes: ``ranks[l]`` per level; ``U[leaf]`` (points x ranks[q]); ``E[c]``
    (ranks[l] x ranks[l-1]) for every non-root node c at level l; ``S[b]`` (ranks[l] x
    ranks[l]) for coupling block b of ``orc.blocks()`` order; the intermediate factors
    ``R`` (orthogonalization), ``Rh`` (downsweep), ``T`` (truncation); ``norm_lr``;
    ``sigma[t]`` and ``dropped[t]``, node t's singular values and those it does not keep.
    """

    def __init__(self, orc, tau: float):
        self.orc = orc
        self.tau = float(tau)
        q, nn, k = orc.depth, orc.nnodes, orc.rank
        self.q, self.nnodes, self.k = q, nn, k
        self.lo, self.hi = orc.ranges()
        self.perm = orc.perm
        lvl, bt, bs, dt, ds = orc.blocks()
        self.blk_level, self.blk_t, self.blk_s = lvl, bt, bs
        self.dns_t, self.dns_s = dt, ds
        first = 1 << q
        self.first = first
        rows = {}
        for b in range(len(bt)):
            rows.setdefault(int(bt[b]), []).append(b)
        self.rows = {t: sorted(bl, key=lambda b: int(bs[b])) for t, bl in rows.items()}
        self._orthogonalize()
        self._downsweep()
        self._truncate()
        self._project()

    # ---- 1. orthogonal basis tree
    def _orthogonalize(self):
        orc, q, k, first = self.orc, self.q, self.k, self.first
        self.Q, self.R, self.E1 = {}, {}, {}
        for t in range(first, self.nnodes + 1):
            self.Q[t], self.R[t] = _qr(orc.leaf_basis(t), k)
        for l in range(q, 0, -1):
            for t in range(1 << (l - 1), 1 << l):
                c1, c2 = 2 * t, 2 * t + 1
                Z = np.vstack([self.R[c1] @ orc.transfer(c1), self.R[c2] @ orc.transfer(c2)])
                Qz, self.R[t] = _qr(Z, k)
                self.E1[c1], self.E1[c2] = Qz[:k], Qz[k:]
        self.S1 = [self.R[int(t)] @ orc.coupling(int(t), int(s)) @ self.R[int(s)].T
                   for t, s in zip(self.blk_t, self.blk_s)]

    # ---- 2. downsweep: R factors of the stacked block rows
    def _downsweep(self):
        k = self.k
        self.Rh = {}
        for t in range(1, self.nnodes + 1):  # heap order visits every parent before its children
            parts = []
            if t > 1:
                parts.append(self.Rh[t // 2] @ self.E1[t].T)
            for b in self.rows.get(t, []):
                parts.append(self.S1[b].T)
            self.Rh[t] = _qr_r(np.vstack(parts), k) if parts else np.zeros((k, k))
        self.norm_lr = float(np.sqrt(sum(np.sum(self.Rh[t] ** 2) for t in range(self.first, self.nnodes + 1))))

    def kept(self, s: np.ndarray) -> int:
        """Singular values (descending) of a node that pass the cut tau * sigma_1."""
        return int(np.sum(s > self.tau * s[0])) if len(s) and s[0] > 0 else 0

    # ---- 3. truncation upsweep
    def _truncate(self):
        q, first, nn = self.q, self.first, self.nnodes
        self.ranks = [0] * (q + 1)
        self.U, self.E, self.T, self.dropped, self.sigma = {}, {}, {}, {}, {}
        W = {}
        for t in range(first, nn + 1):
            W[t], self.sigma[t] = _svd_left(self.Q[t] @ self.Rh[t].T)
        self.ranks[q] = max(self.kept(self.sigma[t]) for t in range(first, nn + 1))
        for t in range(first, nn + 1):
            self.U[t] = _pad_cols(W[t], self.ranks[q])
            self.T[t] = self.U[t].T @ self.Q[t]
            self.dropped[t] = self.sigma[t][self.ranks[q]:]
        for l in range(q, 0, -1):
            r = self.ranks[l]
            Z, W = {}, {}
            for t in range(1 << (l - 1), 1 << l):
                c1, c2 = 2 * t, 2 * t + 1
                Z[t] = np.vstack([self.T[c1] @ self.E1[c1], self.T[c2] @ self.E1[c2]])
                W[t], self.sigma[t] = _svd_left(Z[t] @ self.Rh[t].T)
            rp = max(self.kept(self.sigma[t]) for t in Z)
            self.ranks[l - 1] = rp
            for t in Z:
                Wt = _pad_cols(W[t], rp)
                self.E[2 * t], self.E[2 * t + 1] = Wt[:r], Wt[r:]
                self.T[t] = Wt.T @ Z[t]
                self.dropped[t] = self.sigma[t][rp:]

    # ---- 4. projection of the coupling blocks
    def _project(self):
        self.S = [self.T[int(t)] @ self.S1[b] @ self.T[int(s)].T
                  for b, (t, s) in enumerate(zip(self.blk_t, self.blk_s))]

    # ---- the compressed operator
    def matvec(self, X) -> np.ndarray:
        """A' X with A' the compressed operator (dense blocks unchanged), X (n, nv) user order."""
        X = np.asarray(X, dtype=np.float64).reshape(self.orc.n, -1)
        nv = X.shape[1]
        q, first, nn, lo, hi = self.q, self.first, self.nnodes, self.lo, self.hi
        Xt = X[self.perm]
        xh = {t: self.U[t].T @ Xt[lo[t]:hi[t]] for t in range(first, nn + 1)}
        for l in range(q, 0, -1):
            for t in range(1 << (l - 1), 1 << l):
                xh[t] = self.E[2 * t].T @ xh[2 * t] + self.E[2 * t + 1].T @ xh[2 * t + 1]
        level = lambda t: int(t).bit_length() - 1
        yh = {t: np.zeros((self.ranks[level(t)], nv)) for t in range(1, nn + 1)}
        for b, (t, s) in enumerate(zip(self.blk_t, self.blk_s)):
            yh[int(t)] += self.S[b] @ xh[int(s)]
        for t in range(2, nn + 1):
            yh[t] += self.E[t] @ yh[t // 2]
        y = np.zeros((self.orc.n, nv))
        for t in range(first, nn + 1):
            y[lo[t]:hi[t]] += self.U[t] @ yh[t]
        for t, s in zip(self.dns_t, self.dns_s):
            y[lo[t]:hi[t]] += self.orc.dense_block(int(t), int(s)) @ Xt[lo[s]:hi[s]]
        Y = np.empty_like(y)
        Y[self.perm] = y
        return Y

    def nested_basis(self, t: int, orthogonal_only: bool = False) -> np.ndarray:
        """Explicit basis of node t (tree-order rows lo..hi): the compressed one, or the
        orthogonalized one of step 1 (rank k)."""
        first = self.first
        if t >= first:
            return self.Q[t] if orthogonal_only else self.U[t]
        E = self.E1 if orthogonal_only else self.E
        B1 = self.nested_basis(2 * t, orthogonal_only) @ E[2 * t]
        B2 = self.nested_basis(2 * t + 1, orthogonal_only) @ E[2 * t + 1]
        return np.vstack([B1, B2])

    def assemble_lowrank(self, which: str = "compressed") -> np.ndarray:
        """The low-rank part in tree order, explicit (small n only): 'compressed' (A'),
        'orthogonal' (step 1's representation of A)."""
        n = self.orc.n
        A = np.zeros((n, n))
        ortho = which == "orthogonal"
        basis = {}
        for b, (t, s) in enumerate(zip(self.blk_t, self.blk_s)):
            t, s = int(t), int(s)
            for c in (t, s):
                if c not in basis:
                    basis[c] = self.nested_basis(c, ortho)
            blk = self.S1[b] if ortho else self.S[b]
            A[self.lo[t]:self.hi[t], self.lo[s]:self.hi[s]] = basis[t] @ blk @ basis[s].T
        return A

    def lowrank_bytes(self) -> tuple:
        """FP64 bytes of bases, transfers and coupling blocks: (before, after)."""
        k, n = self.k, self.orc.n
        nb = len(self.blk_t)
        before = 8 * (n * k + (self.nnodes - 1) * k * k + nb * k * k)
        lv = lambda t: int(t).bit_length() - 1
        after = 8 * (n * self.ranks[self.q]
                     + sum(self.ranks[lv(c)] * self.ranks[lv(c) - 1] for c in range(2, self.nnodes + 1))
                     + sum(self.ranks[int(l)] ** 2 for l in self.blk_level))
        return before, after


def lowrank_part(orc) -> np.ndarray:
    """The oracle's low-rank part in tree order: its explicit H^2 matrix with the dense
    blocks removed (small n only)."""
    A = orc.assemble_dense()
    perm = orc.perm
    At = A[np.ix_(perm, perm)]
    lo, hi = orc.ranges()
    _, _, _, dt, ds = orc.blocks()
    for t, s in zip(dt, ds):
        At[lo[t]:hi[t], lo[s]:hi[s]] = 0.0
    return At
