"""Oracle-R: plain CPU fp64 recursive skeletonization factorization (RSF).

ORACLE -- test infrastructure only (tests, smoke check, benchmark CPU leg).

Follows Sec. 2 step by step, with no blocking or fusion:

* Sec. 2.1, Def. (ID): for each box with active DOFs I, an ID of Sigma(I^c, I)
  splits I into skeleton S and redundant R with interpolation matrix T,
  Sigma(I^c, R) ~ Sigma(I^c, S) T.  The ID is computed by column-pivoted QR
  (Sec. 2.3) and the rank is k = #{j : |R_jj| > eps |R_11|}.
* Sec. 2.3.1, Eq. (proxyid): the ID is taken of [Sigma(N, I); M(Gamma, I)],
  near rows plus proxy-annulus rows, instead of all of I^c.
* Sec. 2.1 block equations: L_I^-1 (row_R -= T^T row_S, col_R -= col_S T)
  gives X_SR = A_SR - A_SS T and X_RR = A_RR - T^T A_SR - A_RS T + T^T A_SS T;
  U_I with E = X_SR X_RR^-1 decouples R and leaves X_SS = A_SS - E X_RS.
* Sec. 2.2, Eq. (rskelf): leaf level first, then each level up with the
  children's skeletons as the parent's DOFs; the blocks between skeletons of
  distinct boxes stay the original kernel entries; the root block is factored
  densely, Sigma_1 = C C^T.
* Remark (indefinite): for a derivative matrix the diagonal blocks are factored
  by LU with partial pivoting instead of Cholesky (F_k is only applied).
* Sec. 2.3.2 (apply/solve): F = Q D Q^T with Q = prod_l prod_I L_I U_I and
  D = blockdiag(X_RR, root); F^-1 reverses the order; F^1/2 = Q C;
  log|F| = 2 log|C|.

Vectors are in *tree order* (see tree.Tree.perm); ``Factorization.solve`` etc.
accept (n,) or (n, q) arrays.
"""
from __future__ import annotations

import numpy as np
from scipy import linalg

from . import kernels as K
from .tree import Tree, proxy_points, DEFAULT_OPTS


class BoxRecord:
    __slots__ = ("box", "level", "I", "S", "R", "T", "E", "C", "XRR", "near",
                 "k", "rnorm")


def interpolative_decomposition(A, tol):
    """Column-pivoted QR ID of A (m x c): returns (perm, k, T) with
    A[:, perm[k:]] ~ A[:, perm[:k]] @ T (Def. ID, Sec. 2.3)."""
    m, c = A.shape
    if c == 0:
        return np.arange(0), 0, np.zeros((0, 0))
    if m == 0:
        return np.arange(c), 0, np.zeros((0, c))
    R, perm = linalg.qr(A, mode="r", pivoting=True)
    d = np.abs(np.diag(R))
    if d.size == 0 or d[0] == 0.0:
        return perm, 0, np.zeros((0, c))
    k = int(np.sum(d > tol * d[0]))
    T = linalg.solve_triangular(R[:k, :k], R[:k, k:], lower=False) if k > 0 else np.zeros((0, c))
    return perm, k, T


class Factorization:
    """RSF F ~ Sigma (which=0) or F_k ~ dSigma/dtheta_k (which>0)."""

    def __init__(self, x, family, theta, which=K.SIGMA, tol=1e-9, alpha=0.0,
                 opts=None, tree=None):
        self.opts = dict(DEFAULT_OPTS)
        if opts:
            self.opts.update(opts)
        o = self.opts
        self.tree = tree if tree is not None else Tree(x, o["n_occ"])
        t = self.tree
        self.family, self.theta, self.which, self.alpha = family, tuple(theta), which, alpha
        self.tol = tol
        self.spd = which == K.SIGMA
        self.n = t.n
        xt = t.xt
        self.records = {}          # level -> list of BoxRecord
        self.active = {}           # level -> active DOFs before that level
        skel = {}                  # box -> (S dofs, X_SS)
        for lev in range(t.L, 0, -1):
            boxes = t.boxes_at(lev)
            Iset = {}
            for b in boxes:
                if t.is_leaf[b]:
                    Iset[b] = t.dofs(b)
                else:
                    Iset[b] = np.concatenate([skel[c][0] for c in t.children[b] if c >= 0])
            # Active DOFs at this level: every level-lev box's I plus the points
            # of leaves at coarser levels (not yet eliminated).
            coarse = [t.dofs(b) for b in np.nonzero(t.is_leaf & (t.level < lev))[0]]
            active = np.concatenate([Iset[b] for b in boxes] + coarse)
            owner = np.concatenate([np.full(Iset[b].size, b) for b in boxes]
                                   + [np.full(c.size, -1) for c in coarse])
            self.active[lev] = active
            recs = []
            for b in boxes:
                I = Iset[b]
                cen, w = t.centre[b], t.width[b]
                d = xt[active] - cen[None, :]
                dist2 = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]
                rn = o["r_near"] * w
                near = active[(dist2 < rn * rn) & (owner != b)]
                prox = proxy_points(cen, w, o["n_prox"], o["r_in"], o["r_out"], o["n_rings"])
                A = np.vstack([
                    K.kernel_block(xt[near], xt[I], family, theta, which, alpha, near, I),
                    K.kernel_block(prox, xt[I], family, theta, which, alpha)])
                perm, k, T = interpolative_decomposition(A, tol)
                # Current diagonal block A_II (children's X_SS on the diagonal,
                # original kernel entries between different children).
                if t.is_leaf[b]:
                    AII = K.kernel_block(xt[I], xt[I], family, theta, which, alpha, I, I)
                else:
                    AII = K.kernel_block(xt[I], xt[I], family, theta, which, alpha, I, I)
                    off = 0
                    for c in t.children[b]:
                        if c < 0:
                            continue
                        Sc, Xc = skel[c]
                        AII[off:off + Sc.size, off:off + Sc.size] = Xc
                        off += Sc.size
                Sidx, Ridx = perm[:k], perm[k:]
                ASS = AII[np.ix_(Sidx, Sidx)]
                ASR = AII[np.ix_(Sidx, Ridx)]
                ARR = AII[np.ix_(Ridx, Ridx)]
                XSR = ASR - ASS @ T
                XRR = ARR - T.T @ ASR - XSR.T @ T
                XRR = 0.5 * (XRR + XRR.T)
                rec = BoxRecord()
                rec.box, rec.level, rec.I = b, lev, I
                rec.S, rec.R, rec.T, rec.k = I[Sidx], I[Ridx], T, k
                rec.near = near
                if Ridx.size == 0:
                    rec.E = np.zeros((k, 0)); rec.C = np.zeros((0, 0)); rec.XRR = XRR
                    XSS = ASS
                elif self.spd:
                    C = linalg.cholesky(XRR, lower=True)
                    V = linalg.solve_triangular(C, XSR.T, lower=True).T   # X_SR C^-T
                    rec.E = linalg.solve_triangular(C, V.T, lower=True, trans="T").T  # V C^-1
                    rec.C, rec.XRR = C, None
                    XSS = ASS - V @ V.T
                else:
                    lu = linalg.lu_factor(XRR)
                    rec.E = linalg.lu_solve(lu, XSR.T).T        # X_SR X_RR^-1 (X_RR symmetric)
                    rec.C, rec.XRR = None, XRR
                    XSS = ASS - rec.E @ XSR.T
                XSS = 0.5 * (XSS + XSS.T)
                skel[b] = (rec.S, XSS)
                recs.append(rec)
            self.records[lev] = recs
        # Root block: children's skeletons, or all points when the root is a leaf.
        if t.is_leaf[0]:
            I0 = t.dofs(0)
            A00 = K.kernel_block(xt[I0], xt[I0], family, theta, which, alpha, I0, I0)
        else:
            I0 = np.concatenate([skel[c][0] for c in t.children[0] if c >= 0])
            A00 = K.kernel_block(xt[I0], xt[I0], family, theta, which, alpha, I0, I0)
            off = 0
            for c in t.children[0]:
                if c < 0:
                    continue
                Sc, Xc = skel[c]
                A00[off:off + Sc.size, off:off + Sc.size] = Xc
                off += Sc.size
        self.I0 = I0
        self.A00 = 0.5 * (A00 + A00.T)
        if self.spd:
            self.C0 = linalg.cholesky(self.A00, lower=True)

    # ----- derived quantities -------------------------------------------
    def all_records(self):
        for lev in sorted(self.records):
            for r in self.records[lev]:
                yield r

    def logdet(self):
        """log|F| = 2 log|C| (Sec. 2.3.2)."""
        assert self.spd
        s = 2.0 * float(np.sum(np.log(np.diag(self.C0))))
        for r in self.all_records():
            if r.C.size:
                s += 2.0 * float(np.sum(np.log(np.diag(r.C))))
        return s

    def ranks(self):
        return {lev: [r.k for r in recs] for lev, recs in self.records.items()}

    def storage(self):
        """Number of factor entries (T, E and the diagonal blocks)."""
        s = self.I0.size ** 2
        for r in self.all_records():
            s += r.T.size + r.E.size + r.R.size ** 2
        return s

    # ----- the block unit-triangular passes ------------------------------
    def _up_inv(self, y):       # Q^-1: leaves first, L_I^-1 then U_I^-1
        for lev in range(self.tree.L, 0, -1):
            for r in self.records[lev]:
                y[r.R] -= r.T.T @ y[r.S]
                y[r.S] -= r.E @ y[r.R]

    def _down_inv(self, y):     # Q^-T: root side first, U_I^-T then L_I^-T
        for lev in range(1, self.tree.L + 1):
            for r in self.records[lev]:
                y[r.R] -= r.E.T @ y[r.S]
                y[r.S] -= r.T @ y[r.R]

    def _up_fwd(self, y):       # Q^T: leaves first, L_I^T then U_I^T
        for lev in range(self.tree.L, 0, -1):
            for r in self.records[lev]:
                y[r.S] += r.T @ y[r.R]
                y[r.R] += r.E.T @ y[r.S]

    def _down_fwd(self, y):     # Q: root side first, U_I then L_I
        for lev in range(1, self.tree.L + 1):
            for r in self.records[lev]:
                y[r.S] += r.E @ y[r.R]
                y[r.R] += r.T.T @ y[r.S]

    def _diag(self, y, op):
        """Block-diagonal middle factor: op in {'D', 'Dinv', 'C', 'CT', 'Cinv', 'CinvT'}."""
        blocks = [(r.R, r.C, r.XRR) for r in self.all_records() if r.R.size]
        blocks.append((self.I0, self.C0 if self.spd else None, None if self.spd else self.A00))
        for idx, C, X in blocks:
            v = y[idx]
            if op == "D":
                y[idx] = (C @ (C.T @ v)) if C is not None else X @ v
            elif op == "Dinv":
                y[idx] = linalg.cho_solve((C, True), v)
            elif op == "C":
                y[idx] = C @ v
            elif op == "CT":
                y[idx] = C.T @ v
            elif op == "Cinv":
                y[idx] = linalg.solve_triangular(C, v, lower=True)
            elif op == "CinvT":
                y[idx] = linalg.solve_triangular(C, v, lower=True, trans="T")

    def apply(self, x):
        """F x = Q D Q^T x."""
        y = np.array(x, dtype=np.float64, copy=True)
        self._up_fwd(y); self._diag(y, "D"); self._down_fwd(y)
        return y

    def solve(self, x):
        """F^-1 x = Q^-T D^-1 Q^-1 x."""
        assert self.spd
        y = np.array(x, dtype=np.float64, copy=True)
        self._up_inv(y); self._diag(y, "Dinv"); self._down_inv(y)
        return y

    def sqrt(self, x):
        """F^1/2 x = Q C x."""
        y = np.array(x, dtype=np.float64, copy=True)
        self._diag(y, "C"); self._down_fwd(y)
        return y

    def sqrt_t(self, x):
        """(F^1/2)^T x = C^T Q^T x."""
        y = np.array(x, dtype=np.float64, copy=True)
        self._up_fwd(y); self._diag(y, "CT")
        return y

    def inv_sqrt(self, x):
        """F^-1/2 x = C^-1 Q^-1 x."""
        y = np.array(x, dtype=np.float64, copy=True)
        self._up_inv(y); self._diag(y, "Cinv")
        return y

    def inv_sqrt_t(self, x):
        """(F^-1/2)^T x = Q^-T C^-T x."""
        y = np.array(x, dtype=np.float64, copy=True)
        self._diag(y, "CinvT"); self._down_inv(y)
        return y

    def dense(self):
        """F as a dense matrix (tree order), column by column; small n only."""
        return self.apply(np.eye(self.n))
