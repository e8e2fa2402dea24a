"""Weak-admissibility matrix peeling for Tr(G) of a symmetric black-box G.

ORACLE -- test infrastructure only (tests, smoke check, benchmark CPU leg).

Sec. 3, step by step:

* Sec. 3.1, Eq. (lowrankapprox): A ~ U1 [(W2^T U1)^+ (W2^T A W1) (U2^T W1)^+] U2^T
  with U1, U2 bases of the column spaces of A W1 and A^T W2, W i.i.d. N(0,1)
  with r + c columns.
* Sec. 3.2: top-down over levels l = 1..L.  At level l, W_k (k = 1..4) is
  nonzero only on the boxes in child slot k of their parent; applying
  G - sum_{m<l} G^(m) to W_k samples every sibling block G_ij with j in slot k
  (Def. sibs).  By symmetry the samples of G_ji give the row space of G_ij.
* Sec. 3.2.4: at the bottom, H = (G - sum_m G^(m)) E with E the stacked leaf
  identities; Tr(G) ~ sum over leaves of Tr H(I_i, [n_i]).

Readings where the paper is silent (they are the product's readings too):

* adaptive tree: the families at level l are the non-leaf boxes of level l-1;
  leaves at coarser levels keep their diagonal block until the extraction;
* sample count: r_l + c columns with c = 10 (Sec. 3.2.1); the adaptive rank
  procedure starts from q = max(q0, r_prev) + c columns, compresses every
  sibling block by column-pivoted QR with relative cut-off eps_peel, and if a
  detected rank exceeds q - c appends q fresh columns and recompresses;
* bases U are the orthonormal Q factors of the pivoted QR truncated at the
  detected rank; pseudo-inverses via SVD with cut-off eps_mach * max(size);
* each unordered sibling pair is compressed once with the symmetrised core
  (W_i^T Y_ij + (W_j^T Y_ji)^T)/2, and G^(l)_ji = (G^(l)_ij)^T;
* W entries come from Philox4x32-10 (see philox.py), stream 0.
"""
from __future__ import annotations

import numpy as np
from scipy import linalg

from . import philox


def _basis(Y, tol):
    """Orthonormal basis of range(Y) by column-pivoted QR, rank at relative
    cut-off tol on |R_jj| / |R_11|."""
    if Y.shape[1] == 0 or Y.shape[0] == 0:
        return np.zeros((Y.shape[0], 0)), 0
    Q, R, _ = linalg.qr(Y, mode="economic", pivoting=True)
    d = np.abs(np.diag(R))
    if d[0] == 0.0:
        return np.zeros((Y.shape[0], 0)), 0
    r = int(np.sum(d > tol * d[0]))
    return Q[:, :r], r


class PeelLevel:
    def __init__(self):
        self.blocks = []   # (a_start, a_count, b_start, b_count, U_ab, M_ab, U_ba)

    def apply(self, X, out):
        """out += G^(l) X (both in tree order)."""
        for a0, na, b0, nb, Uab, Mab, Uba in self.blocks:
            out[a0:a0 + na] += Uab @ (Mab @ (Uba.T @ X[b0:b0 + nb]))


def peel_trace(apply_G, tree, tol_peel, c=10, seed=0, q0=32, max_q=None):
    """Trace of the symmetric operator ``apply_G`` (X (n,q) -> G X, tree
    order) by weak peeling over ``tree``.  Returns (trace, info)."""
    t = tree
    n = t.n
    levels = []
    info = dict(ranks={}, samples={}, applies=0)
    r_prev = 0
    for lev in range(1, t.L + 1):
        fam = [b for b in t.boxes_at(lev - 1) if not t.is_leaf[b]]
        kids = {b: [(int(s), int(t.children[b][s])) for s in range(4) if t.children[b][s] >= 0]
                for b in fam}
        boxes = t.boxes_at(lev)
        if not any(len(v) > 1 for v in kids.values()):
            levels.append(PeelLevel())
            continue
        # rows belonging to level-lev boxes, grouped by child slot
        slot_rows = [np.concatenate([t.dofs(b) for b in boxes if t.slot[b] == s] or [np.zeros(0, np.int64)])
                     for s in range(4)]
        q = max(q0, r_prev) + c
        Wc = np.zeros((n, 0)); Y = [np.zeros((n, 0)) for _ in range(4)]
        while True:
            qa = Wc.shape[1]
            new_cols = np.arange(qa, q)
            rows_all = np.concatenate([t.dofs(b) for b in boxes])
            Wn = np.zeros((n, q - qa))
            Wn[rows_all] = philox.normals(rows_all, new_cols, lev, 0, seed)
            Wc = np.hstack([Wc, Wn])
            for s in range(4):
                Ws = np.zeros((n, q - qa))
                Ws[slot_rows[s]] = Wn[slot_rows[s]]
                Ys = apply_G(Ws)
                info["applies"] += q - qa
                for L_ in levels:
                    corr = np.zeros_like(Ys)
                    L_.apply(Ws, corr)
                    Ys = Ys - corr
                Y[s] = np.hstack([Y[s], Ys])
            # compress all sibling pairs
            PL = PeelLevel()
            rmax = 0
            for b in fam:
                ch = kids[b]
                for ii in range(len(ch)):
                    for jj in range(ii + 1, len(ch)):
                        si, bi = ch[ii]
                        sj, bj = ch[jj]
                        Ii, Ij = t.dofs(bi), t.dofs(bj)
                        Yij = Y[sj][Ii]          # ~ G_ij W_j
                        Yji = Y[si][Ij]          # ~ G_ji W_i
                        U1, r1 = _basis(Yij, tol_peel)
                        U2, r2 = _basis(Yji, tol_peel)
                        rmax = max(rmax, r1, r2)
                        Wi, Wj = Wc[Ii], Wc[Ij]
                        core = 0.5 * (Wi.T @ Yij + (Wj.T @ Yji).T)
                        M = np.linalg.pinv(Wi.T @ U1) @ core @ np.linalg.pinv(U2.T @ Wj)
                        PL.blocks.append((Ii[0], Ii.size, Ij[0], Ij.size, U1, M, U2))
                        PL.blocks.append((Ij[0], Ij.size, Ii[0], Ii.size, U2, M.T, U1))
            if rmax <= q - c or (max_q is not None and q >= max_q):
                break
            q = q + q
        info["ranks"][lev] = rmax
        info["samples"][lev] = q
        r_prev = rmax
        levels.append(PL)
    # extraction
    pos = t.leaf_pos()
    nL = int(t.count[t.is_leaf].max())
    E = np.zeros((n, nL))
    E[np.arange(n), pos] = 1.0
    H = apply_G(E)
    info["applies"] += nL
    for L_ in levels:
        corr = np.zeros_like(H)
        L_.apply(E, corr)
        H = H - corr
    tr = float(np.sum(H[np.arange(n), pos]))
    info["levels"] = levels
    return tr, info


def hutchinson(apply_G, n, q, seed=0):
    """Hutchinson estimator (Sec. 3, Eq. (hutch)) with Rademacher vectors
    drawn from Philox stream 1 (sign of the normal draw)."""
    u = np.sign(philox.normals(np.arange(n), np.arange(q), 0, 1, seed))
    u[u == 0] = 1.0
    Gu = apply_G(u)
    vals = np.sum(u * Gu, axis=0)
    return float(np.mean(vals)), float(np.std(vals, ddof=1) / np.sqrt(q))
