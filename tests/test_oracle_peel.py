"""Pins of the oracle peeling trace (Sec. 3) and of its random generator."""
import os

import numpy as np
import pytest

from oracle import dense, peel, philox, rsf
from oracle import kernels as K
from oracle.tree import Tree
from paper_1603_08057_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def test_philox_known_answers():
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        out = philox.philox4x32_10(*v[:6])
        assert [int(o) for o in out] == v[6:]


def test_philox_normals_are_standard():
    z = philox.normals(np.arange(400), np.arange(100), 3, 0, 99)
    assert abs(z.mean()) < 0.02 and abs(z.std() - 1.0) < 0.02
    # independent of how the matrix is cut: entries depend on (row, col) only
    z2 = philox.normals(np.arange(100, 200), np.arange(37, 61), 3, 0, 99)
    np.testing.assert_array_equal(z2, z[100:200, 37:61])


def _synthetic_hierarchical(tree, ranks, seed):
    """Dense symmetric G whose sibling blocks are exactly low rank (rank
    ranks[l] at level l) plus arbitrary leaf diagonal blocks."""
    rng = np.random.default_rng(seed)
    n = tree.n
    G = np.zeros((n, n))
    for b in range(len(tree.level)):
        if tree.is_leaf[b]:
            I = tree.dofs(b)
            B = rng.standard_normal((I.size, I.size))
            G[np.ix_(I, I)] += B + B.T
        ch = [c for c in tree.children[b] if c >= 0]
        r = ranks[min(tree.level[b] + 1, len(ranks) - 1)]
        for i in range(len(ch)):
            for j in range(i + 1, len(ch)):
                Ii, Ij = tree.dofs(ch[i]), tree.dofs(ch[j])
                blk = rng.standard_normal((Ii.size, r)) @ rng.standard_normal((r, Ij.size))
                G[np.ix_(Ii, Ij)] += blk
                G[np.ix_(Ij, Ii)] += blk.T
    return G


def test_peeling_exact_on_exactly_low_rank_blocks():
    x = W.mixture(2000, 51)
    t = Tree(x, 64)
    G = _synthetic_hierarchical(t, [0, 12, 9, 7, 5, 4, 3, 3, 3], 52)
    tr, info = peel.peel_trace(lambda X: G @ X, t, 1e-10, seed=7)
    assert tr == pytest.approx(np.trace(G), rel=1e-10, abs=1e-8 * np.abs(np.diag(G)).sum())


def test_peeling_inverse_covariance_trace():
    x = W.uniform(1500, 61)
    th = (0.1, 1.0, 1e-2)
    F = rsf.Factorization(x, K.MATERN32, th, K.SIGMA, 1e-10)
    S = dense.cov_matrix(F.tree.xt, K.MATERN32, th)
    exact = np.trace(np.linalg.inv(S))
    tr, info = peel.peel_trace(F.solve, F.tree, 1e-6, seed=3)
    assert tr == pytest.approx(exact, rel=1e-5)
    # the naive trace of Sec. 5.2: G applied to every unit vector
    brute = np.trace(F.solve(np.eye(F.n)))
    assert tr == pytest.approx(brute, rel=1e-5)


def test_peeling_agrees_with_hutchinson_within_its_error():
    x = W.uniform(1000, 71)
    th = (0.1, 1.0, 1e-2)
    F = rsf.Factorization(x, K.MATERN32, th, K.SIGMA, 1e-10)
    tr, _ = peel.peel_trace(F.solve, F.tree, 1e-6, seed=3)
    h, se = peel.hutchinson(F.solve, F.n, 4000, seed=5)
    assert abs(h - tr) < 4 * se


def test_variance_and_nugget_traces_sum_to_n():
    # Sigma = s2 Sigma_s2 + nug I  =>  s2 Tr(S^-1 S_s2) + nug Tr(S^-1) = n
    x = W.mixture(1200, 81)
    th = (0.05, 2.0, 1e-2)
    F = rsf.Factorization(x, K.MATERN32, th, K.SIGMA, 1e-10)
    Fs = rsf.Factorization(x, K.MATERN32, th, K.D_S2, 1e-10, tree=F.tree)
    t_nug, _ = peel.peel_trace(F.solve, F.tree, 1e-7, seed=1)
    t_s2, _ = peel.peel_trace(lambda X: 0.5 * (F.solve(Fs.apply(X)) + Fs.apply(F.solve(X))),
                              F.tree, 1e-7, seed=2)
    assert th[1] * t_s2 + th[2] * t_nug == pytest.approx(1200, rel=1e-6)
