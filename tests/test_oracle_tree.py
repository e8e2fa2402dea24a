"""Pins of the oracle quadtree (Sec. 2.1, Remark (tree)) by brute force."""
import numpy as np
import pytest

from oracle.tree import Tree, proxy_points
from paper_1603_08057_gb300 import workloads as W


@pytest.mark.parametrize("kind,n", [("uniform", 3000), ("mixture", 5000)])
def test_tree_partitions_points(kind, n):
    x = W.make_points(kind, n, 5)
    t = Tree(x, 64)
    assert np.array_equal(np.sort(t.perm), np.arange(n))
    assert np.all(np.diff(t.key.astype(np.float64)) >= 0)
    for b in range(len(t.level)):
        pts = t.xt[t.start[b]:t.start[b] + t.count[b]]
        lo = t.centre[b] - t.width[b] / 2 - 1e-12
        hi = t.centre[b] + t.width[b] / 2 + 1e-12
        assert np.all(pts >= lo) and np.all(pts <= hi)
        if t.is_leaf[b]:
            assert t.count[b] <= 64
        else:
            assert t.count[b] > 64
            ch = t.children[b][t.children[b] >= 0]
            assert t.count[ch].sum() == t.count[b]
            assert t.start[ch[0]] == t.start[b]
            assert np.all(t.start[ch[1:]] == t.start[ch[:-1]] + t.count[ch[:-1]])
            assert np.all(t.level[ch] == t.level[b] + 1)


def test_tree_matches_direct_recursion():
    # brute force: recursive split by comparing coordinates with box mid-lines
    x = W.uniform(700, 9)
    t = Tree(x, 16)
    leaves_tree = sorted(tuple(sorted(t.perm[t.start[b]:t.start[b] + t.count[b]]))
                         for b in np.nonzero(t.is_leaf)[0])
    out = []

    def rec(idx, lo, w):
        if idx.size <= 16:
            out.append(tuple(sorted(idx)))
            return
        mid = lo + w / 2
        for sy in (0, 1):
            for sx in (0, 1):
                m = ((x[idx, 0] >= mid[0]) == bool(sx)) & ((x[idx, 1] >= mid[1]) == bool(sy))
                if np.any(m):
                    rec(idx[m], lo + w / 2 * np.array([sx, sy]), w / 2)

    rec(np.arange(700), t.lo, t.side)
    assert sorted(out) == leaves_tree


def test_proxy_annulus():
    p = proxy_points(np.array([0.3, 0.4]), 0.1, 256, 1.0, 2.0, 8)
    r = np.hypot(p[:, 0] - 0.3, p[:, 1] - 0.4)
    assert p.shape == (256, 2) and r.min() > 0.1 and r.max() < 0.2
