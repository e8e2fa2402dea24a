"""Batched datasets: one forest over independent point sets, through the C ABI.

A batch of independent datasets has the block-diagonal covariance
diag(Sigma_1, ..., Sigma_m); rsf_build_batched factors it as one forest (one
quadtree per set, all sets' boxes of a level in the same launches).  Checked:

* per-set log-likelihood and score against the dense fp64 oracle (the same
  bars as the single-set parity tests: l 1e-6, score 1e-3 relative and 1e-5
  of the term scale), on sets of ragged sizes including 1, 64 and 65 points;
* the forest against single-set factorizations of each set: per-set
  log-determinants and block-diagonal solves agree to 1e-12 (the per-box
  arithmetic is the same; only summation groupings differ);
* the RQ (alpha = 1) batch of 64 datasets with n_i = round(exp(U[log 2048,
  log 32768])) (dataset i: points seed 100 + i, z seed 200 + i), l = 0.05,
  s2 = 1, nugget 1e-3: per-set log-likelihoods against single-set ones, and
  the scores of the first 8 sets against single-set scores: 1e-3 relative
  (the acceptance bar of the score) and 5e-5 of the term scale, since the
  two peelings draw different test matrices and sample counts and each
  carries its own error (measured up to 1.4e-5 of the scale, g_l of set 5).
"""
import math

import numpy as np
import pytest

from oracle import dense
from oracle import kernels as K
from paper_1603_08057_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_08057_gb300 import build
    build.build()
    from paper_1603_08057_gb300 import binding
    return binding


def T(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def _sets(sizes, seed0, mixture=False):
    pts = [W.mixture(n, seed0 + i) if mixture and n > 200 else W.uniform(n, seed0 + i) for i, n in enumerate(sizes)]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return pts, off


def test_batched_matches_dense_per_set(B):
    sizes = [700, 1, 2000, 64, 65, 1500]
    th = (0.06, 1.5, 5e-3)
    pts, off = _sets(sizes, 501, mixture=True)
    zs = [dense.sample_z_dense(p, K.MATERN32, th, W.standard_normal(len(p), 601 + i)) for i, p in enumerate(pts)]
    ll, g, t = B.loglik_and_score_batched(T(np.concatenate(pts)), off, T(np.concatenate(zs)), B.MATERN32, th,
                                          1e-9, 1e-6)
    for i, (p, z) in enumerate(zip(pts, zs)):
        d = dense.score_dense(p, z, K.MATERN32, th)
        assert abs(ll[i] - d["ell"]) <= 1e-6 * abs(d["ell"]), i
        scale = 0.5 * np.abs(d["quadk"]) + 0.5 * np.abs(d["trace"])
        assert np.all(np.abs(g[i] - d["g"]) <= 1e-5 * scale + 1e-3 * np.abs(d["g"])), i
        np.testing.assert_allclose(t[i, :3], d["quadk"], rtol=1e-6)
        np.testing.assert_allclose(t[i, 3:], d["trace"], rtol=1e-5, atol=1e-9 * len(p))


def test_forest_equals_single_set_factorizations(B):
    sizes = [3000, 517, 1, 2048]
    th = (0.05, 2.0, 1e-2)
    pts, off = _sets(sizes, 511, mixture=True)
    Fb = B.Factorization(T(np.concatenate(pts)), B.MATERN32, th, B.SIGMA, 1e-9, offsets=off)
    assert Fb.info()["nsets"] == len(sizes)
    lds = Fb.logdet_sets()
    assert Fb.logdet() == pytest.approx(float(np.sum(lds)), rel=1e-13)
    V = W.standard_normal(int(off[-1]), 512, 3)
    Yb = Fb.solve(T(V), B.OP_INV).cpu().numpy()
    for i, p in enumerate(pts):
        Fi = B.Factorization(T(p), B.MATERN32, th, B.SIGMA, 1e-9)
        assert lds[i] == pytest.approx(Fi.logdet(), rel=1e-12, abs=1e-12)
        yi = Fi.solve(T(V[off[i]:off[i + 1]]), B.OP_INV).cpu().numpy()
        assert np.max(np.abs(Yb[off[i]:off[i + 1]] - yi)) <= 1e-12 * max(1.0, np.max(np.abs(yi)))


def test_rq_batch_of_64_datasets(B):
    rng = np.random.default_rng(7)
    sizes = [int(round(math.exp(v))) for v in rng.uniform(math.log(2048), math.log(32768), 64)]
    th = (0.05, 1.0, 1e-3)
    pts = [W.uniform(n, 100 + i) for i, n in enumerate(sizes)]
    zs = [W.standard_normal(n, 200 + i) for i, n in enumerate(sizes)]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    P, Z = T(np.concatenate(pts)), T(np.concatenate(zs))
    ll, _, _ = B.loglik_and_score_batched(P, off, Z, B.RQ, th, 1e-9, 1e-6, 1.0, want_score=False)
    for i in range(64):
        Fi = B.Factorization(T(pts[i]), B.RQ, th, B.SIGMA, 1e-9, 1.0)
        lli, _, _ = Fi.loglik(T(zs[i]))
        assert ll[i] == pytest.approx(lli, rel=1e-12), i
    m = 8
    ll8, g8, t8 = B.loglik_and_score_batched(T(np.concatenate(pts[:m])), off[:m + 1], T(np.concatenate(zs[:m])),
                                             B.RQ, th, 1e-9, 1e-6, 1.0)
    for i in range(m):
        lli, gi, ti = B.loglik_and_score(T(pts[i]), T(zs[i]), B.RQ, th, 1e-9, 1e-6, 1.0)
        gi, ti = gi.numpy(), ti.numpy()
        assert ll8[i] == pytest.approx(lli, rel=1e-12)
        scale = 0.5 * np.abs(ti[:3]) + 0.5 * np.abs(ti[3:])
        assert np.all(np.abs(g8[i] - gi) <= 5e-5 * scale), i
        assert np.all(np.abs(g8[i] - gi) <= 1e-3 * np.abs(gi)), i
