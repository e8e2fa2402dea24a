"""Pin of the oracle's Algorithm 1 (Sec. 4) against the dense exact
log-likelihood and score: the acceptance bars 1e-6 (l) and 1e-3 (g)."""
import numpy as np
import pytest

from oracle import dense, mle
from oracle import kernels as K
from paper_1603_08057_gb300 import workloads as W


@pytest.mark.parametrize("kind,n,fam,alpha,th", [
    ("uniform", 2048, K.MATERN32, 0.0, (0.1, 1.0, 1e-2)),
    ("mixture", 1536, K.RQ, 1.0, (0.05, 1.0, 1e-3)),
])
def test_algorithm1_matches_dense(kind, n, fam, alpha, th):
    x = W.make_points(kind, n, 2)
    z = dense.sample_z_dense(x, fam, th, W.standard_normal(n, 3), alpha)
    d = dense.score_dense(x, z, fam, th, alpha)
    r = mle.loglik_and_score(x, z, fam, th, 1e-9, 1e-6, alpha, seed=4)
    assert abs(r["ell"] - d["ell"]) <= 1e-6 * abs(d["ell"])
    assert np.all(np.abs(r["g"] - d["g"]) <= 1e-3 * np.abs(d["g"]))
    scale = 0.5 * np.abs(d["quadk"]) + 0.5 * np.abs(d["trace"])
    assert np.all(np.abs(r["g"] - d["g"]) <= 1e-6 * scale)
