"""Pins of Oracle-D (dense Cholesky log-likelihood and exact score, Sec. 1
Eqs. (loglikelihood), (gradient)) against library routines and finite
differences."""
import numpy as np
import pytest
from scipy import stats

from oracle import dense
from oracle import kernels as K
from paper_1603_08057_gb300 import workloads as W


@pytest.fixture(scope="module")
def prob():
    x = W.uniform(300, 11)
    th = (0.1, 1.3, 1e-2)
    z = dense.sample_z_dense(x, K.MATERN32, th, W.standard_normal(300, 12))
    return x, z, th


def test_loglik_matches_scipy_logpdf(prob):
    x, z, th = prob
    S = dense.cov_matrix(x, K.MATERN32, th)
    ref = stats.multivariate_normal(mean=np.zeros(len(z)), cov=S).logpdf(z)
    ell, quad, logdet = dense.loglik_dense(x, z, K.MATERN32, th)
    assert ell == pytest.approx(ref, rel=1e-11)
    assert logdet == pytest.approx(np.linalg.slogdet(S)[1], rel=1e-12)


@pytest.mark.parametrize("fam,alpha", [(K.MATERN32, 0.0), (K.RQ, 1.0), (K.MATERN1, 0.0)])
def test_score_matches_central_differences(prob, fam, alpha):
    x, z, th = prob
    d = dense.score_dense(x, z, fam, th, alpha)
    for k in range(3):
        h = 1e-5 * th[k]
        tp = list(th); tp[k] += h
        tm = list(th); tm[k] -= h
        fd = (dense.loglik_dense(x, z, fam, tp, alpha)[0] - dense.loglik_dense(x, z, fam, tm, alpha)[0]) / (2 * h)
        scale = 0.5 * abs(d["quadk"][k]) + 0.5 * abs(d["trace"][k])
        assert abs(d["g"][k] - fd) <= 1e-7 * scale


def test_dlogdet_is_trace(prob):
    # d log|S| / d theta_k = Tr(S^-1 S_k), checked by central differences
    x, z, th = prob
    d = dense.score_dense(x, z, K.MATERN32, th)
    for k in range(3):
        h = 1e-5 * th[k]
        tp = list(th); tp[k] += h
        tm = list(th); tm[k] -= h
        fd = (dense.loglik_dense(x, z, K.MATERN32, tp)[2] - dense.loglik_dense(x, z, K.MATERN32, tm)[2]) / (2 * h)
        assert d["trace"][k] == pytest.approx(fd, rel=1e-7)


def test_sampled_z_has_the_model_covariance():
    # z = C w: with many w the empirical covariance approaches Sigma
    x = W.uniform(20, 3)
    th = (0.3, 1.0, 0.1)
    Wm = W.standard_normal(20, 4, 20000)
    Z = dense.sample_z_dense(x, K.MATERN32, th, Wm)
    S = dense.cov_matrix(x, K.MATERN32, th)
    assert np.max(np.abs(Z @ Z.T / 20000 - S)) < 0.05
