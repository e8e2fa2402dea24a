"""Pins of the oracle's profile likelihood (Sec. 5.5, Eq. (prof) and its
gradient) and conditional distribution (Remark conditional, Sec. 4) against
scipy's Gaussian density, finite differences, the Sherman-Morrison identity,
the block-inverse identity and closed forms at observed locations."""
import numpy as np
import pytest
from scipy import linalg, stats

from oracle import dense
from oracle import kernels as K
from oracle import profile as P
from oracle.rsf import Factorization
from oracle.tree import Tree
from paper_1603_08057_gb300 import workloads as W

TH = (0.1, 1.0, 1e-2)


@pytest.fixture(scope="module")
def prob():
    x = W.uniform(300, 21)
    z = 0.7 + 1.5 * dense.sample_z_dense(x, K.MATERN32, TH, W.standard_normal(300, 22))
    return x, z


def test_profile_is_the_maximum_over_the_variance_level(prob):
    # lt = max over s of log N(z; 0, s A) with log|A| replaced by log|Sigma|;
    # scipy's density fixes the constant (log n - 1 - log 2 pi)
    x, z = prob
    n = len(z)
    lt, qt, logdet = P.profile_loglik_dense(x, z, K.MATERN32, TH)
    S = dense.cov_matrix(x, K.MATERN32, TH)
    A = S + np.ones((n, n))
    ldA = np.linalg.slogdet(A)[1]
    assert logdet == pytest.approx(np.linalg.slogdet(S)[1], rel=1e-12)
    s_hat = qt / n

    def ell(s):
        return stats.multivariate_normal(mean=np.zeros(n), cov=s * A).logpdf(z)

    assert ell(s_hat) + 0.5 * ldA - 0.5 * logdet == pytest.approx(lt, rel=1e-11)
    assert ell(s_hat * 1.001) < ell(s_hat) and ell(s_hat * 0.999) < ell(s_hat)


def test_profile_quadratic_by_sherman_morrison(prob):
    # z^T (Sigma + 1 1^T)^-1 z through solves with Sigma alone
    x, z = prob
    n = len(z)
    S = dense.cov_matrix(x, K.MATERN32, TH)
    a = np.linalg.solve(S, z)
    b = np.linalg.solve(S, np.ones(n))
    q_sm = z @ a - (np.sum(a)) ** 2 / (1.0 + np.sum(b))
    assert P.profile_loglik_dense(x, z, K.MATERN32, TH)[1] == pytest.approx(q_sm, rel=1e-11)


@pytest.mark.parametrize("fam,alpha", [(K.MATERN32, 0.0), (K.MATERN52, 0.0), (K.RQ, 2.0)])
def test_profile_gradient_matches_central_differences(prob, fam, alpha):
    x, z = prob
    d = P.profile_score_dense(x, z, fam, TH, alpha)
    n = len(z)
    for k in range(3):
        h = 1e-5 * TH[k]
        tp = list(TH); tp[k] += h
        tm = list(TH); tm[k] -= h
        fd = (P.profile_loglik_dense(x, z, fam, tp, alpha)[0] - P.profile_loglik_dense(x, z, fam, tm, alpha)[0]) / (2 * h)
        scale = 0.5 * abs(d["trace"][k]) + 0.5 * n * abs(d["quadk"][k]) / d["qt"]
        assert abs(d["g"][k] - fd) <= 1e-7 * scale


def test_profile_level_invariance(prob):
    # scaling z by c moves lt by -n log c and leaves the gradient unchanged
    x, z = prob
    n = len(z)
    d1 = P.profile_score_dense(x, z, K.MATERN32, TH)
    d2 = P.profile_score_dense(x, 3.0 * z, K.MATERN32, TH)
    assert d2["lt"] == pytest.approx(d1["lt"] - n * np.log(3.0), rel=1e-12)
    np.testing.assert_allclose(d2["g"], d1["g"], rtol=1e-10)


def test_conditional_mean_at_observed_points(prob):
    # at an observed location the cross covariance is that row of Sigma minus
    # the nugget: mean_j = z_j - nug (Sigma^-1 z)_j; without nugget the
    # conditional law collapses on z_j
    x, z = prob
    idx = np.array([3, 17, 150, 299])
    mean, cov = P.conditional_dense(x, z, x[idx], K.MATERN32, TH)
    a = np.linalg.solve(dense.cov_matrix(x, K.MATERN32, TH), z)
    np.testing.assert_allclose(mean, z[idx] - TH[2] * a[idx], rtol=1e-9, atol=1e-12)
    th0 = (0.1, 1.0, 0.0)
    xm = x[:120]
    zm = dense.sample_z_dense(xm, K.MATERN12, th0, W.standard_normal(120, 23))
    mean0, cov0 = P.conditional_dense(xm, zm, xm[idx[:2]], K.MATERN12, th0)
    np.testing.assert_allclose(mean0, zm[idx[:2]], rtol=1e-8, atol=1e-10)
    assert np.max(np.abs(cov0)) <= 1e-9


def test_conditional_covariance_is_the_schur_complement(prob):
    # S11 - S12 S22^-1 S21 = ((Sigma_joint^-1)_11)^-1
    x, z = prob
    xs = W.uniform(25, 24)
    mean, cov = P.conditional_dense(x, z, xs, K.MATERN32, TH)
    xj = np.vstack([xs, x])
    Sj = dense.cov_matrix(xj, K.MATERN32, TH)
    inv11 = np.linalg.inv(Sj)[:25, :25]
    np.testing.assert_allclose(cov, np.linalg.inv(inv11), rtol=1e-8, atol=1e-10 * np.max(np.abs(cov)))
    # and the mean is the joint's regression: -(inv11)^-1 (Sigma_joint^-1)_12 z
    inv12 = np.linalg.inv(Sj)[:25, 25:]
    np.testing.assert_allclose(mean, -np.linalg.solve(inv11, inv12 @ z), rtol=1e-8, atol=1e-10)


def test_conditional_samples_have_the_conditional_covariance(prob):
    # with w = I the sample deviations D satisfy D D^T = conditional covariance,
    # for the dense Cholesky root and for the RSF root F^1/2 of the joint matrix
    x, z = prob
    m = 25
    xs = W.uniform(m, 24)
    mean, cov = P.conditional_dense(x, z, xs, K.MATERN32, TH)
    xj = np.vstack([xs, x])
    Sj = dense.cov_matrix(xj, K.MATERN32, TH)
    C = linalg.cholesky(Sj, lower=True)
    S22 = Sj[m:, m:]
    Ij = np.eye(len(xj))
    s = P.conditional_samples(mean, lambda v: Sj @ v, lambda v: C @ v, lambda v: np.linalg.solve(S22, v), Ij, m)
    D = s - mean[:, None]
    np.testing.assert_allclose(D @ D.T, cov, atol=1e-10 * np.max(np.abs(cov)))

    tj = Tree(xj, 64)
    t2 = Tree(x, 64)
    Fj = Factorization(xj, K.MATERN32, TH, K.SIGMA, 1e-12, tree=tj)
    F2 = Factorization(x, K.MATERN32, TH, K.SIGMA, 1e-12, tree=t2)
    s = P.conditional_samples(mean, _caller(Fj.apply, tj.perm), _caller(Fj.sqrt, tj.perm),
                              _caller(F2.solve, t2.perm), Ij, m)
    D = s - mean[:, None]
    np.testing.assert_allclose(D @ D.T, cov, atol=1e-8 * np.max(np.abs(cov)))


def _caller(op, perm):
    """Operator on caller-order (k, q) arrays from a tree-order one."""
    def f(v):
        out = np.empty_like(v)
        out[perm] = op(v[perm])
        return out
    return f
