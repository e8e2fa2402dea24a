"""Pins of the oracle's anisotropic kernels (Sec. 5.1: scaled distance
||x - y||_theta, Eqs. (specrq) and (specmatern)) and of the four-component
score built on them."""
import numpy as np
import pytest

from oracle import dense
from oracle import kernels as K
from oracle import mle as omle
from paper_1603_08057_gb300 import workloads as W

TH = (10.0, 1.0, 1e-4, 7.0)   # theta = [10, 7], unit variance, nugget 1e-4 (Sec. 5.1)


@pytest.fixture(scope="module")
def pts():
    return W.grid(12, 0.0, 100.0)


def test_paper_kernels_written_out(pts):
    # Eq. (specrq): (1 + ||x-y||_theta^2)^(-1/2) + nug delta; Eq. (specmatern):
    # (1 + sqrt3 ||x-y||_theta) exp(-sqrt3 ||x-y||_theta) + nug delta
    x = pts
    d2 = ((x[:, None, 0] - x[None, :, 0]) / 10.0) ** 2 + ((x[:, None, 1] - x[None, :, 1]) / 7.0) ** 2
    d = np.sqrt(d2)
    nug = 1e-4 * np.eye(len(x))
    np.testing.assert_allclose(dense.cov_matrix(x, K.RQ, TH, alpha=0.5), (1.0 + d2) ** -0.5 + nug, rtol=1e-14)
    np.testing.assert_allclose(dense.cov_matrix(x, K.MATERN32, TH),
                               (1.0 + np.sqrt(3.0) * d) * np.exp(-np.sqrt(3.0) * d) + nug, rtol=1e-13, atol=1e-300)


@pytest.mark.parametrize("fam,alpha", [(K.MATERN12, 0), (K.MATERN32, 0), (K.MATERN52, 0), (K.MATERN1, 0), (K.RQ, 0.5)])
def test_equal_length_scales_reduce_to_isotropic(pts, fam, alpha):
    x = pts / 100.0
    iso = (0.2, 1.3, 1e-2)
    an = (0.2, 1.3, 1e-2, 0.2)
    for which in (K.SIGMA, K.D_S2, K.D_NUG):
        np.testing.assert_allclose(dense.cov_matrix(x, fam, an, which, alpha), dense.cov_matrix(x, fam, iso, which, alpha),
                                   rtol=1e-13, atol=1e-15)
    # d/dl of the isotropic kernel = d/dl1 + d/dl2 at l1 = l2 = l
    s = dense.cov_matrix(x, fam, an, K.D_L, alpha) + dense.cov_matrix(x, fam, an, K.D_L2, alpha)
    np.testing.assert_allclose(s, dense.cov_matrix(x, fam, iso, K.D_L, alpha), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("fam,alpha", [(K.MATERN32, 0), (K.MATERN52, 0), (K.MATERN1, 0), (K.RQ, 0.5), (K.RQ, 2.0)])
def test_length_scale_derivatives_by_central_differences(pts, fam, alpha):
    x = pts
    for k, which in ((0, K.D_L), (3, K.D_L2)):
        h = 1e-6 * TH[k]
        tp = list(TH); tp[k] += h
        tm = list(TH); tm[k] -= h
        fd = (dense.cov_matrix(x, fam, tp, K.SIGMA, alpha) - dense.cov_matrix(x, fam, tm, K.SIGMA, alpha)) / (2 * h)
        an = dense.cov_matrix(x, fam, TH, which, alpha)
        np.testing.assert_allclose(an, fd, rtol=1e-6, atol=1e-9 * np.max(np.abs(an)))


def test_swapping_axes_swaps_length_scales(pts):
    x = W.uniform(50, 5) * 100.0
    xs = x[:, ::-1].copy()
    sw = (TH[3], TH[1], TH[2], TH[0])
    for a, b in ((K.SIGMA, K.SIGMA), (K.D_L, K.D_L2), (K.D_L2, K.D_L)):
        np.testing.assert_allclose(dense.cov_matrix(x, K.MATERN32, TH, a), dense.cov_matrix(xs, K.MATERN32, sw, b),
                                   rtol=1e-14, atol=1e-300)


def test_dense_score_four_components_by_finite_differences():
    x = W.grid(16, 0.0, 100.0)
    th = (10.0, 1.0, 1e-2, 7.0)
    z = dense.sample_z_dense(x, K.MATERN32, th, W.standard_normal(len(x), 31))
    d = dense.score_dense(x, z, K.MATERN32, th)
    assert d["g"].shape == (4,)
    for k in range(4):
        h = 1e-5 * th[k]
        tp = list(th); tp[k] += h
        tm = list(th); tm[k] -= h
        fd = (dense.loglik_dense(x, z, K.MATERN32, tp)[0] - dense.loglik_dense(x, z, K.MATERN32, tm)[0]) / (2 * h)
        scale = 0.5 * abs(d["quadk"][k]) + 0.5 * abs(d["trace"][k])
        assert abs(d["g"][k] - fd) <= 1e-7 * scale


def test_rsf_algorithm1_anisotropic_matches_dense():
    # Algorithm 1 on the paper's grid form with its four score components
    x = W.grid(24, 0.0, 100.0)
    th = (10.0, 1.0, 1e-2, 7.0)
    z = dense.sample_z_dense(x, K.MATERN32, th, W.standard_normal(len(x), 32))
    d = dense.score_dense(x, z, K.MATERN32, th)
    r = omle.loglik_and_score(x, z, K.MATERN32, th, 1e-9, 1e-6)
    assert abs(r["ell"] - d["ell"]) <= 1e-6 * abs(d["ell"])
    scale = 0.5 * np.abs(d["quadk"]) + 0.5 * np.abs(d["trace"])
    assert np.all(np.abs(r["g"] - d["g"]) <= 1e-3 * np.abs(d["g"]))
    assert np.all(np.abs(r["g"] - d["g"]) <= 1e-5 * scale)
