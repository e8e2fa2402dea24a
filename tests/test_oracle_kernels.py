"""Pins of the oracle's covariance kernels against closed forms, library
Bessel functions and finite differences (Sec. 1 Eqs. (matern),
(rationalquadratic); Sec. 5.5 Eq. (diffkernels))."""
import numpy as np
import pytest
from scipy import special

from oracle import kernels as K

R = np.linspace(0.0, 0.7, 57)


def test_matern_half_is_exponential():
    # nu = 1/2 of the Bessel form is exp(-r/l) (closed form), Sec. 5.5
    l = 0.13
    np.testing.assert_allclose(K.matern_general(R, 0.5, l), np.exp(-R / l), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(K.correlation(R, K.MATERN12, l), np.exp(-R / l), rtol=1e-15)


@pytest.mark.parametrize("fam,nu", [(K.MATERN12, 0.5), (K.MATERN32, 1.5), (K.MATERN52, 2.5), (K.MATERN1, 1.0)])
def test_matern_closed_forms_match_bessel(fam, nu):
    l = 0.09
    np.testing.assert_allclose(K.correlation(R, fam, l), K.matern_general(R, nu, l), rtol=1e-12, atol=1e-15)


def test_matern32_via_half_integer_bessel():
    # K_{3/2}(x) = sqrt(pi/(2x)) e^{-x} (1 + 1/x): an independent route to nu = 3/2
    l = 0.2
    r = R[1:]
    x = np.sqrt(3.0) * r / l
    k32 = np.sqrt(np.pi / (2 * x)) * np.exp(-x) * (1 + 1 / x)
    ref = 2 ** (1 - 1.5) / special.gamma(1.5) * x ** 1.5 * k32
    np.testing.assert_allclose(K.correlation(r, K.MATERN32, l), ref, rtol=1e-13)


def test_rq_tends_to_gaussian():
    # Sec. 1: the Gaussian kernel is the alpha -> infinity limit of RQ
    l = 0.1
    g = np.exp(-R ** 2 / (2 * l * l))
    np.testing.assert_allclose(K.correlation(R, K.RQ, l, alpha=1e7), g, rtol=2e-5, atol=1e-12)


@pytest.mark.parametrize("fam,alpha", [(K.MATERN12, 0), (K.MATERN32, 0), (K.MATERN52, 0), (K.MATERN1, 0), (K.RQ, 1.0), (K.RQ, 2.0), (K.RQ, 0.5)])
def test_unit_value_at_zero(fam, alpha):
    assert K.correlation(np.array([0.0]), fam, 0.3, alpha)[0] == pytest.approx(1.0, abs=1e-15)


@pytest.mark.parametrize("fam,alpha", [(K.MATERN12, 0), (K.MATERN32, 0), (K.MATERN52, 0), (K.MATERN1, 0), (K.RQ, 1.0), (K.RQ, 2.0)])
def test_length_scale_derivative_finite_difference(fam, alpha):
    theta = (0.11, 1.7, 0.01)
    r = R[1:]
    h = 1e-6 * theta[0]
    up = K.kernel_offdiag(r, fam, (theta[0] + h, theta[1], theta[2]), K.SIGMA, alpha)
    dn = K.kernel_offdiag(r, fam, (theta[0] - h, theta[1], theta[2]), K.SIGMA, alpha)
    fd = (up - dn) / (2 * h)
    an = K.kernel_offdiag(r, fam, theta, K.D_L, alpha)
    np.testing.assert_allclose(an, fd, rtol=1e-7, atol=1e-9 * np.max(np.abs(an)))


def test_variance_and_nugget_derivatives():
    theta = (0.1, 2.0, 0.03)
    r = R[1:]
    np.testing.assert_allclose(K.kernel_offdiag(r, K.MATERN32, theta, K.D_S2) * theta[1],
                               K.kernel_offdiag(r, K.MATERN32, theta, K.SIGMA), rtol=1e-15)
    assert np.all(K.kernel_offdiag(r, K.MATERN32, theta, K.D_NUG) == 0.0)
    assert K.diag_value(K.MATERN32, theta, K.SIGMA) == theta[1] + theta[2]
    assert K.diag_value(K.MATERN32, theta, K.D_L) == 0.0
    assert K.diag_value(K.MATERN32, theta, K.D_NUG) == 1.0


def test_nugget_on_index_diagonal_not_on_location():
    # two coincident points stay distinct observations: nugget only on i == j
    x = np.array([[0.2, 0.2], [0.2, 0.2], [0.5, 0.1]])
    S = K.kernel_block(x, x, K.MATERN32, (0.1, 1.0, 0.5), K.SIGMA, 0.0, np.arange(3), np.arange(3))
    assert S[0, 0] == 1.5 and S[0, 1] == 1.0 and S[1, 1] == 1.5


def _bessel_k_integral(nu, x, h=0.02):
    """K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt (DLMF 10.32.9) by the
    trapezoid rule, exponentially convergent for this integrand: a pin of the
    oracle's nu = 1 Matern kernel that shares nothing with its Bessel
    routines."""
    t = np.arange(0.0, np.arccosh(1.0 + 60.0 / x) + h, h)
    f = np.exp(-x * np.cosh(t)) * np.cosh(nu * t)
    return h * (f.sum() - 0.5 * f[0])


def test_matern_nu1_against_the_bessel_integral():
    # Matern nu = 1 (Eq. (matern)): k(r) = x K_1(x), d k / d l = x^2 K_0(x) / l
    # with x = sqrt(2) r / l
    l = 0.07
    for r in (1e-4, 3e-3, 0.02, 0.07, 0.3, 1.1):
        x = np.sqrt(2.0) * r / l
        k_ref = x * _bessel_k_integral(1.0, x)
        dk_ref = x * x * _bessel_k_integral(0.0, x) / l
        assert K.correlation(np.array([r]), K.MATERN1, l)[0] == pytest.approx(k_ref, rel=1e-13)
        assert K.dcorrelation_dl(np.array([r]), K.MATERN1, l)[0] == pytest.approx(dk_ref, rel=1e-13)
