"""Pins of Oracle-R, the CPU recursive skeletonization factorization
(Sec. 2): exact algebraic identities of the computed factors, the ID error
contract (Def. ID) against all complement rows, the approximation error
O(eps) (Thm. 1) and convergence to the dense Cholesky result as eps -> 0."""
import numpy as np
import pytest

from oracle import dense, rsf
from oracle import kernels as K
from paper_1603_08057_gb300 import workloads as W

TH = (0.1, 1.0, 1e-2)


@pytest.fixture(scope="module")
def fac():
    x = W.uniform(1500, 21)
    F = rsf.Factorization(x, K.MATERN32, TH, K.SIGMA, 1e-9)
    S = dense.cov_matrix(F.tree.xt, K.MATERN32, TH)
    return x, F, S


def test_solve_inverts_apply(fac):
    _, F, _ = fac
    v = W.standard_normal(F.n, 1, 3)
    np.testing.assert_allclose(F.solve(F.apply(v)), v, rtol=0, atol=1e-10 * np.abs(v).max())


def test_sqrt_factors(fac):
    _, F, _ = fac
    Fd = F.dense()
    Sq = F.sqrt(np.eye(F.n))
    assert np.max(np.abs(Sq @ Sq.T - Fd)) <= 1e-12 * np.max(np.abs(Fd))
    np.testing.assert_allclose(F.sqrt_t(np.eye(F.n)), Sq.T, atol=1e-13)
    np.testing.assert_allclose(F.inv_sqrt(Sq), np.eye(F.n), atol=1e-9)
    np.testing.assert_allclose(F.inv_sqrt_t(F.sqrt_t(np.eye(F.n))), np.eye(F.n), atol=1e-9)


def test_logdet_is_slogdet_of_factor(fac):
    _, F, _ = fac
    sign, ld = np.linalg.slogdet(F.dense())
    assert sign > 0 and F.logdet() == pytest.approx(ld, rel=1e-12)


def test_factor_is_symmetric(fac):
    _, F, _ = fac
    Fd = F.dense()
    assert np.max(np.abs(Fd - Fd.T)) <= 1e-13 * np.max(np.abs(Fd))


def test_apply_error_is_order_eps(fac):
    _, F, S = fac
    err = np.linalg.norm(F.dense() - S, 2) / np.linalg.norm(S, 2)
    assert 1e-13 < err < 1e-8


def test_id_error_against_all_complement_rows(fac):
    # Def. ID with the full active complement, not only the proxy rows:
    # validates the modified proxy trick of Sec. 2.3.1
    _, F, S = fac
    worst = 0.0
    for lev, recs in F.records.items():
        for r in recs:
            if r.R.size == 0:
                continue
            Ic = np.setdiff1d(F.active[lev], r.I)
            A = S[np.ix_(Ic, r.I)]
            e = np.linalg.norm(S[np.ix_(Ic, r.R)] - S[np.ix_(Ic, r.S)] @ r.T, 2) / np.linalg.norm(A, 2)
            worst = max(worst, e)
    assert worst <= 10 * 1e-9


def test_tolerance_to_zero_recovers_dense_loglik():
    x = W.uniform(1200, 31)
    z = dense.sample_z_dense(x, K.MATERN32, TH, W.standard_normal(1200, 32))
    ell_d, quad_d, ld_d = dense.loglik_dense(x, z, K.MATERN32, TH)
    F = rsf.Factorization(x, K.MATERN32, TH, K.SIGMA, 1e-15)
    zt = z[F.tree.perm]
    assert F.logdet() == pytest.approx(ld_d, rel=1e-11)
    assert float(zt @ F.solve(zt)) == pytest.approx(quad_d, rel=1e-9)
    F9 = rsf.Factorization(x, K.MATERN32, TH, K.SIGMA, 1e-9, tree=F.tree)
    ell9 = -0.5 * float(zt @ F9.solve(zt)) - 0.5 * F9.logdet() - 0.5 * 1200 * np.log(2 * np.pi)
    assert abs(ell9 - ell_d) <= 1e-6 * abs(ell_d)


@pytest.mark.parametrize("fam,alpha,which", [(K.MATERN32, 0.0, K.D_L), (K.RQ, 1.0, K.D_L), (K.RQ, 1.0, K.SIGMA), (K.MATERN32, 0.0, K.D_S2)])
def test_other_kernels_and_derivative_factorizations(fam, alpha, which):
    x = W.mixture(1500, 41)
    th = (0.05, 2.0, 1e-2)
    F = rsf.Factorization(x, fam, th, which, 1e-9, alpha)
    S = dense.cov_matrix(F.tree.xt, fam, th, which, alpha)
    v = W.standard_normal(F.n, 42)
    err = np.linalg.norm(F.apply(v) - S @ v) / np.linalg.norm(S @ v)
    assert err < 1e-7
    if which == K.SIGMA:
        assert F.logdet() == pytest.approx(np.linalg.slogdet(S)[1], rel=1e-7)


def test_tiny_problem_is_dense_root():
    x = W.uniform(50, 3)
    F = rsf.Factorization(x, K.MATERN32, TH, K.SIGMA, 1e-9)
    S = dense.cov_matrix(F.tree.xt, K.MATERN32, TH)
    assert F.tree.L == 0
    np.testing.assert_allclose(F.dense(), S, rtol=1e-13, atol=1e-14)
