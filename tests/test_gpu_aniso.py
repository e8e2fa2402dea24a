"""The anisotropic kernels of Sec. 5.1 (scaled distance ||x - y||_theta,
theta = [l1, l2], Eqs. (specrq) and (specmatern)) through the C ABI, on the
paper's regular grid of [0, 100]^2, against the dense oracle.

Bars as in test_gpu_parity: F and F_k against Sigma and dSigma/dl_k 1e-8 of
a row's absolute sum (eps_fact = 1e-9); log-likelihood 1e-6 relative; the
four score components 1e-3 relative and 1e-5 of their term scale (the peeled
traces carry eps_peel = 1e-6).
"""
import numpy as np
import pytest

from oracle import dense
from oracle import kernels as K
from paper_1603_08057_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TH = (10.0, 1.0, 1e-2, 7.0)


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


@pytest.mark.parametrize("which", [K.SIGMA, K.D_L, K.D_L2])
def test_aniso_apply_matches_dense_elementwise(B, which):
    x = W.grid(48, 0.0, 100.0)
    n = len(x)
    F = B.Factorization(T(x), B.MATERN32, TH, which, 1e-9)
    v = W.standard_normal(n, 901)
    y = F.solve(T(v), B.OP_APPLY).cpu().numpy()
    S = dense.cov_matrix(x, K.MATERN32, TH, which)
    err = np.abs(y - S @ v)
    print(f"aniso apply which {which}: max err / row scale {np.max(err / (np.abs(S) @ np.abs(v))):.2e}")
    assert np.all(err <= 1e-8 * (np.abs(S) @ np.abs(v)))


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("fam,alpha", [(K.MATERN32, 0.0), (K.RQ, 0.5)])
def test_aniso_loglik_and_score_match_dense(B, prec, fam, alpha):
    x = W.grid(48, 0.0, 100.0)
    n = len(x)
    z = dense.sample_z_dense(x, fam, TH, W.standard_normal(n, 902), alpha)
    ll, g, terms = B.loglik_and_score(T(x), T(z), fam, TH, 1e-9, 1e-6, alpha, B.opts(precision=prec))
    g, terms = g.numpy(), terms.numpy()
    d = dense.score_dense(x, z, fam, TH, alpha)
    scale = 0.5 * np.abs(d["quadk"]) + 0.5 * np.abs(d["trace"])
    print(f"aniso fam {fam} prec {prec}: loglik {abs(ll - d['ell']) / abs(d['ell']):.2e}, "
          f"score rel {np.abs(g - d['g']) / np.abs(d['g'])}, traces rel {np.abs(terms[4:] - d['trace']) / np.abs(d['trace'])}")
    assert g.shape == (4,) and terms.shape == (8,)
    assert abs(ll - d["ell"]) <= 1e-6 * abs(d["ell"])
    assert np.all(np.abs(g - d["g"]) <= 1e-3 * np.abs(d["g"]))
    assert np.all(np.abs(g - d["g"]) <= 1e-5 * scale)


def test_aniso_peeled_trace_of_the_paper_operator(B):
    # Tables peelingresults_*: the trace of G = (Sigma^-1 Sigma_1 + Sigma_1 Sigma^-1)/2
    # with Sigma_1 = dSigma/dtheta_1, peeled at eps_peel = 1e-6, nugget 1e-4
    th = (10.0, 1.0, 1e-4, 7.0)
    x = W.grid(48, 0.0, 100.0)
    for fam, alpha in ((B.MATERN32, 0.0), (B.RQ, 0.5)):
        F = B.Factorization(T(x), fam, th, B.SIGMA, 1e-9, alpha)
        F1 = B.Factorization(T(x), fam, th, B.D_L, 1e-9, alpha)
        t = B.peel_trace(F, F1, 1e-6)
        S = dense.cov_matrix(x, fam, th, K.SIGMA, alpha)
        S1 = dense.cov_matrix(x, fam, th, K.D_L, alpha)
        exact = np.trace(np.linalg.solve(S, S1))
        e = abs(t - exact) / abs(exact)
        print(f"peeled Tr(G_1) family {fam}: {t:.10g} vs {exact:.10g}, e_peel {e:.2e}")
        assert e <= 1e-4


def test_equal_length_scales_match_the_isotropic_kernel(B):
    x = W.mixture(3000, 903)
    th_iso = (0.05, 1.0, 1e-2)
    th_an = (0.05, 1.0, 1e-2, 0.05)
    z = dense.sample_z_dense(x, K.MATERN32, th_iso, W.standard_normal(3000, 904))
    ll0, g0, _ = B.loglik_and_score(T(x), T(z), B.MATERN32, th_iso)
    ll1, g1, _ = B.loglik_and_score(T(x), T(z), B.MATERN32, th_an)
    g0, g1 = g0.numpy(), g1.numpy()
    # the same matrix up to the rounding of the distance (r/l against |(dx/l, dy/l)|)
    assert abs(ll1 - ll0) <= 1e-8 * abs(ll0)
    np.testing.assert_allclose(g1[1:3], g0[1:3], rtol=1e-5)
    assert abs((g1[0] + g1[3]) - g0[0]) <= 1e-3 * abs(g0[0])
