"""Profile log-likelihood (Sec. 5.5, Eq. (prof) and its gradient) and the
conditional distribution (Remark conditional, Sec. 4) through the C ABI,
against the dense oracle (oracle/profile.py).

Bars, as for the plain log-likelihood and score (test_gpu_parity):
* lt, z^T (Sigma + 1 1^T)^-1 z, log|F|, 1^T Sigma^-1 1: 1e-6 relative at
  eps_fact = 1e-9 (the factorization's error amplified by the conditioning);
* the gradient: 1e-3 relative and 1e-5 of its term scale
  |Tr_k|/2 + n |gamma^T Sigma_k gamma| / (2 z^T gamma), since the peeled traces
  carry eps_peel = 1e-6 relative error;
* the conditional mean: 1e-6 of (|Sigma_12| |Sigma_22^-1 z|) per entry -- the
  size of the sum whose cancellation the factorization's relative error
  (~1e-8 of a row's absolute sum, test_gpu_full_size) acts on;
* the conditional covariance from samples with w = I (D D^T, D = samples -
  mean): 1e-6 of s2 + nug, the scale of the joint matrix the factorization
  approximates to eps_fact.
"""
import numpy as np
import pytest

from oracle import dense
from oracle import kernels as K
from oracle import profile as P
from paper_1603_08057_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TH = (0.05, 1.0, 1e-2)


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


def _data(n, seed, fam=K.MATERN32, alpha=0.0, mu=0.7, sd=1.5):
    x = W.mixture(n, seed)
    z = mu + sd * dense.sample_z_dense(x, fam, TH, W.standard_normal(n, seed + 1), alpha)
    return x, z


def _check_profile(lt, g, terms, d, n):
    assert abs(lt - d["lt"]) <= 1e-6 * abs(d["lt"])
    assert abs(terms[6] - d["qt"]) <= 1e-6 * d["qt"]
    assert abs(terms[7] - d["logdet"]) <= 1e-6 * abs(d["logdet"])
    scale = 0.5 * np.abs(d["trace"]) + 0.5 * n * np.abs(d["quadk"]) / d["qt"]
    assert np.all(np.abs(g - d["g"]) <= 1e-3 * np.abs(d["g"]) + 1e-12)
    assert np.all(np.abs(g - d["g"]) <= 1e-5 * scale)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("fam", [K.MATERN32, K.MATERN52])
def test_profile_matches_dense(B, prec, fam):
    n = 3000
    x, z = _data(n, 801, fam)
    lt, g, terms = B.profile_loglik_and_score(T(x), T(z), fam, TH, 1e-9, 1e-6, o=B.opts(precision=prec))
    g, terms = g.numpy(), terms.numpy()
    d = P.profile_score_dense(x, z, fam, TH)
    S = dense.cov_matrix(x, fam, TH)
    ones_b = float(np.sum(np.linalg.solve(S, np.ones(n))))
    print(f"profile fam {fam} prec {prec}: lt {abs(lt - d['lt']) / abs(d['lt']):.2e}, qt "
          f"{abs(terms[6] - d['qt']) / d['qt']:.2e}, 1'S^-1 1 {abs(terms[9] - ones_b) / ones_b:.2e}, "
          f"g rel {np.abs(g - d['g']) / np.abs(d['g'])}")
    assert abs(terms[9] - ones_b) <= 1e-6 * ones_b
    _check_profile(lt, g, terms, d, n)
    # lt alone (no peeling) is the same number
    lt2, g2, _ = B.profile_loglik_and_score(T(x), T(z), fam, TH, 1e-9, 1e-6, o=B.opts(precision=prec),
                                            want_score=False)
    assert g2 is None and lt2 == lt


def test_profile_batched_sets(B):
    sizes = [1200, 2000]
    data = [_data(m, 810 + 3 * i, mu=0.3 * (i + 1)) for i, m in enumerate(sizes)]
    off = np.concatenate([[0], np.cumsum(sizes)])
    P_ = T(np.vstack([d[0] for d in data]))
    Z_ = T(np.concatenate([d[1] for d in data]))
    lt, g, terms = B.profile_loglik_and_score_batched(P_, off, Z_, B.MATERN32, TH)
    for i, (x, z) in enumerate(data):
        d = P.profile_score_dense(x, z, K.MATERN32, TH)
        _check_profile(lt[i], g[i], terms[i], d, sizes[i])


def test_profile_mle_matches_dense_maximizer(B):
    from scipy import optimize
    from paper_1603_08057_gb300 import mle
    n = 1024
    x, z = _data(n, 820)
    th0 = (0.2, 0.1)

    def f(phi):
        th = np.exp(phi)
        d = P.profile_score_dense(x, z, K.MATERN32, (th[0], 1.0, th[1]))
        return -d["lt"] / n, -np.array([d["g"][0], d["g"][2]]) * th / n

    r = optimize.minimize(f, np.log(th0), jac=True, method="L-BFGS-B", options={"maxiter": 100, "gtol": 1e-10})
    th_ref = np.exp(r.x)
    th_gpu, info = mle.fit_profile(T(x), T(z), B.MATERN32, th0, max_iter=30)
    print(f"profile MLE: GPU {th_gpu} ({info['evals']} evaluations, sigma2 {info['sigma2']:.6g}, mu "
          f"{info['mu']:.6g}); dense {th_ref}")
    np.testing.assert_allclose(th_gpu, th_ref, rtol=1e-2)
    S = dense.cov_matrix(x, K.MATERN32, (th_gpu[0], 1.0, th_gpu[1]))
    a = np.linalg.solve(S, z)
    b = np.linalg.solve(S, np.ones(n))
    assert info["mu"] == pytest.approx(np.sum(a) / np.sum(b), rel=1e-5)
    assert info["sigma2"] == pytest.approx(P.profile_loglik_dense(x, z, K.MATERN32, (th_gpu[0], 1.0, th_gpu[1]))[1]
                                           / n, rel=1e-6)


@pytest.mark.parametrize("method", [0, 1])
def test_conditional_mean_matches_dense(B, method):
    n = 3000
    x, z = _data(n, 830, mu=0.0, sd=1.0)
    xs = np.vstack([W.uniform(390, 831) * 1.2 - 0.1, x[:10]])  # beyond the data, and at observed points
    mean, S = B.conditional(T(x), T(z), T(xs), B.MATERN32, TH, 1e-9, method=method)
    assert S is None
    mean = mean.cpu().numpy()
    ref, _ = P.conditional_dense(x, z, xs, K.MATERN32, TH)
    a = np.linalg.solve(dense.cov_matrix(x, K.MATERN32, TH), z)
    scale = np.abs(K.kernel_block(xs, x, K.MATERN32, TH, K.SIGMA)) @ np.abs(a)
    err = np.abs(mean - ref)
    print(f"conditional mean method {method}: max err / scale {np.max(err / scale):.2e}")
    assert np.all(err <= 1e-6 * scale)


def test_conditional_samples_have_conditional_covariance(B):
    n, m = 600, 30
    x, z = _data(n, 840, mu=0.0, sd=1.0)
    xs = W.uniform(m, 841)
    w = np.eye(n + m)
    mean, S = B.conditional(T(x), T(z), T(xs), B.MATERN32, TH, 1e-9, w=T(w))
    D = S.cpu().numpy() - mean.cpu().numpy()[:, None]
    _, cov = P.conditional_dense(x, z, xs, K.MATERN32, TH)
    err = np.max(np.abs(D @ D.T - cov))
    print(f"conditional covariance from samples: max err {err:.2e} (max |cov| {np.max(np.abs(cov)):.3g})")
    assert err <= 1e-6 * (TH[1] + TH[2])
    # samples are linear in w: a random w gives mean + D w
    wr = W.standard_normal(n + m, 842, 3)
    _, S3 = B.conditional(T(x), T(z), T(xs), B.MATERN32, TH, 1e-9, w=T(wr))
    np.testing.assert_allclose(S3.cpu().numpy(), mean.cpu().numpy()[:, None] + D @ wr, atol=1e-9)


def test_conditional_rejects_samples_without_the_joint_factorization(B):
    x, z = _data(200, 850)
    xs = W.uniform(5, 851)
    with pytest.raises(B.RsfError):
        B.conditional(T(x), T(z), T(xs), B.MATERN32, TH, 1e-9, method=B.COND_DIRECT, w=T(np.eye(205)))
