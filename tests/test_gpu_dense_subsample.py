"""The benchmark's clustered workload checked against the dense oracle.

The benchmark runs at n = 262,144, where Sigma cannot be factored densely.
This file takes a 16,384-point subsample (seed 4) of the same point cloud
(uniform + 4 clusters, seed 3), the same kernel and theta (Matern 3/2,
l = 0.05, s2 = 2, nugget 1e-2) and tolerances (eps_fact 1e-9, eps_peel 1e-6),
so the quadtree reaches the clusters' depth, and compares the CUDA path in
both precision forms with the exact dense fp64 values (Oracle-D: Cholesky of
Sigma, Eq. (loglikelihood) and Eq. (gradient)):

* log-likelihood, log|Sigma| and z^T Sigma^-1 z: the acceptance bar 1e-6
  relative at eps_fact = 1e-9;
* each score component g_k: 1e-3 relative (the acceptance bar), and 1e-5 of
  its term scale (|z^T S^-1 S_k S^-1 z| + |Tr(S^-1 S_k)|) / 2, the size of the
  two terms whose difference g_k is (eps_peel = 1e-6 relative error of the
  peeled traces plus the solves).
z is drawn at the true theta through the dense Cholesky factor (seed 5), so
every g_k is about 1% of its term scale and the two bars coincide.
"""
import numpy as np
import pytest

from oracle import dense
from oracle import kernels as K
from paper_1603_08057_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

WL = W.WORKLOADS["matern32_mixture_n262144"]
M = WL["subsample"]


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


@pytest.fixture(scope="module")
def case():
    x_full = W.mixture(WL["n"], WL["seed_points"])
    x, _ = W.subsample(x_full, M, WL["seed_subsample"])
    z = dense.sample_z_dense(x, K.MATERN32, WL["theta"], W.standard_normal(M, WL["seed_z"]))
    d = dense.score_dense(x, z, K.MATERN32, WL["theta"])
    return x, z, d


@pytest.mark.parametrize("prec", [0, 1])
def test_subsample_loglik_and_score_vs_dense(B, case, prec):
    x, z, d = case
    th = WL["theta"]
    o = B.opts(precision=prec)
    ll, g, terms = B.loglik_and_score(T(x), T(z), B.MATERN32, th, WL["tol_fact"], WL["tol_peel"], 0.0, o)
    F = B.Factorization(T(x), B.MATERN32, th, B.SIGMA, WL["tol_fact"], 0.0, o)
    ll2, quad, _ = F.loglik(T(z))
    logdet = F.logdet()
    g = g.numpy()
    scale = 0.5 * np.abs(d["quadk"]) + 0.5 * np.abs(d["trace"])
    err = {"loglik": abs(ll - d["ell"]) / abs(d["ell"]), "logdet": abs(logdet - d["logdet"]) / abs(d["logdet"]),
           "quad": abs(quad - d["quad"]) / abs(d["quad"]),
           "score_rel": np.abs(g - d["g"]) / np.abs(d["g"]), "score_term_scale": np.abs(g - d["g"]) / scale}
    print(f"precision {prec}: {err}")
    assert ll == ll2
    assert err["loglik"] <= 1e-6
    assert err["logdet"] <= 1e-6
    assert err["quad"] <= 1e-6
    assert np.all(err["score_rel"] <= 1e-3)
    assert np.all(err["score_term_scale"] <= 1e-5)
    np.testing.assert_allclose(terms.numpy()[:3], d["quadk"], rtol=1e-6)
    np.testing.assert_allclose(terms.numpy()[3:], d["trace"], rtol=1e-5)


def test_subsample_derivative_factorization_keeps_df64(B, case):
    # In mixed precision the derivative factorization keeps df64 solve factors
    # when a df64 apply agrees with the fp64 apply to 10 tol; either way its
    # apply matches dSigma/dl to the factorization's accuracy.
    x, _, _ = case
    th = WL["theta"]
    Fl = B.Factorization(T(x), B.MATERN32, th, B.D_L, WL["tol_fact"], 0.0, B.opts(precision=1))
    info = Fl.info()
    print(f"derivative factorization: solve_df64 {info['solve_df64']}, probe {info['probe_rel_diff']:.3e}")
    assert 0.0 <= info["probe_rel_diff"]
    assert info["solve_df64"] == (1 if info["probe_rel_diff"] <= 10 * WL["tol_fact"] else 0)
    rows = np.random.default_rng(41).choice(M, 64, replace=False)
    v = W.standard_normal(M, 42)
    got = Fl.solve(T(v), B.OP_APPLY).cpu().numpy()[rows]
    Kr = K.kernel_block(x[rows], x, K.MATERN32, th, K.D_L, ia=rows, ib=np.arange(M))
    ref = Kr @ v
    assert np.all(np.abs(got - ref) <= 1e-7 * (np.abs(Kr) @ np.abs(v)))
