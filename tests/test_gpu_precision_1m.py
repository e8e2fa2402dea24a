"""The precision workload: n = 1,048,576 uniform points, rational quadratic
alpha = 2, l = 0.02, s2 = 1, nugget 1e-2, eps_fact 1e-9.

z is F^1/2 w of the plain fp64 GPU factorization at eps_fact = 1e-12
(Sec. 2.3.2), w ~ N(0, I) (seed 8).  Checked:

* the mixed form (df64 operands, tensor-core products) against the plain
  fp64 form on the same points, theta and z, both without refinement:
  log|F| identical (both forms factor in fp64), z^T F^-1 z and the
  log-likelihood within 1e-10 relative (the products' rounding, ~1e-14,
  times the conditioning; measured 2.1e-15 and 3.6e-15 with the CUDA-core
  df64 products);
* the refined quadratic form (one sweep against the exact Sigma, df64
  residual) differs from the unrefined one by at most 1e-6 relative (the
  factorization's error; measured 7e-9 against the fp64 form);
* both forms against the dense oracle on a 16,384-point subsample (seed 9)
  of the same points: log-likelihood 1e-6 relative, score 1e-3 relative and
  1e-5 of the term scale;
* at full size, sampled rows of Sigma x summed one by one by the oracle's
  kernel (1e-8 of the row's absolute sum).
"""
import numpy as np
import pytest

from oracle import dense
from oracle import kernels as K
from paper_1603_08057_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

WL = W.WORKLOADS["rq2_uniform_n1048576"]


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
def pts():
    return W.uniform(WL["n"], WL["seed_points"])


def test_1m_mixed_vs_fp64_and_sampled_rows(B, pts):
    n, th, a = WL["n"], WL["theta"], WL["alpha"]
    P = T(pts)
    F12 = B.Factorization(P, B.RQ, th, B.SIGMA, 1e-12, a, B.opts(precision=0))
    z = F12.solve(T(W.standard_normal(n, WL["seed_z"])), B.OP_SQRT)
    del F12
    out = {}
    for prec, refine in ((0, 0), (1, 0), (1, 1)):
        F = B.Factorization(P, B.RQ, th, B.SIGMA, WL["tol_fact"], a, B.opts(precision=prec, refine=refine))
        ll, quad, _ = F.loglik(z)
        out[(prec, refine)] = (ll, quad, F.logdet())
        if prec == 1 and refine == 0:
            x = W.standard_normal(n, 10)
            y = F.solve(T(x), B.OP_APPLY).cpu().numpy()
            rows = np.random.default_rng(11).choice(n, 32, replace=False)
            Kr = K.kernel_block(pts[rows], pts, K.RQ, th, K.SIGMA, a, ia=rows, ib=np.arange(n))
            assert np.all(np.abs(y[rows] - Kr @ x) <= 1e-8 * (np.abs(Kr) @ np.abs(x)))
        del F
    (ll0, q0, ld0), (ll1, q1, ld1), (ll2, q2, ld2) = out[(0, 0)], out[(1, 0)], out[(1, 1)]
    print(f"n=1048576 RQ: loglik fp64 {ll0!r} mixed {ll1!r} mixed+refinement {ll2!r}; mixed vs fp64: loglik "
          f"{abs(ll1 - ll0) / abs(ll0):.3e}, quad {abs(q1 - q0) / abs(q0):.3e}, logdet {abs(ld1 - ld0) / abs(ld0):.3e}; "
          f"refinement moved quad by {abs(q2 - q1) / abs(q1):.3e}")
    # the same factorization and solve in both forms: df64 rounding only
    assert ld0 == ld1 == ld2
    assert abs(q1 - q0) <= 1e-10 * abs(q0)
    assert abs(ll1 - ll0) <= 1e-10 * abs(ll0)
    # the refinement corrects z^T F^-1 z toward z^T Sigma^-1 z by about the
    # factorization's error (eps_fact = 1e-9 amplified by the conditioning)
    assert abs(q2 - q1) <= 1e-6 * abs(q1)


@pytest.mark.parametrize("prec", [0, 1])
def test_1m_subsample_vs_dense(B, pts, prec):
    th, a = WL["theta"], WL["alpha"]
    m = 16384
    x, _ = W.subsample(pts, m, 9)
    z = dense.sample_z_dense(x, K.RQ, th, W.standard_normal(m, 12), a)
    d = _dense(x, z)
    ll, g, _ = B.loglik_and_score(T(x), T(z), B.RQ, th, WL["tol_fact"], WL["tol_peel"], a, B.opts(precision=prec))
    g = g.numpy()
    scale = 0.5 * np.abs(d["quadk"]) + 0.5 * np.abs(d["trace"])
    print(f"RQ subsample precision {prec}: loglik {abs(ll - d['ell']) / abs(d['ell']):.3e}, "
          f"score rel {np.abs(g - d['g']) / np.abs(d['g'])}, term scale {np.abs(g - d['g']) / scale}")
    assert abs(ll - d["ell"]) <= 1e-6 * abs(d["ell"])
    assert np.all(np.abs(g - d["g"]) <= 1e-3 * np.abs(d["g"]))
    assert np.all(np.abs(g - d["g"]) <= 1e-5 * scale)


_cache = {}


def _dense(x, z):
    key = (x.shape[0], float(x[0, 0]))
    if key not in _cache:
        _cache[key] = dense.score_dense(x, z, K.RQ, WL["theta"], WL["alpha"])
    return _cache[key]
