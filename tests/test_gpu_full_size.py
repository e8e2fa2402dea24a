"""Parity at the benchmark's full size, through the C-ABI calls bench.py times.

Workload: n = 262,144 clustered points (uniform + 4 clusters), Matern 3/2,
theta = (l, s2, nug) = (0.05, 2, 1e-2), eps_fact = 1e-9, eps_peel = 1e-6, the
default (mixed-precision) options.  The oracle cannot factor or invert Sigma
at this size, so the checks are

* sampled outputs the oracle computes one by one: rows of Sigma x, summed
  directly from the kernel (Sec. 2: F approximates Sigma to eps_fact);
* properties that hold at any size:
  - F^-1 (F x) = x (Sec. 2.3.2: the solve inverts the factored form exactly,
    up to rounding),
  - d log|Sigma| / d theta_k = Tr(Sigma^-1 Sigma_k) (Sec. 1, the identity
    behind Eq. (gradient)), checked by central differences of RSF
    log-determinants against the peeled traces of the score for the length
    scale, the variance and the nugget,
  - n / (s2 + nug) <= Tr(Sigma^-1) <= n / nug (Sigma >= nug I and
    Tr(Sigma) = n (s2 + nug)),
  - s2 g_s2 + nug g_nug = (z^T Sigma^-1 z - n) / 2 (Sigma = s2 Sigma_s2 + nug I).

and, for the score itself, central differences of the log-likelihood of
tight (eps_fact = 1e-12) fp64 factorizations (Eq. (gradient)).

Tolerances: the applied rows carry the ID error, <= 1e-8 of the row's
absolute sum sum_j |K_ij x_j| (eps_fact = 1e-9 per level, amplified through
the levels; measured 1.4e-10 on GB300); F^-1 F x = x to 1e-6 of max |x|
(df64 solves, ~48-bit significands, times the conditioning of the factors;
measured 1.0e-8); the central differences use h = 1e-3 relative steps and
must match the peeled traces to 1e-5 (eps_peel = 1e-6 plus the O(h^2)
truncation and the log-determinant errors; measured at most 1.1e-6).
"""
import math

import numpy as np
import pytest

from oracle import kernels as K
from paper_1603_08057_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

WL = W.WORKLOADS["matern32_mixture_n262144"]


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_08057_gb300 import build
    build.build()
    from paper_1603_08057_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def pts():
    return W.mixture(WL["n"], WL["seed_points"])


def T(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def test_full_size_apply_rows_and_solve(B, pts):
    n = WL["n"]
    th = WL["theta"]
    F = B.Factorization(T(pts), B.MATERN32, th, B.SIGMA, WL["tol_fact"])
    x = W.standard_normal(n, 901)
    y = F.solve(T(x), B.OP_APPLY).cpu().numpy()
    rows = np.random.default_rng(902).choice(n, 48, replace=False)
    Krows = K.kernel_block(pts[rows], pts, K.MATERN32, th, K.SIGMA, ia=rows, ib=np.arange(n))
    ref = Krows @ x
    scale = np.abs(Krows) @ np.abs(x)
    assert np.all(np.abs(y[rows] - ref) <= 1e-8 * scale)
    back = F.solve(T(y), B.OP_INV).cpu().numpy()
    assert np.max(np.abs(back - x)) <= 1e-6 * np.max(np.abs(x))


def test_full_size_score_traces_match_logdet_derivatives(B, pts):
    n = WL["n"]
    th = WL["theta"]
    tf = WL["tol_fact"]
    P = T(pts)
    z = W.standard_normal(n, 903)
    ll, g, terms = B.loglik_and_score(P, T(z), B.MATERN32, th, tf, WL["tol_peel"])
    g = g.numpy()
    t = terms.numpy()           # [quad_l, quad_s2, quad_nug, tr_l, tr_s2, tr_nug]
    tr_l, tr_s2, tr_nug = t[3], t[4], t[5]
    l, s2, nug = th

    assert n / (s2 + nug) <= tr_nug <= n / nug

    F = B.Factorization(P, B.MATERN32, th, B.SIGMA, tf)
    logdet = F.logdet()
    del F
    quad = -2.0 * (ll + 0.5 * logdet + 0.5 * n * math.log(2.0 * math.pi))
    assert s2 * g[1] + nug * g[2] == pytest.approx(0.5 * (quad - n), rel=1e-9, abs=1e-6 * n)

    def logdet_at(theta):
        Fh = B.Factorization(P, B.MATERN32, theta, B.SIGMA, tf)
        v = Fh.logdet()
        del Fh
        return v

    h = 1e-3
    for k, tr in ((0, tr_l), (1, tr_s2), (2, tr_nug)):
        step = h * th[k]
        up = list(th)
        dn = list(th)
        up[k] += step
        dn[k] -= step
        fd = (logdet_at(tuple(up)) - logdet_at(tuple(dn))) / (2.0 * step)
        assert fd == pytest.approx(tr, rel=1e-5), (k, fd, tr)


def test_full_size_score_vs_loglik_differences(B, pts):
    # Eq. (gradient): g_k = d loglik / d theta_k.  Reference: central
    # differences of the RSF log-likelihood at eps_fact = 1e-12 in plain fp64,
    # Richardson-extrapolated from the steps h = 1e-3 theta_k and h / 2 (the
    # O(h^2) term of a single difference is not small here: the score
    # components are small differences of terms of size ~n, and so is the
    # third derivative, which put a plain h = 1e-3 difference ~0.4 off g_l).
    # The extrapolated reference carries the log-likelihood's rounding and
    # rank-decision noise (~1e-6 absolute at eps_fact = 1e-12) divided by the
    # step, ~0.02.  The score under test is the benchmark's configuration
    # (mixed precision, eps_fact 1e-9, eps_peel 1e-6) at theta of one
    # benchmark step (l * 1.005); z = F^1/2 w drawn at the workload's theta.
    # Bars: 1e-3 relative per component, and 1e-6 of the term scale
    # (|quad_k| + |trace_k|) / 2.
    n = WL["n"]
    th0 = WL["theta"]
    P = T(pts)
    o64 = B.opts(precision=0)
    F = B.Factorization(P, B.MATERN32, th0, B.SIGMA, 1e-12, 0.0, o64)
    z = F.solve(T(W.standard_normal(n, WL["seed_z"])), B.OP_SQRT)
    del F
    th = (th0[0] * 1.005, th0[1], th0[2])
    ll, g, terms = B.loglik_and_score(P, z, B.MATERN32, th, WL["tol_fact"], WL["tol_peel"])
    g, t = g.numpy(), terms.numpy()

    def loglik_at(theta):
        Fh = B.Factorization(P, B.MATERN32, theta, B.SIGMA, 1e-12, 0.0, o64)
        v = Fh.loglik(z)[0]
        del Fh
        return v

    def central(k, h):
        up, dn = list(th), list(th)
        up[k] += h * th[k]
        dn[k] -= h * th[k]
        return (loglik_at(tuple(up)) - loglik_at(tuple(dn))) / (2.0 * h * th[k])

    fd = np.zeros(3)
    for k in range(3):
        fd[k] = (4.0 * central(k, 5e-4) - central(k, 1e-3)) / 3.0
    scale = 0.5 * np.abs(t[:3]) + 0.5 * np.abs(t[3:])
    print(f"full size score {g} vs loglik differences {fd}: rel {np.abs(g - fd) / np.abs(fd)}, "
          f"term scale {np.abs(g - fd) / scale}")
    assert np.all(np.abs(g - fd) <= 1e-6 * scale)
    assert np.all(np.abs(g - fd) <= 1e-3 * np.abs(fd))
