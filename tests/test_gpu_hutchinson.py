"""Hutchinson's trace estimator as the cheap GPU trace mode (Sec. 3,
Eq. (hutch)), through the C ABI (rsf_peel_trace with trace_form =
RSF_TRACE_HUTCH).

The GPU draws the same Rademacher probes as the oracle (the sign of Philox
stream 1's normal at (tree position, probe), key = seed), so its estimate of
Tr(Sigma^-1) and of Tr(Sigma^-1 Sigma_l) must equal the oracle's estimate with
the dense exact operators in tree order, up to F versus Sigma (eps_fact =
1e-9, ~1e-7 relative in these quadratic forms) -- bar 1e-6 relative.  Both
estimates must lie within 5 standard errors of the exact traces, and a
forest's per-set estimates must add up to the single estimate over the same
probes.
"""
import numpy as np
import pytest

from oracle import dense
from oracle import kernels as K
from oracle import peel as opeel
from oracle.tree import Tree
from paper_1603_08057_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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


def test_hutchinson_matches_oracle_estimate_and_exact_traces(B):
    n, q, seed = 3000, 256, 7
    th = (0.05, 2.0, 1e-2)
    x = W.mixture(n, 701)
    o = B.opts(trace_form=B.TRACE_HUTCH, probes=q, seed=seed)
    F = B.Factorization(T(x), B.MATERN32, th, B.SIGMA, 1e-9)
    Fl = B.Factorization(T(x), B.MATERN32, th, B.D_L, 1e-9)
    t0 = B.peel_trace(F, None, 1e-6, o)
    t1 = B.peel_trace(F, Fl, 1e-6, o)

    perm = Tree(x, 64).perm
    S = dense.cov_matrix(x, K.MATERN32, th)[np.ix_(perm, perm)]
    Sl = dense.cov_matrix(x, K.MATERN32, th, K.D_L)[np.ix_(perm, perm)]
    Sinv = np.linalg.inv(S)
    G1 = 0.5 * (Sinv @ Sl + Sl @ Sinv)
    e0, se0 = opeel.hutchinson(lambda U: Sinv @ U, n, q, seed)
    e1, se1 = opeel.hutchinson(lambda U: G1 @ U, n, q, seed)
    x0, x1 = np.trace(Sinv), np.trace(G1)
    print(f"Hutchinson q={q}: GPU {t0:.8g}, {t1:.8g}; oracle {e0:.8g} (se {se0:.3g}), {e1:.8g} (se {se1:.3g}); "
          f"exact {x0:.8g}, {x1:.8g}")
    assert t0 == pytest.approx(e0, rel=1e-6)
    assert t1 == pytest.approx(e1, rel=1e-6)
    assert abs(e0 - x0) <= 5 * se0 and abs(e1 - x1) <= 5 * se1


def test_hutchinson_in_a_forest(B):
    sizes = [1200, 2000]
    th = (0.05, 2.0, 1e-2)
    xs = [W.mixture(m, 710 + i) for i, m in enumerate(sizes)]
    off = np.concatenate([[0], np.cumsum(sizes)])
    o = B.opts(trace_form=B.TRACE_HUTCH, probes=128, seed=3)
    P = T(np.vstack(xs))
    z = T(W.standard_normal(int(off[-1]), 711))
    _, g, terms = B.loglik_and_score_batched(P, off, z, B.MATERN32, th, o=o)
    F = B.Factorization(P, B.MATERN32, th, B.SIGMA, 1e-9, 0.0, o, offsets=off)
    total = B.peel_trace(F, None, 1e-6, o)
    # per-set Tr(Sigma_i^-1) estimates (terms[:, 5]) add up to the whole-forest estimate
    assert np.sum(terms[:, 5]) == pytest.approx(total, rel=1e-9)
    for i, x in enumerate(xs):
        exact = np.trace(np.linalg.inv(dense.cov_matrix(x, K.MATERN32, th)))
        assert abs(terms[i, 5] - exact) <= 0.05 * exact
