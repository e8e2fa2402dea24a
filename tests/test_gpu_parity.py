"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances (derived from the arithmetic):
* exact identities of the computed factors (F^-1 F = I, F^1/2 F^1/2^T = F):
  rounding only, g kappa(F) u with kappa <~ 1e4 here and a growth g of the
  order of the number of GEMM passes of a solve (about 2 per level, 10-15):
  1e-10 relative in fp64 (u = 2^-53; measured 1.1e-12) and 1e-9 in the
  mixed forms, whose solve operands are df64 pairs (u = 2^-48 = 3.6e-15:
  1e4 x 3.6e-15 x 15 = 5e-10; measured 2.3e-10 on 3,000 uniform points and
  1.0e-10 on 3,000 clustered points with df64 products on the CUDA cores);
* F vs Sigma: the ID tolerance eps_fact = 1e-9 with modest growth -> 1e-8;
* log|F| vs log|Sigma|, log-likelihood vs dense: the acceptance bar 1e-6
  relative at eps_fact = 1e-9;
* score vs the dense exact score: the acceptance bar 1e-3 relative, and
  1e-5 of the term scale (|quad_k| + |trace_k|)/2 since the peeled traces
  carry eps_peel = 1e-6 relative error;
* GPU vs oracle RSF (same algorithm, different pivots by rounding): the
  same bars as against the exact values.
"""
import numpy as np
import pytest

from oracle import dense
from oracle import kernels as K
from oracle import rsf as orsf
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


TH1 = (0.1, 1.0, 1e-2)


@pytest.fixture(scope="module")
def uni(B):
    n = 3000
    x = W.uniform(n, 101)
    F = B.Factorization(T(x), B.MATERN32, TH1, B.SIGMA, 1e-9)
    S = dense.cov_matrix(x, K.MATERN32, TH1)
    return x, F, S


def test_apply_matches_sigma_elementwise(B, uni):
    x, F, S = uni
    V = W.standard_normal(x.shape[0], 7, 5)
    FV = F.solve(T(V), B.OP_APPLY).cpu().numpy()
    ref = S @ V
    assert np.max(np.abs(FV - ref)) <= 1e-8 * np.max(np.abs(ref))


def test_apply_matches_oracle_rsf(B, uni):
    x, F, S = uni
    Fo = orsf.Factorization(x, K.MATERN32, TH1, K.SIGMA, 1e-9)
    v = W.standard_normal(x.shape[0], 8)
    ref = np.empty_like(v)
    ref[Fo.tree.perm] = Fo.apply(v[Fo.tree.perm])
    got = F.solve(T(v), B.OP_APPLY).cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-8 * np.max(np.abs(ref))


def test_solve_inverts_apply(B, uni):
    x, F, S = uni
    V = W.standard_normal(x.shape[0], 9, 3)
    Y = F.solve(F.solve(T(V), B.OP_APPLY), B.OP_INV).cpu().numpy()
    err = np.max(np.abs(Y - V)) / np.max(np.abs(V))
    print(f"F^-1 F V - V: {err:.3e}")
    assert err <= 1e-9      # default (mixed) form


def test_square_root_identities(B, uni):
    x, F, S = uni
    n = x.shape[0]
    E = np.eye(n)[:, ::97]
    FE = F.solve(T(E), B.OP_APPLY)
    SS = F.solve(F.solve(T(E), B.OP_SQRT_T), B.OP_SQRT)
    assert torch.max(torch.abs(SS - FE)).item() <= 1e-11 * torch.max(torch.abs(FE)).item()
    I1 = F.solve(F.solve(T(E), B.OP_INV_SQRT), B.OP_SQRT).cpu().numpy()
    I2 = F.solve(F.solve(T(E), B.OP_SQRT_T), B.OP_INV_SQRT_T).cpu().numpy()
    e1, e2 = np.max(np.abs(I1 - E)), np.max(np.abs(I2 - E))
    print(f"F^1/2 F^-1/2 - I: {e1:.3e}, F^-T/2 F^T/2 - I: {e2:.3e}")
    assert e1 <= 1e-9 and e2 <= 1e-9


def test_logdet_matches_dense(B, uni):
    x, F, S = uni
    ref = np.linalg.slogdet(S)[1]
    assert abs(F.logdet() - ref) <= 1e-9 * abs(ref)


@pytest.mark.parametrize("which", [1, 2])
def test_derivative_factorizations_apply(B, which):
    x = W.mixture(2500, 111)
    th = (0.05, 2.0, 1e-2)
    Fk = B.Factorization(T(x), B.MATERN32, th, which, 1e-9)
    Sk = dense.cov_matrix(x, K.MATERN32, th, which)
    V = W.standard_normal(2500, 112, 4)
    got = Fk.solve(T(V), B.OP_APPLY).cpu().numpy()
    ref = Sk @ V
    assert np.max(np.abs(got - ref)) <= 1e-7 * np.max(np.abs(ref))


def _check_loglik_score(B, x, z, fam, th, alpha=0.0, o=None):
    d = dense.score_dense(x, z, fam, th, alpha)
    ll, g, terms = B.loglik_and_score(T(x), T(z), fam, th, 1e-9, 1e-6, alpha, o)
    assert abs(ll - d["ell"]) <= 1e-6 * abs(d["ell"])
    g = g.numpy()
    assert np.all(np.abs(g - d["g"]) <= 1e-3 * np.abs(d["g"]))
    scale = 0.5 * np.abs(d["quadk"]) + 0.5 * np.abs(d["trace"])
    assert np.all(np.abs(g - d["g"]) <= 1e-5 * scale)
    t = terms.numpy()
    np.testing.assert_allclose(t[:3], d["quadk"], rtol=1e-6)
    np.testing.assert_allclose(t[3:], d["trace"], rtol=1e-5)
    return ll, g


def test_loglik_and_score_matern32_uniform_n4096(B):
    # Matern 3/2, n = 4096 uniform points, l = 0.1, s2 = 1, nugget 1e-2,
    # z from the dense Cholesky factor, eps_fact 1e-9, eps_peel 1e-6
    wl = W.WORKLOADS["matern32_uniform_n4096"]
    x = W.uniform(wl["n"], wl["seed_points"])
    z = dense.sample_z_dense(x, K.MATERN32, wl["theta"], W.standard_normal(wl["n"], wl["seed_z"]))
    _check_loglik_score(B, x, z, K.MATERN32, wl["theta"])


def test_loglik_and_score_rq_mixture(B):
    x = W.mixture(3000, 121)
    th = (0.05, 1.0, 1e-3)
    z = dense.sample_z_dense(x, K.RQ, th, W.standard_normal(3000, 122), 1.0)
    _check_loglik_score(B, x, z, K.RQ, th, 1.0)


def test_sqrt_trace_form_matches_dense(B):
    # the traces peeled on F^-1/2 F_k F^-T/2 and F^-1/2 F^-T/2 (same traces
    # as F^-1 F_k and F^-1) meet the same bars as the paper's symmetrized form
    o = B.opts(trace_form=B.TRACE_SQRT)
    wl = W.WORKLOADS["matern32_uniform_n4096"]
    x = W.uniform(wl["n"], wl["seed_points"])
    z = dense.sample_z_dense(x, K.MATERN32, wl["theta"], W.standard_normal(wl["n"], wl["seed_z"]))
    _check_loglik_score(B, x, z, K.MATERN32, wl["theta"], o=o)
    x = W.mixture(3000, 121)
    th = (0.05, 1.0, 1e-3)
    z = dense.sample_z_dense(x, K.RQ, th, W.standard_normal(3000, 122), 1.0)
    _check_loglik_score(B, x, z, K.RQ, th, 1.0, o=o)


def test_sqrt_trace_form_nugget_identity(B):
    x = W.mixture(3000, 151)
    th = (0.05, 2.0, 1e-2)
    o = B.opts(trace_form=B.TRACE_SQRT)
    F = B.Factorization(T(x), B.MATERN32, th, B.SIGMA, 1e-9)
    Fs = B.Factorization(T(x), B.MATERN32, th, B.D_S2, 1e-9)
    tn = B.peel_trace(F, None, 1e-6, o)
    ts = B.peel_trace(F, Fs, 1e-6, o)
    assert th[1] * ts + th[2] * tn == pytest.approx(3000, rel=1e-6)
    exact = np.trace(np.linalg.inv(dense.cov_matrix(x, K.MATERN32, th)))
    assert abs(tn - exact) <= 1e-6 * abs(exact)


@pytest.mark.parametrize("fam", [K.MATERN12, K.MATERN52, K.MATERN1])
def test_loglik_other_matern(B, fam):
    x = W.uniform(1500, 131)
    th = (0.08, 1.5, 5e-3)
    z = dense.sample_z_dense(x, fam, th, W.standard_normal(1500, 132))
    _check_loglik_score(B, x, z, fam, th)


def test_peeled_traces_match_oracle_peeling(B):
    from oracle import peel
    x = W.mixture(2000, 141)
    th = (0.05, 2.0, 1e-2)
    F = B.Factorization(T(x), B.MATERN32, th, B.SIGMA, 1e-9)
    Fo = orsf.Factorization(x, K.MATERN32, th, K.SIGMA, 1e-9)
    t_gpu = B.peel_trace(F, None, 1e-6)
    t_or, _ = peel.peel_trace(Fo.solve, Fo.tree, 1e-6)
    exact = np.trace(np.linalg.inv(dense.cov_matrix(x, K.MATERN32, th)))
    assert abs(t_gpu - exact) <= 1e-6 * abs(exact)
    assert abs(t_gpu - t_or) <= 1e-6 * abs(exact)


def test_variance_nugget_trace_identity(B):
    # Sigma = s2 Sigma_s2 + nug I  =>  s2 Tr(S^-1 S_s2) + nug Tr(S^-1) = n
    x = W.mixture(3000, 151)
    th = (0.05, 2.0, 1e-2)
    F = B.Factorization(T(x), B.MATERN32, th, B.SIGMA, 1e-9)
    Fs = B.Factorization(T(x), B.MATERN32, th, B.D_S2, 1e-9)
    tn = B.peel_trace(F, None, 1e-6)
    ts = B.peel_trace(F, Fs, 1e-6)
    assert th[1] * ts + th[2] * tn == pytest.approx(3000, rel=1e-6)


@pytest.mark.parametrize("n", [1, 2, 64, 65, 200])
def test_small_and_ragged_sizes(B, n):
    x = W.uniform(n, 161)
    th = (0.2, 1.0, 1e-1)
    z = dense.sample_z_dense(x, K.MATERN32, th, W.standard_normal(n, 162))
    d = dense.score_dense(x, z, K.MATERN32, th)
    ll, g, _ = B.loglik_and_score(T(x), T(z), B.MATERN32, th)
    assert abs(ll - d["ell"]) <= 1e-8 * max(1.0, abs(d["ell"]))
    scale = 0.5 * np.abs(d["quadk"]) + 0.5 * np.abs(d["trace"])
    assert np.all(np.abs(g.numpy() - d["g"]) <= 1e-6 * scale + 1e-12)


def test_coincident_and_collinear_points(B):
    x = W.uniform(700, 171)
    x[350:400] = x[0]            # 51 copies of one location (nugget keeps them apart)
    x[400:600, 1] = 0.5          # a line of points
    th = (0.1, 1.0, 5e-2)
    z = dense.sample_z_dense(x, K.MATERN32, th, W.standard_normal(700, 172))
    _check_loglik_score(B, x, z, K.MATERN32, th)


def test_autograd_backward_is_the_score(B):
    x = W.uniform(1200, 181)
    th = (0.1, 1.0, 1e-2)
    z = dense.sample_z_dense(x, K.MATERN32, th, W.standard_normal(1200, 182))
    d = dense.score_dense(x, z, K.MATERN32, th)
    theta = torch.tensor(th, dtype=torch.float64, requires_grad=True)
    ll = B.gp_loglik(theta, T(x), T(z), B.MATERN32)
    ll.backward()
    assert ll.item() == pytest.approx(d["ell"], rel=1e-6)
    np.testing.assert_allclose(theta.grad.numpy(), d["g"], rtol=1e-3)


def test_deterministic(B):
    x = W.mixture(2000, 191)
    z = W.standard_normal(2000, 192)
    th = (0.05, 2.0, 1e-2)
    a = B.loglik_and_score(T(x), T(z), B.MATERN32, th)
    b = B.loglik_and_score(T(x), T(z), B.MATERN32, th)
    assert a[0] == b[0] and torch.equal(a[1], b[1])


def test_invalid_arguments_raise(B):
    x = T(W.uniform(100, 1))
    with pytest.raises(B.RsfError) as e:
        B.Factorization(x, B.MATERN32, (0.1, 1.0, 1e-2), B.SIGMA, 0.0)
    assert e.value.code == 1
    with pytest.raises(B.RsfError):
        B.Factorization(x, 17, (0.1, 1.0, 1e-2))
    with pytest.raises(B.RsfError):
        B.Factorization(x, B.MATERN32, (-0.1, 1.0, 1e-2))
    bad = W.uniform(100, 1)
    bad[3, 0] = np.nan
    with pytest.raises(B.RsfError):
        B.Factorization(T(bad), B.MATERN32, (0.1, 1.0, 1e-2))
    Fl = B.Factorization(x, B.MATERN32, (0.1, 1.0, 1e-2), B.D_L)
    with pytest.raises(B.RsfError):
        Fl.logdet()
    with pytest.raises(B.RsfError):
        Fl.solve(T(np.ones(100)), B.OP_INV)
    with pytest.raises(B.RsfError) as e:
        B.Factorization(x, B.MATERN32, (0.1, 1.0, 1e-2), B.SIGMA, 1e-9, 0.0, B.opts(trace_form=7))
    assert e.value.code == 1


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_precision_modes_match_dense(B, prec):
    # plain fp64 (0) and the mixed forms (df64 operands; products on the
    # tensor cores (1) or the CUDA cores (2)) all meet the bars
    x = W.mixture(3000, 201)
    th = (0.05, 2.0, 1e-2)
    z = dense.sample_z_dense(x, K.MATERN32, th, W.standard_normal(3000, 202))
    o = B.opts(precision=prec)
    d = dense.score_dense(x, z, K.MATERN32, th)
    ll, g, terms = B.loglik_and_score(T(x), T(z), B.MATERN32, th, 1e-9, 1e-6, 0.0, o)
    assert abs(ll - d["ell"]) <= 1e-6 * abs(d["ell"])
    scale = 0.5 * np.abs(d["quadk"]) + 0.5 * np.abs(d["trace"])
    assert np.all(np.abs(g.numpy() - d["g"]) <= 1e-5 * scale)
    F = B.Factorization(T(x), B.MATERN32, th, B.SIGMA, 1e-9, 0.0, o)
    V = W.standard_normal(3000, 203, 4)
    Y = F.solve(F.solve(T(V), B.OP_APPLY), B.OP_INV).cpu().numpy()
    err = np.max(np.abs(Y - V)) / np.max(np.abs(V))
    print(f"precision {prec}: F^-1 F V - V: {err:.3e}")
    assert err <= (1e-10 if prec == 0 else 1e-9)


def test_mixed_close_to_fp64(B):
    x = W.uniform(2500, 211)
    th = (0.1, 1.0, 1e-2)
    F0 = B.Factorization(T(x), B.MATERN32, th, B.SIGMA, 1e-9, 0.0, B.opts(precision=0))
    V = T(W.standard_normal(2500, 212, 3))
    for prec in (1, 2):
        F1 = B.Factorization(T(x), B.MATERN32, th, B.SIGMA, 1e-9, 0.0, B.opts(precision=prec))
        for op in (B.OP_INV, B.OP_APPLY, B.OP_SQRT, B.OP_INV_SQRT_T):
            a, b = F0.solve(V, op), F1.solve(V, op)
            err = torch.max(torch.abs(a - b)).item() / torch.max(torch.abs(a)).item()
            print(f"precision {prec} op {op}: mixed vs fp64 {err:.3e}")
            assert err <= 1e-10
        assert F0.logdet() == F1.logdet()
