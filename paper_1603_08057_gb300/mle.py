"""Maximum-likelihood estimation of theta = (l, s2, nug) (the MLE runs of
Sec. 5.4) with L-BFGS over log theta, driving the differentiable
log-likelihood of the binding (GPLogLikelihood: forward = RSF log-likelihood,
backward = the score from the peeled traces, Algorithm 1).

Host-side driver only: every evaluation is one call of the C-ABI library
(factorization, solves, peeling and score run in its CUDA kernels); the
optimizer's vectors have three entries.
"""
from __future__ import annotations

import math
import time

import torch

from . import binding as B


def fit(points: torch.Tensor, z: torch.Tensor, family: int, theta0, alpha: float = 0.0, tol_fact: float = 1e-9,
        tol_peel: float = 1e-6, o: B.RsfOpts | None = None, max_iter: int = 30, history_size: int = 10):
    """Maximizes the log-likelihood from theta0; returns (theta, info) with
    info = {"evals", "seconds", "loglik", "trace": [(theta, loglik, score)]}.
    The objective is -loglik / n in the variables log theta (positivity and
    scale balance), minimized by torch's L-BFGS with a strong-Wolfe line
    search for at most max_iter iterations."""
    n = points.shape[0]
    phi = torch.tensor([math.log(float(v)) for v in theta0], dtype=torch.float64, requires_grad=True)
    opt = torch.optim.LBFGS([phi], lr=1.0, max_iter=max_iter, history_size=history_size,
                            line_search_fn="strong_wolfe", tolerance_grad=1e-9, tolerance_change=1e-12)
    trace = []
    t0 = time.perf_counter()

    def closure():
        opt.zero_grad()
        theta = torch.exp(phi)
        ll = B.gp_loglik(theta, points, z, family, alpha, tol_fact, tol_peel, o)
        loss = -ll / n
        loss.backward()
        # d loglik / d theta from d loss / d phi = -(theta / n) d loglik / d theta
        g = -phi.grad.detach() * n / theta.detach()
        trace.append((theta.detach().tolist(), float(ll.item()), g.tolist()))
        return loss

    opt.step(closure)
    theta = torch.exp(phi.detach())
    info = {"evals": len(trace), "seconds": time.perf_counter() - t0, "loglik": trace[-1][1] if trace else None,
            "trace": trace}
    return theta.tolist(), info


def fit_profile(points: torch.Tensor, z: torch.Tensor, family: int, theta0, alpha: float = 0.0,
                tol_fact: float = 1e-9, tol_peel: float = 1e-6, o: B.RsfOpts | None = None, max_iter: int = 30,
                history_size: int = 10):
    """Maximizes the profile log-likelihood of Sec. 5.5 (Eq. (prof): mean and
    variance level profiled out, unit variance in Sigma) over theta = (l, nug)
    from theta0 = (l0, nug0), by L-BFGS over log theta as in fit.  Returns
    (theta, info) with info = {"evals", "seconds", "loglik", "sigma2",
    "mu", "trace"}: sigma2 = z^T (Sigma + 1 1^T)^-1 z / n (the maximizing
    variance level) and mu = 1^T Sigma^-1 z / 1^T Sigma^-1 1 (the
    generalized-least-squares mean) at the final theta."""
    n = points.shape[0]
    phi = torch.tensor([math.log(float(v)) for v in theta0], dtype=torch.float64, requires_grad=True)
    opt = torch.optim.LBFGS([phi], lr=1.0, max_iter=max_iter, history_size=history_size,
                            line_search_fn="strong_wolfe", tolerance_grad=1e-9, tolerance_change=1e-12)
    trace = []
    t0 = time.perf_counter()

    def closure():
        opt.zero_grad()
        th = torch.exp(phi.detach())
        lt, g, _ = B.profile_loglik_and_score(points, z, family, (float(th[0]), 1.0, float(th[1])), tol_fact,
                                              tol_peel, alpha, o)
        gt = torch.stack([g[0], g[2]])
        # loss = -lt / n in the variables phi = log theta
        phi.grad = -(gt * th) / n
        trace.append((th.tolist(), lt, gt.tolist()))
        return torch.tensor(-lt / n, dtype=torch.float64)

    opt.step(closure)
    theta = torch.exp(phi.detach())
    lt, _, t = B.profile_loglik_and_score(points, z, family, (float(theta[0]), 1.0, float(theta[1])), tol_fact,
                                          tol_peel, alpha, o, want_score=False)
    info = {"evals": len(trace), "seconds": time.perf_counter() - t0, "loglik": lt,
            "sigma2": float(t[6]) / n, "mu": float(t[8] / t[9]), "trace": trace}
    return theta.tolist(), info
