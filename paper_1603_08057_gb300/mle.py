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


# (tol_fact, tol_peel, L-BFGS iterations) per stage: two orders looser, one
# order looser, then the paper's pairing eps_fact = eps_peel / 1000 (Sec. 5.3).
DEFAULT_STAGES = ((1e-7, 1e-4, 10), (1e-8, 1e-5, 10), (1e-9, 1e-6, 30))


def fit_staged(points: torch.Tensor, z: torch.Tensor, family: int, theta0, stages=DEFAULT_STAGES,
               alpha: float = 0.0, o: B.RsfOpts | None = None, history_size: int = 10):
    """Maximum likelihood with the tolerances tightened as the optimization
    proceeds (the dynamic tolerances the paper suggests in Sec. 6): the
    L-BFGS of fit runs at each (tol_fact, tol_peel, max_iter) stage in turn,
    each started from the previous stage's theta, so the early iterations far
    from the maximizer run on cheaper, looser factorizations and peelings.
    Returns (theta, info) with info = {"evals", "seconds", "loglik",
    "stages": [per-stage info of fit, with its tolerances]}; loglik is the
    last stage's, at its tolerances."""
    theta = [float(v) for v in theta0]
    per = []
    for tol_fact, tol_peel, iters in stages:
        theta, info = fit(points, z, family, theta, alpha, tol_fact, tol_peel, o, iters, history_size)
        info = dict(info, tol_fact=tol_fact, tol_peel=tol_peel)
        per.append(info)
    return theta, {"evals": sum(i["evals"] for i in per), "seconds": sum(i["seconds"] for i in per),
                   "loglik": per[-1]["loglik"] if per else None, "stages": per}
