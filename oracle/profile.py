"""Profile log-likelihood (Sec. 5.5, Eq. (prof) and its gradient) and the
conditional distribution (Remark conditional, Sec. 4), CPU fp64.

ORACLE -- test infrastructure only (tests, smoke check, benchmark CPU leg).

Profile likelihood.  The model z ~ N(mu 1, sigma^2 Sigma(theta)) with the
mean level mu and the variance level sigma^2 profiled out.  Written exactly as
Eq. (prof) prints it, with A = Sigma + 1 1^T:

    lt(theta) = -1/2 log|Sigma| - n/2 log(z^T A^-1 z) + n/2 (log n - 1 - log 2 pi)
    gt_i      = -1/2 Tr(Sigma^-1 Sigma_i) + n/2 (z^T A^-1 Sigma_i A^-1 z) / (z^T A^-1 z)

The printed constant reads "log n - 1 - 2 pi"; the maximum over sigma^2 of the
Gaussian log-density fixes it as log n - 1 - log 2 pi (sigma^2-hat =
z^T A^-1 z / n), which is the reading taken.  The printed gradient is the
exact derivative of the printed lt (dA/dtheta_i = Sigma_i), so the pair is
consistent as printed.

Conditional distribution.  For [z', z] jointly Gaussian with covariance
[[S11, S12], [S12^T, S22]] (the same kernel, nugget on equal indices only, so
S12 holds no nugget):

    z' | z ~ N(S12 S22^-1 z, S11 - S12 S22^-1 S12^T).

A sample is mean + y1 - S12 S22^-1 y2 with y = G w for any square root G of
the joint covariance (G G^T = Sigma) and w ~ N(0, I): its covariance is
[I, -S12 S22^-1] Sigma [I, -S12 S22^-1]^T, the conditional covariance.  The
remark applies S12 through the joint operator on a zero-padded vector,
S12 v = (Sigma [0; v])[:m].
"""
from __future__ import annotations

import numpy as np
from scipy import linalg

from . import kernels as K
from .dense import cov_matrix, params


def profile_loglik_dense(x, z, family, theta, alpha=0.0):
    """Eq. (prof) by dense Cholesky.  Returns (lt, qt, logdet) with
    qt = z^T (Sigma + 1 1^T)^-1 z and logdet = log|Sigma|."""
    n = x.shape[0]
    S = cov_matrix(x, family, theta, K.SIGMA, alpha)
    logdet = 2.0 * float(np.sum(np.log(np.diag(linalg.cholesky(S, lower=True)))))
    A = S + np.ones((n, n))
    qt = float(z @ linalg.cho_solve(linalg.cho_factor(A, lower=True), z))
    lt = -0.5 * logdet - 0.5 * n * np.log(qt) + 0.5 * n * (np.log(n) - 1.0 - np.log(2.0 * np.pi))
    return lt, qt, logdet


def profile_score_dense(x, z, family, theta, alpha=0.0):
    """Gradient of Eq. (prof), as printed, for theta = (l, s2, nug) (or the
    anisotropic (l1, s2, nug, l2)).

    Returns dict with g (3,), quadk (gamma^T Sigma_k gamma, gamma = A^-1 z),
    trace (Tr(Sigma^-1 Sigma_k)), lt, qt, logdet."""
    n = x.shape[0]
    S = cov_matrix(x, family, theta, K.SIGMA, alpha)
    Sinv = linalg.cho_solve(linalg.cho_factor(S, lower=True), np.eye(n))
    lt, qt, logdet = profile_loglik_dense(x, z, family, theta, alpha)
    A = S + np.ones((n, n))
    gamma = linalg.cho_solve(linalg.cho_factor(A, lower=True), z)
    p = len(params(theta))
    g = np.zeros(p)
    quadk = np.zeros(p)
    trace = np.zeros(p)
    for k, which in enumerate(params(theta)):
        Sk = cov_matrix(x, family, theta, which, alpha)
        quadk[k] = float(gamma @ (Sk @ gamma))
        trace[k] = float(np.sum(Sinv * Sk))
        g[k] = -0.5 * trace[k] + 0.5 * n * quadk[k] / qt
    return dict(g=g, quadk=quadk, trace=trace, lt=lt, qt=qt, logdet=logdet)


def conditional_dense(x, z, xs, family, theta, alpha=0.0):
    """Mean S12 S22^-1 z and covariance S11 - S12 S22^-1 S12^T of z' at the
    m new points xs given z at the n points x (Remark conditional)."""
    n, m = x.shape[0], xs.shape[0]
    ix, isx = np.arange(n), np.arange(m)
    S22 = K.kernel_block(x, x, family, theta, K.SIGMA, alpha, ix, ix)
    S11 = K.kernel_block(xs, xs, family, theta, K.SIGMA, alpha, isx, isx)
    S12 = K.kernel_block(xs, x, family, theta, K.SIGMA, alpha)
    c = linalg.cho_factor(S22, lower=True)
    mean = S12 @ linalg.cho_solve(c, z)
    cov = S11 - S12 @ linalg.cho_solve(c, S12.T)
    return mean, cov


def conditional_samples(mean, apply_joint, sqrt_joint, solve22, w, m):
    """Samples of z' | z by the remark's identity, with the joint operators
    given as callables on (m + n, q) arrays (joint order: new points first)
    and solve22 on (n, q) arrays:

        y = sqrt_joint(w);  s = mean + y[:m] - apply_joint([0; solve22(y[m:])])[:m]
    """
    w = np.asarray(w, dtype=np.float64)
    if w.ndim == 1:
        w = w[:, None]
    y = sqrt_joint(w)
    v = solve22(y[m:])
    t = apply_joint(np.vstack([np.zeros((m, w.shape[1])), v]))[:m]
    return np.asarray(mean)[:, None] + y[:m] - t
