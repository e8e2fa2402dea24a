"""Oracle-D: exact dense fp64 log-likelihood and score (O(n^3)).

ORACLE -- test infrastructure only (tests, smoke check, benchmark CPU leg).

* Eq. (loglikelihood), Sec. 1:  l = -1/2 z^T S^-1 z - 1/2 log|S| - n/2 log 2pi
* Eq. (gradient), Sec. 1:       g_k = 1/2 z^T S^-1 S_k S^-1 z - 1/2 Tr(S^-1 S_k)
computed through a dense Cholesky factorization, the "naive" method the paper
sets out to replace (Sec. 1).
"""
from __future__ import annotations

import numpy as np
from scipy import linalg

from . import kernels as K


def cov_matrix(x, family, theta, which=K.SIGMA, alpha=0.0):
    """Dense Sigma (which=0) or dSigma/dtheta_k, nugget on delta_ij."""
    n = x.shape[0]
    idx = np.arange(n)
    return K.kernel_block(x, x, family, theta, which, alpha, idx, idx)


def loglik_dense(x, z, family, theta, alpha=0.0):
    """Returns (l, quad, logdet) with quad = z^T Sigma^-1 z."""
    S = cov_matrix(x, family, theta, K.SIGMA, alpha)
    c = linalg.cho_factor(S, lower=True)
    a = linalg.cho_solve(c, z)
    quad = float(z @ a)
    logdet = 2.0 * float(np.sum(np.log(np.diag(c[0]))))
    n = x.shape[0]
    ell = -0.5 * quad - 0.5 * logdet - 0.5 * n * np.log(2.0 * np.pi)
    return ell, quad, logdet


def params(theta):
    """Matrix selectors of the score's components: (l, s2, nug), then l2
    for the anisotropic theta of Sec. 5.1."""
    return (K.D_L, K.D_S2, K.D_NUG) + ((K.D_L2,) if len(theta) == 4 else ())


def score_dense(x, z, family, theta, alpha=0.0):
    """Exact score g (3,), or (4,) for an anisotropic theta, plus its terms.

    Returns dict with g, quadk (z^T S^-1 S_k S^-1 z), trace (Tr(S^-1 S_k)),
    ell, quad, logdet.
    """
    n = x.shape[0]
    S = cov_matrix(x, family, theta, K.SIGMA, alpha)
    c = linalg.cho_factor(S, lower=True)
    a = linalg.cho_solve(c, z)
    Sinv = linalg.cho_solve(c, np.eye(n))
    quad = float(z @ a)
    logdet = 2.0 * float(np.sum(np.log(np.diag(c[0]))))
    ell = -0.5 * quad - 0.5 * logdet - 0.5 * n * np.log(2.0 * np.pi)
    p = len(params(theta))
    g = np.zeros(p)
    quadk = np.zeros(p)
    trace = np.zeros(p)
    for k, which in enumerate(params(theta)):
        Sk = cov_matrix(x, family, theta, which, alpha)
        quadk[k] = float(a @ (Sk @ a))
        trace[k] = float(np.sum(Sinv * Sk))  # Tr(S^-1 S_k), both symmetric
        g[k] = 0.5 * quadk[k] - 0.5 * trace[k]
    return dict(g=g, quadk=quadk, trace=trace, ell=ell, quad=quad, logdet=logdet)


def sample_z_dense(x, family, theta, w, alpha=0.0):
    """z = C w with Sigma = C C^T (dense Cholesky), so z ~ N(0, Sigma) when
    w ~ N(0, I)."""
    S = cov_matrix(x, family, theta, K.SIGMA, alpha)
    C = linalg.cholesky(S, lower=True)
    return C @ w
