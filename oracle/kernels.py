"""Covariance kernels K(x, y; theta) and their theta-derivatives, in fp64.

ORACLE -- test infrastructure only.  Nothing on the product path may import
this module; only tests, the smoke check and the benchmark's CPU-baseline leg.

theta = (l, s2, nug): length scale l, variance s2 and nugget (white-noise
variance on the index diagonal, delta_ij).  Families:

* Matern nu=1/2, 3/2, 5/2 closed forms (Sec. 5.5, Eq. (diffkernels)),
  multiplied by s2;
* Matern nu=1 via the Bessel form of Eq. (matern) (Sec. 1), s2 * x K_1(x)
  with x = sqrt(2) r / l;
* rational quadratic (Sec. 1, Eq. (rationalquadratic) with length scale),
  s2 * (1 + r^2 / (2 alpha l^2))^(-alpha);
* the general-nu Matern of Eq. (matern) through scipy's K_nu, used to pin the
  closed forms.

``which`` selects the matrix: 0 -> Sigma, 1 -> dSigma/dl, 2 -> dSigma/ds2,
3 -> dSigma/dnug.  The nugget lives on equal *indices* (delta_ij), so two
coincident points remain distinct observations.
"""
from __future__ import annotations

import numpy as np
from scipy import special

MATERN12, MATERN32, MATERN52, MATERN1, RQ = 0, 1, 2, 3, 4
SIGMA, D_L, D_S2, D_NUG = 0, 1, 2, 3

SQRT3 = np.sqrt(3.0)
SQRT5 = np.sqrt(5.0)
SQRT2 = np.sqrt(2.0)


def _xk1(x):
    """x K_1(x) with its limit 1 at x = 0."""
    x = np.asarray(x, dtype=np.float64)
    out = np.ones_like(x)
    nz = x > 0
    out[nz] = x[nz] * special.k1(x[nz])
    return out


def _x2k0(x):
    """x^2 K_0(x) with its limit 0 at x = 0."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    nz = x > 0
    out[nz] = x[nz] ** 2 * special.k0(x[nz])
    return out


def correlation(r, family, l, alpha=0.0):
    """Unit-variance correlation k(r) of the family (no s2, no nugget)."""
    r = np.asarray(r, dtype=np.float64)
    if family == MATERN12:
        return np.exp(-r / l)
    if family == MATERN32:
        a = SQRT3 * r / l
        return (1.0 + a) * np.exp(-a)
    if family == MATERN52:
        a = SQRT5 * r / l
        return (1.0 + a + a * a / 3.0) * np.exp(-a)
    if family == MATERN1:
        return _xk1(SQRT2 * r / l)
    if family == RQ:
        return (1.0 + r * r / (2.0 * alpha * l * l)) ** (-alpha)
    raise ValueError(f"unknown kernel family {family}")


def dcorrelation_dl(r, family, l, alpha=0.0):
    """d k(r) / d l, closed forms derived from the expressions above."""
    r = np.asarray(r, dtype=np.float64)
    if family == MATERN12:
        return (r / (l * l)) * np.exp(-r / l)
    if family == MATERN32:
        a = SQRT3 * r / l
        return a * a * np.exp(-a) / l
    if family == MATERN52:
        a = SQRT5 * r / l
        return (a * a / 3.0) * (1.0 + a) * np.exp(-a) / l
    if family == MATERN1:
        # (x K_1(x))' = -x K_0(x) and dx/dl = -x/l.
        return _x2k0(SQRT2 * r / l) / l
    if family == RQ:
        u = 1.0 + r * r / (2.0 * alpha * l * l)
        return u ** (-alpha - 1.0) * r * r / (l ** 3)
    raise ValueError(f"unknown kernel family {family}")


def kernel_offdiag(r, family, theta, which, alpha=0.0):
    """Entry of Sigma (which=0) or dSigma/dtheta_k for two distinct indices."""
    l, s2, nug = theta
    if which == SIGMA:
        return s2 * correlation(r, family, l, alpha)
    if which == D_L:
        return s2 * dcorrelation_dl(r, family, l, alpha)
    if which == D_S2:
        return correlation(r, family, l, alpha)
    if which == D_NUG:
        return np.zeros_like(np.asarray(r, dtype=np.float64))
    raise ValueError(f"unknown matrix selector {which}")


def diag_value(family, theta, which, alpha=0.0):
    """Diagonal entry (r = 0, same index) of Sigma or dSigma/dtheta_k."""
    l, s2, nug = theta
    if which == SIGMA:
        return s2 + nug
    if which == D_L:
        return 0.0
    if which == D_S2:
        return 1.0
    if which == D_NUG:
        return 1.0
    raise ValueError(f"unknown matrix selector {which}")


def pairwise_dist(xa, xb):
    """Euclidean distances between rows of xa (m,2) and xb (k,2)."""
    dx = xa[:, 0:1] - xb[None, :, 0]
    dy = xa[:, 1:2] - xb[None, :, 1]
    return np.sqrt(dx * dx + dy * dy)


def kernel_block(xa, xb, family, theta, which, alpha=0.0, ia=None, ib=None):
    """Block K(xa, xb) of Sigma or one of its derivatives.

    ``ia``/``ib`` are the global indices of the rows/columns; entries with
    equal indices get the diagonal value (nugget on delta_ij).  Without
    indices all entries are treated as off-diagonal (distinct observations).
    """
    r = pairwise_dist(xa, xb)
    out = kernel_offdiag(r, family, theta, which, alpha)
    if ia is not None and ib is not None:
        same = np.asarray(ia)[:, None] == np.asarray(ib)[None, :]
        if np.any(same):
            out = np.where(same, diag_value(family, theta, which, alpha), out)
    return out


def matern_general(r, nu, l):
    """Eq. (matern) with length scale: 2^(1-nu)/Gamma(nu) x^nu K_nu(x),
    x = sqrt(2 nu) r / l; value 1 at r = 0.  Uses scipy's Bessel K_nu."""
    r = np.asarray(r, dtype=np.float64)
    x = np.sqrt(2.0 * nu) * r / l
    out = np.ones_like(x)
    nz = x > 0
    out[nz] = (2.0 ** (1.0 - nu) / special.gamma(nu)) * x[nz] ** nu * special.kv(nu, x[nz])
    return out
