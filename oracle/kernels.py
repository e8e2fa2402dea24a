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

Anisotropic form (Sec. 5.1): with theta = (l1, s2, nug, l2) (four entries)
the family's unit-length correlation is taken at the scaled distance
||x - y||_theta = sqrt((x1 - y1)^2 / l1^2 + (x2 - y2)^2 / l2^2), so
Eqs. (specmatern) and (specrq) are Matern 3/2 and RQ alpha = 1/2 with
s2 = 1; which = 1 is then d/dl1 and which = 4 (D_L2) is d/dl2.
"""
from __future__ import annotations

import numpy as np
from scipy import special

MATERN12, MATERN32, MATERN52, MATERN1, RQ = 0, 1, 2, 3, 4
SIGMA, D_L, D_S2, D_NUG, D_L2 = 0, 1, 2, 3, 4

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
    """Entry of Sigma (which=0) or dSigma/dtheta_k for two distinct indices
    (isotropic theta = (l, s2, nug))."""
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


def aniso_offdiag(dx, dy, family, theta, which, alpha=0.0):
    """Off-diagonal entries for the anisotropic theta = (l1, s2, nug, l2) of
    Sec. 5.1 at coordinate differences dx, dy.  The correlation depends on
    r = ||x - y||_theta only; its theta_k-derivative is k'(r) dr/dtheta_k with
    dr/dl1 = -(dx/l1)^2 / (l1 r) and dr/dl2 = -(dy/l2)^2 / (l2 r), and k'(r)
    follows from the unit-length l-derivative of k(r/l): d/dl k(r/l) at l = 1
    is -r k'(r)."""
    l1, s2, nug, l2 = theta
    u = np.asarray(dx, dtype=np.float64) / l1
    v = np.asarray(dy, dtype=np.float64) / l2
    r = np.sqrt(u * u + v * v)
    if which == SIGMA:
        return s2 * correlation(r, family, 1.0, alpha)
    if which == D_S2:
        return correlation(r, family, 1.0, alpha)
    if which == D_NUG:
        return np.zeros_like(r)
    if which in (D_L, D_L2):
        w = u * u / l1 if which == D_L else v * v / l2
        out = np.zeros_like(r)
        nz = r > 0
        kprime = -dcorrelation_dl(r[nz], family, 1.0, alpha) / r[nz]
        out[nz] = s2 * kprime * (-w[nz] / r[nz])
        return out
    raise ValueError(f"unknown matrix selector {which}")


def diag_value(family, theta, which, alpha=0.0):
    """Diagonal entry (r = 0, same index) of Sigma or dSigma/dtheta_k."""
    l, s2, nug = theta[:3]
    if which == SIGMA:
        return s2 + nug
    if which in (D_L, D_L2):
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
    if len(theta) == 4:
        dx = xa[:, 0:1] - xb[None, :, 0]
        dy = xa[:, 1:2] - xb[None, :, 1]
        out = aniso_offdiag(dx, dy, family, theta, which, alpha)
    else:
        out = kernel_offdiag(pairwise_dist(xa, xb), family, theta, which, alpha)
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
