"""Algorithm 1 (Sec. 4): RSF log-likelihood and peeled score, CPU fp64.

ORACLE -- test infrastructure only (tests, smoke check, benchmark CPU leg).

theta = (l, s2, nug) for K = s2 k(r/l) + nug delta_ij, or the anisotropic
(l1, s2, nug, l2) of Sec. 5.1 (a fourth score component, d/dl2, from its own
factorization and peeled trace).  Readings:

* the constant is -(n/2) log 2 pi as in Eq. (loglikelihood) (the algorithm box
  prints -1/2 log 2 pi, read as a typo);
* only Sigma and Sigma_l are factored.  Sigma_nug = I, so its trace is
  Tr(F^-1), peeled directly; Sigma_s2 = (Sigma - nug I)/s2 exactly, so
  Tr(Sigma^-1 Sigma_s2) = (n - nug Tr(Sigma^-1))/s2 and
  z^T S^-1 S_s2 S^-1 z = (z^T a - nug a^T a)/s2 with a = F^-1 z;
* Tr(Sigma^-1 Sigma_l) is peeled from G = (F^-1 F_l + F_l F^-1)/2.
"""
from __future__ import annotations

import numpy as np

from . import kernels as K
from .rsf import Factorization
from .tree import Tree, DEFAULT_OPTS
from .peel import peel_trace


def loglik_and_score(x, z, family, theta, tol_fact=1e-9, tol_peel=1e-6,
                     alpha=0.0, opts=None, seed=0, want_score=True):
    o = dict(DEFAULT_OPTS)
    if opts:
        o.update(opts)
    tree = Tree(x, o["n_occ"])
    n = tree.n
    zt = np.asarray(z, dtype=np.float64)[tree.perm]
    F = Factorization(x, family, theta, K.SIGMA, tol_fact, alpha, o, tree)
    a = F.solve(zt)
    quad = float(zt @ a)
    logdet = F.logdet()
    ell = -0.5 * quad - 0.5 * logdet - 0.5 * n * np.log(2.0 * np.pi)
    out = dict(ell=ell, quad=quad, logdet=logdet, tree=tree, F=F)
    if not want_score:
        return out
    l, s2, nug = theta[:3]
    Fl = Factorization(x, family, theta, K.D_L, tol_fact, alpha, o, tree)
    t_nug, info_nug = peel_trace(F.solve, tree, tol_peel, seed=seed)
    t_l, info_l = peel_trace(lambda X: 0.5 * (F.solve(Fl.apply(X)) + Fl.apply(F.solve(X))),
                             tree, tol_peel, seed=seed)
    aa = float(a @ a)
    q_l = float(a @ Fl.apply(a))
    q_s2 = (quad - nug * aa) / s2
    t_s2 = (n - nug * t_nug) / s2
    quadk = [q_l, q_s2, aa]
    trace = [t_l, t_s2, t_nug]
    if len(theta) == 4:
        # anisotropic theta (Sec. 5.1): the second length scale's factorization and trace
        Fl2 = Factorization(x, family, theta, K.D_L2, tol_fact, alpha, o, tree)
        t_l2, _ = peel_trace(lambda X: 0.5 * (F.solve(Fl2.apply(X)) + Fl2.apply(F.solve(X))),
                             tree, tol_peel, seed=seed)
        quadk.append(float(a @ Fl2.apply(a)))
        trace.append(t_l2)
        out.update(Fl2=Fl2)
    quadk = np.array(quadk)
    trace = np.array(trace)
    g = 0.5 * quadk - 0.5 * trace
    out.update(g=g, quadk=quadk, trace=trace, Fl=Fl, info_l=info_l, info_nug=info_nug)
    return out
