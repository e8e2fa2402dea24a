"""Thin ctypes binding of the C-ABI library ``librsf.so`` (include/rsf.h).

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels.  PyTorch supplies device memory (float64 CUDA tensors)
and the current CUDA stream.  There is no CPU fallback: if the library is not
built, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "librsf.so")

# rsf_family, rsf_which, rsf_op (include/rsf.h)
MATERN12, MATERN32, MATERN52, MATERN1, RQ = 0, 1, 2, 3, 4
SIGMA, D_L, D_S2, D_NUG, D_L2 = 0, 1, 2, 3, 4
OP_INV, OP_APPLY, OP_SQRT, OP_SQRT_T, OP_INV_SQRT, OP_INV_SQRT_T = range(6)
STATUS = {0: "RSF_OK", 1: "RSF_EINVAL", 2: "RSF_ENOMEM", 3: "RSF_ENOTPD",
          4: "RSF_ENUMERIC", 5: "RSF_ETIMEOUT", 6: "RSF_ECUDA"}

EXPORTS = ["rsf_opts_default", "rsf_last_error", "rsf_tree_build", "rsf_tree_destroy",
           "rsf_build", "rsf_build_on_tree", "rsf_logdet", "rsf_solve", "rsf_peel_trace",
           "gp_loglik", "gp_score", "gp_loglik_and_score", "rsf_get_info",
           "rsf_launch_count", "rsf_profile_enable", "rsf_profile_read", "rsf_destroy",
           "rsf_solve_noalloc", "rsf_set_allocator", "rsf_build_batched", "rsf_logdet_sets",
           "gp_loglik_and_score_batched", "rsf_selftest_wait_limit", "rsf_selftest_gemm",
           "gp_profile_loglik_and_score", "gp_profile_loglik_and_score_batched", "gp_conditional",
           "rsf_tree_export"]


class RsfKernel(C.Structure):
    _fields_ = [("family", C.c_int), ("alpha", C.c_double), ("anisotropic", C.c_int)]


class RsfOpts(C.Structure):
    _fields_ = [("n_occ", C.c_int), ("n_prox", C.c_int), ("n_rings", C.c_int),
                ("r_near", C.c_double), ("r_in", C.c_double), ("r_out", C.c_double),
                ("oversample", C.c_int), ("q0", C.c_int), ("seed", C.c_uint64),
                ("precision", C.c_int), ("trace_form", C.c_int), ("refine", C.c_int), ("probes", C.c_int)]


PREC_FP64, PREC_MIXED, PREC_MIXED_DF64 = 0, 1, 2
TRACE_SYM, TRACE_SQRT, TRACE_HUTCH = 0, 1, 2
COND_RSF, COND_DIRECT = 0, 1


class RsfInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("levels", C.c_int), ("boxes", C.c_int64),
                ("root_size", C.c_int), ("max_rank", C.c_int), ("max_active", C.c_int),
                ("factor_entries", C.c_int64), ("flops", C.c_double),
                ("kernel_evals", C.c_double), ("nsets", C.c_int), ("solve_df64", C.c_int),
                ("probe_rel_diff", C.c_double)]


class RsfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def lib():
    """Loads the library (built in-tree by ``build.build()``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIBPATH):
            raise RuntimeError(f"{LIBPATH} is missing: run paper_1603_08057_gb300.build.build() first")
        L = C.CDLL(LIBPATH)
        vp, dp, i64, ip = C.c_void_p, C.POINTER(C.c_double), C.c_int64, C.c_int
        L.rsf_last_error.restype = C.c_char_p
        L.rsf_opts_default.argtypes = [C.POINTER(RsfOpts)]
        L.rsf_opts_default.restype = None
        L.rsf_tree_build.argtypes = [vp, i64, C.POINTER(RsfOpts), vp, C.POINTER(vp)]
        L.rsf_tree_destroy.argtypes = [vp]
        L.rsf_tree_export.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int), vp, vp]
        L.rsf_tree_destroy.restype = None
        L.rsf_build.argtypes = [vp, i64, C.POINTER(RsfKernel), dp, ip, C.c_double,
                                C.POINTER(RsfOpts), vp, C.POINTER(vp)]
        L.rsf_build_on_tree.argtypes = [vp, C.POINTER(RsfKernel), dp, ip, C.c_double,
                                        C.POINTER(RsfOpts), C.POINTER(vp)]
        L.rsf_logdet.argtypes = [vp, dp]
        L.rsf_set_allocator.argtypes = [_ALLOC_FN, _FREE_FN, vp]
        L.rsf_solve.argtypes = [vp, vp, i64, ip, ip]
        L.rsf_solve_noalloc.argtypes = [vp, vp, i64, ip, ip]
        L.rsf_peel_trace.argtypes = [vp, vp, C.c_double, C.POINTER(RsfOpts), dp]
        L.gp_loglik.argtypes = [vp, vp, vp, dp, dp]
        L.gp_score.argtypes = [vp, vp, C.c_double, C.c_double, C.POINTER(RsfOpts), dp, dp]
        L.gp_loglik_and_score.argtypes = [vp, vp, i64, C.POINTER(RsfKernel), dp, C.c_double,
                                          C.c_double, C.POINTER(RsfOpts), vp, dp, dp, dp]
        L.rsf_get_info.argtypes = [vp, C.POINTER(RsfInfo)]
        L.rsf_build_batched.argtypes = [ip, C.POINTER(C.c_int64), vp, C.POINTER(RsfKernel), dp, ip,
                                        C.c_double, C.POINTER(RsfOpts), vp, C.POINTER(vp)]
        L.rsf_logdet_sets.argtypes = [vp, dp]
        L.rsf_selftest_wait_limit.argtypes = [vp]
        L.rsf_selftest_gemm.argtypes = [ip, ip, ip, ip, ip, ip, C.c_double, vp, ip, vp, ip, C.c_double, vp, ip, vp]
        L.gp_loglik_and_score_batched.argtypes = [ip, C.POINTER(C.c_int64), vp, vp, C.POINTER(RsfKernel), dp,
                                                  C.c_double, C.c_double, C.POINTER(RsfOpts), vp, dp, dp, dp]
        L.gp_profile_loglik_and_score.argtypes = L.gp_loglik_and_score.argtypes
        L.gp_profile_loglik_and_score_batched.argtypes = L.gp_loglik_and_score_batched.argtypes
        L.gp_conditional.argtypes = [vp, i64, vp, vp, i64, C.POINTER(RsfKernel), dp, C.c_double,
                                     C.POINTER(RsfOpts), vp, ip, vp, vp, ip, vp]
        L.rsf_profile_enable.argtypes = [ip]
        L.rsf_profile_enable.restype = None
        L.rsf_profile_read.argtypes = [ip, ip, C.POINTER(C.c_int64), dp, dp, dp]
        L.rsf_launch_count.argtypes = [ip]
        L.rsf_launch_count.restype = C.c_int64
        L.rsf_destroy.argtypes = [vp]
        L.rsf_destroy.restype = None
        for name in EXPORTS:
            if name not in ("rsf_opts_default", "rsf_last_error", "rsf_tree_destroy",
                            "rsf_launch_count", "rsf_profile_enable", "rsf_destroy"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(code):
    if code != 0:
        raise RsfError(code, lib().rsf_last_error().decode())


def opts(**kw) -> RsfOpts:
    o = RsfOpts()
    lib().rsf_opts_default(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _dev(t: torch.Tensor, shape=None) -> torch.Tensor:
    if not (t.is_cuda and t.dtype == torch.float64):
        raise TypeError("expected a float64 CUDA tensor")
    t = t.contiguous()
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {shape}, got {tuple(t.shape)}")
    return t


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _theta(theta):
    """theta (l, s2, nug) or, anisotropic (Sec. 5.1), (l1, s2, nug, l2)."""
    th = [float(v) for v in (theta.tolist() if isinstance(theta, torch.Tensor) else theta)]
    if len(th) not in (3, 4):
        raise ValueError("theta must have 3 entries (l, s2, nug) or 4 (l1, s2, nug, l2)")
    return (C.c_double * len(th))(*th)


def _kernel(family, alpha, theta) -> RsfKernel:
    """The kernel descriptor; a 4-entry theta selects the anisotropic form."""
    return RsfKernel(family, alpha, 1 if len(theta) == 4 else 0)


def launch_count(reset=False) -> int:
    return int(lib().rsf_launch_count(1 if reset else 0))


PROF_GEMM, PROF_QR_UPDATE, PROF_QR_PIVOT = 0, 1, 2
PROF_PEEL_APPLY, PROF_PEEL_SUB, PROF_PEEL_QR, PROF_PEEL_REST, PROF_FACTOR, PROF_GEMM_DF = 3, 4, 5, 6, 7, 8
PROF_GEMM_TC = 9
PROF_NAMES = ["gemm_fp64", "qr", "qr_pivot", "peel_apply", "peel_sub", "peel_qr", "peel_rest",
              "factor", "gemm_df64", "gemm_tc"]


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_hooks = None   # keeps the ctypes callbacks alive while installed


def use_torch_allocator(enable: bool = True) -> None:
    """rsf_set_allocator with PyTorch's caching allocator (enable) or the
    library's default cudaMallocAsync (disable).  Every device buffer the
    library allocates afterwards comes from, and returns to, the torch pool of
    the current device, on the library's stream."""
    global _hooks
    if not enable:
        _check(lib().rsf_set_allocator(_ALLOC_FN(), _FREE_FN(), None))
        _hooks = None
        return
    dev = torch.cuda.current_device()

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(stream or 0))
        except Exception:   # reported by the library as RSF_ENOMEM
            return None

    def _free(ptr, nbytes, stream, ctx):
        try:
            torch.cuda.caching_allocator_delete(ptr)
        except Exception:   # interpreter shutdown: torch already torn down
            pass

    hooks = (_ALLOC_FN(_alloc), _FREE_FN(_free))
    _check(lib().rsf_set_allocator(hooks[0], hooks[1], None))
    _hooks = hooks


def selftest_wait_limit() -> None:
    """rsf_selftest_wait_limit: runs the bounded grid barrier into its time
    limit on the current stream; raises RsfError unless it reported
    RSF_ETIMEOUT and returned."""
    _check(lib().rsf_selftest_wait_limit(_stream()))


def selftest_gemm(engine: int, A: torch.Tensor, B: torch.Tensor, C: torch.Tensor | None = None,
                  ta=False, tb=False, alpha=1.0, beta=0.0) -> torch.Tensor:
    """rsf_selftest_gemm: alpha op(A) op(B) + beta C with batched-GEMM engine
    `engine` (0 fp64, 1 tensor cores on pre-sliced df64 operands, 2 df64 CUDA
    cores, 3 tensor cores slicing inside the kernel) for
    float64 CUDA matrices in torch's row-major layout.  A row-major matrix is
    the column-major transpose, so the library computes the column-major
    C^T = op(B)^T op(A)^T, whose memory is the row-major C."""
    A, B = _dev(A), _dev(B)
    m = A.shape[1] if ta else A.shape[0]
    k = A.shape[0] if ta else A.shape[1]
    n = B.shape[0] if tb else B.shape[1]
    out = torch.zeros((m, n), dtype=torch.float64, device=A.device) if C is None else _dev(C, (m, n)).clone()
    _check(lib().rsf_selftest_gemm(engine, n, m, k, 1 if tb else 0, 1 if ta else 0, alpha,
                                   B.data_ptr(), B.shape[1], A.data_ptr(), A.shape[1], beta,
                                   out.data_ptr(), n, _stream()))
    return out


def profile(enable: bool) -> None:
    """Turns the library's per-kernel event timing on or off."""
    lib().rsf_profile_enable(1 if enable else 0)


def profile_read(category: int, reset: bool = False) -> dict:
    """Totals of one kernel category: launches, ms (summed CUDA-event time on
    the launching stream), algorithmic flops and bytes."""
    n = C.c_int64()
    ms, fl, by = C.c_double(), C.c_double(), C.c_double()
    _check(lib().rsf_profile_read(category, 1 if reset else 0, C.byref(n), C.byref(ms), C.byref(fl), C.byref(by)))
    return dict(launches=n.value, ms=ms.value, flops=fl.value, bytes=by.value)


class Tree:
    """rsf_tree_build: quadtree over a (n, 2) float64 CUDA tensor."""

    def __init__(self, points: torch.Tensor, o: RsfOpts | None = None):
        self.points = _dev(points)
        self.n = self.points.shape[0]
        self.h = C.c_void_p()
        _check(lib().rsf_tree_build(self.points.data_ptr(), self.n, C.byref(o) if o else None,
                                    _stream(), C.byref(self.h)))

    def export(self):
        """rsf_tree_export: (perm (n,), boxes (nbox, 6): level, start, count,
        parent, slot, set) as numpy int arrays."""
        n, nb = C.c_int64(), C.c_int()
        _check(lib().rsf_tree_export(self.h, C.byref(n), C.byref(nb), None, None))
        perm = np.empty(n.value, dtype=np.int32)
        boxes = np.empty((nb.value, 6), dtype=np.int32)
        _check(lib().rsf_tree_export(self.h, C.byref(n), C.byref(nb), perm.ctypes.data, boxes.ctypes.data))
        return perm, boxes

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.rsf_tree_destroy(self.h)
            self.h = None


class Factorization:
    """rsf_build / rsf_build_on_tree: RSF of Sigma (which=SIGMA) or of
    dSigma/dtheta (which=D_L, D_S2)."""

    def __init__(self, points_or_tree, family, theta, which=SIGMA, tol=1e-9, alpha=0.0,
                 o: RsfOpts | None = None, offsets=None):
        """offsets (sequence of nsets + 1 ints): points holds nsets independent
        datasets, set i in rows offsets[i]:offsets[i+1] (rsf_build_batched)."""
        self.kernel = _kernel(family, alpha, theta)
        self.h = C.c_void_p()
        th = _theta(theta)
        self.p = len(th)
        if offsets is not None:
            pts = _dev(points_or_tree)
            self.n = pts.shape[0]
            self.tree = None
            off = _offsets(offsets, self.n)
            _check(lib().rsf_build_batched(len(off) - 1, off, pts.data_ptr(), C.byref(self.kernel), th, which, tol,
                                           C.byref(o) if o else None, _stream(), C.byref(self.h)))
        elif isinstance(points_or_tree, Tree):
            self.tree = points_or_tree
            self.n = self.tree.n
            _check(lib().rsf_build_on_tree(self.tree.h, C.byref(self.kernel), th, which, tol,
                                           C.byref(o) if o else None, C.byref(self.h)))
        else:
            pts = _dev(points_or_tree)
            self.n = pts.shape[0]
            self.tree = None
            _check(lib().rsf_build(pts.data_ptr(), self.n, C.byref(self.kernel), th, which, tol,
                                   C.byref(o) if o else None, _stream(), C.byref(self.h)))

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.rsf_destroy(self.h)
            self.h = None

    def logdet_sets(self):
        """rsf_logdet_sets: per-dataset log-determinants (numpy array)."""
        k = self.info()["nsets"]
        v = (C.c_double * k)()
        _check(lib().rsf_logdet_sets(self.h, v))
        return np.array(list(v))

    def logdet(self) -> float:
        v = C.c_double()
        _check(lib().rsf_logdet(self.h, C.byref(v)))
        return v.value

    def solve(self, B: torch.Tensor, op=OP_INV) -> torch.Tensor:
        """op(F) B for B (n,) or (n, nrhs); returns a new tensor."""
        vec = B.dim() == 1
        X = _dev(B).reshape(self.n, -1)
        # column-major n x nrhs = transpose of a row-major nrhs x n array
        Xc = X.t().contiguous()
        _check(lib().rsf_solve(self.h, Xc.data_ptr(), self.n, Xc.shape[0], op))
        out = Xc.t()
        return out.reshape(-1) if vec else out.contiguous()

    def solve_noalloc(self, B: torch.Tensor, op=OP_INV) -> torch.Tensor:
        """op(F) B through rsf_solve_noalloc (no device allocation inside the
        library call; its work buffers live in the library's fixed scratch)."""
        vec = B.dim() == 1
        X = _dev(B).reshape(self.n, -1)
        Xc = X.t().contiguous()
        _check(lib().rsf_solve_noalloc(self.h, Xc.data_ptr(), self.n, Xc.shape[0], op))
        out = Xc.t()
        return out.reshape(-1) if vec else out.contiguous()

    def info(self) -> dict:
        i = RsfInfo()
        _check(lib().rsf_get_info(self.h, C.byref(i)))
        return {k: getattr(i, k) for k, _ in RsfInfo._fields_}

    def loglik(self, z: torch.Tensor):
        """gp_loglik: returns (loglik, quad, alpha = F^-1 z)."""
        z = _dev(z, (self.n,))
        a = torch.empty_like(z)
        ll, q = C.c_double(), C.c_double()
        _check(lib().gp_loglik(self.h, z.data_ptr(), a.data_ptr(), C.byref(ll), C.byref(q)))
        return ll.value, q.value, a

    def score(self, alpha: torch.Tensor, tol_fact=1e-9, tol_peel=1e-6, o: RsfOpts | None = None):
        """gp_score: returns (score (p,), terms (2p,)) as float64 CPU tensors,
        p = 3, or 4 for an anisotropic theta."""
        a = _dev(alpha, (self.n,))
        g = (C.c_double * self.p)()
        t = (C.c_double * (2 * self.p))()
        _check(lib().gp_score(self.h, a.data_ptr(), tol_fact, tol_peel, C.byref(o) if o else None, g, t))
        return torch.tensor(list(g), dtype=torch.float64), torch.tensor(list(t), dtype=torch.float64)


def peel_trace(F: Factorization, Fk: Factorization | None, tol_peel=1e-6, o: RsfOpts | None = None) -> float:
    v = C.c_double()
    _check(lib().rsf_peel_trace(F.h, Fk.h if Fk is not None else None, tol_peel,
                                C.byref(o) if o else None, C.byref(v)))
    return v.value


def loglik_and_score(points, z, family, theta, tol_fact=1e-9, tol_peel=1e-6, alpha=0.0,
                     o: RsfOpts | None = None, want_score=True):
    """gp_loglik_and_score: Algorithm 1 end to end.  Returns (loglik, score,
    terms); score and terms are None when want_score is False."""
    pts = _dev(points)
    n = pts.shape[0]
    zz = _dev(z, (n,))
    k = _kernel(family, alpha, theta)
    p = len(theta)
    ll = C.c_double()
    g = (C.c_double * p)()
    t = (C.c_double * (2 * p))()
    _check(lib().gp_loglik_and_score(pts.data_ptr(), zz.data_ptr(), n, C.byref(k), _theta(theta),
                                     tol_fact, tol_peel, C.byref(o) if o else None, _stream(),
                                     C.byref(ll), g if want_score else None, t if want_score else None))
    if not want_score:
        return ll.value, None, None
    return ll.value, torch.tensor(list(g), dtype=torch.float64), torch.tensor(list(t), dtype=torch.float64)


def _offsets(offsets, n):
    off = [int(v) for v in offsets]
    if len(off) < 2 or off[0] != 0 or off[-1] != n:
        raise ValueError("offsets must start at 0 and end at the number of points")
    return (C.c_int64 * len(off))(*off)


def loglik_and_score_batched(points, offsets, z, family, theta, tol_fact=1e-9, tol_peel=1e-6, alpha=0.0,
                             o: RsfOpts | None = None, want_score=True):
    """gp_loglik_and_score_batched: Algorithm 1 for nsets independent datasets
    in one forest.  Returns numpy arrays loglik (nsets,), score (nsets, 3)
    and terms (nsets, 6); the last two are None when want_score is False."""
    pts = _dev(points)
    n = pts.shape[0]
    zz = _dev(z, (n,))
    off = _offsets(offsets, n)
    k = len(off) - 1
    kern = _kernel(family, alpha, theta)
    p = len(theta)
    ll = (C.c_double * k)()
    g = (C.c_double * (p * k))()
    t = (C.c_double * (2 * p * k))()
    _check(lib().gp_loglik_and_score_batched(k, off, pts.data_ptr(), zz.data_ptr(), C.byref(kern), _theta(theta),
                                             tol_fact, tol_peel, C.byref(o) if o else None, _stream(), ll,
                                             g if want_score else None, t if want_score else None))
    if not want_score:
        return np.array(list(ll)), None, None
    return np.array(list(ll)), np.array(list(g)).reshape(k, p), np.array(list(t)).reshape(k, 2 * p)


def profile_loglik_and_score(points, z, family, theta, tol_fact=1e-9, tol_peel=1e-6, alpha=0.0,
                             o: RsfOpts | None = None, want_score=True):
    """gp_profile_loglik_and_score: the profile log-likelihood of Sec. 5.5
    (mean and variance level profiled out).  Returns (lt, score, terms):
    score (p,) or None, terms (2p + 4,) as documented in the header."""
    pts = _dev(points)
    n = pts.shape[0]
    zz = _dev(z, (n,))
    k = _kernel(family, alpha, theta)
    p = len(theta)
    ll = C.c_double()
    g = (C.c_double * p)()
    t = (C.c_double * (2 * p + 4))()
    _check(lib().gp_profile_loglik_and_score(pts.data_ptr(), zz.data_ptr(), n, C.byref(k), _theta(theta),
                                             tol_fact, tol_peel, C.byref(o) if o else None, _stream(),
                                             C.byref(ll), g if want_score else None, t))
    terms = torch.tensor(list(t), dtype=torch.float64)
    return ll.value, (torch.tensor(list(g), dtype=torch.float64) if want_score else None), terms


def profile_loglik_and_score_batched(points, offsets, z, family, theta, tol_fact=1e-9, tol_peel=1e-6, alpha=0.0,
                                     o: RsfOpts | None = None, want_score=True):
    """gp_profile_loglik_and_score_batched: per-set profile log-likelihoods.
    Returns numpy arrays (nsets,), (nsets, p) or None, (nsets, 2p + 4)."""
    pts = _dev(points)
    n = pts.shape[0]
    zz = _dev(z, (n,))
    off = _offsets(offsets, n)
    k = len(off) - 1
    kern = _kernel(family, alpha, theta)
    p = len(theta)
    ll = (C.c_double * k)()
    g = (C.c_double * (p * k))()
    t = (C.c_double * ((2 * p + 4) * k))()
    _check(lib().gp_profile_loglik_and_score_batched(k, off, pts.data_ptr(), zz.data_ptr(), C.byref(kern),
                                                     _theta(theta), tol_fact, tol_peel, C.byref(o) if o else None,
                                                     _stream(), ll, g if want_score else None, t))
    g = np.array(list(g)).reshape(k, p) if want_score else None
    return np.array(list(ll)), g, np.array(list(t)).reshape(k, 2 * p + 4)


def conditional(points, z, new_points, family, theta, tol=1e-9, alpha=0.0, o: RsfOpts | None = None,
                method=COND_RSF, w=None):
    """gp_conditional: mean (m,) of z' at new_points given z, and, when w
    ((m + n) x q, new points first) is given, the samples (m, q)."""
    pts = _dev(points)
    n = pts.shape[0]
    zz = _dev(z, (n,))
    xs = _dev(new_points)
    m = xs.shape[0]
    kern = _kernel(family, alpha, theta)
    mean = torch.empty(m, dtype=torch.float64, device=pts.device)
    q, wp, sp, S, wt = 0, None, None, None, None
    if w is not None:
        ww = _dev(w)
        if ww.dim() == 1:
            ww = ww.reshape(-1, 1)
        if ww.shape[0] != m + n:
            raise ValueError("w must have m + n rows")
        q = ww.shape[1]
        wt = ww.t().contiguous()  # column-major (m + n) x q
        S = torch.empty(q, m, dtype=torch.float64, device=pts.device)
        wp, sp = wt.data_ptr(), S.data_ptr()
    _check(lib().gp_conditional(pts.data_ptr(), n, zz.data_ptr(), xs.data_ptr(), m, C.byref(kern), _theta(theta),
                                tol, C.byref(o) if o else None, _stream(), method, mean.data_ptr(), wp, q, sp))
    return mean, (S.t() if S is not None else None)


class GPLogLikelihood(torch.autograd.Function):
    """Differentiable Gaussian-process log-likelihood in theta = (l, s2, nug).

    forward: RSF of Sigma, l = -z^T F^-1 z / 2 - log|F| / 2 - n/2 log 2pi;
    backward: the score from the peeled traces and a second solve
    (Algorithm 1), times the incoming gradient.  theta is a float64 CPU
    tensor; points and z are float64 CUDA tensors (constants)."""

    @staticmethod
    def forward(ctx, theta, points, z, family, alpha, tol_fact, tol_peel, o):
        F = Factorization(points, family, theta.detach().cpu(), SIGMA, tol_fact, alpha, o)
        ll, _, a = F.loglik(z)
        ctx.F, ctx.a, ctx.tols, ctx.o = F, a, (tol_fact, tol_peel), o
        return torch.tensor(ll, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_out):
        g, _ = ctx.F.score(ctx.a, ctx.tols[0], ctx.tols[1], ctx.o)
        ctx.F = None
        return grad_out * g, None, None, None, None, None, None, None


def gp_loglik(theta, points, z, family=MATERN32, alpha=0.0, tol_fact=1e-9, tol_peel=1e-6, o=None):
    return GPLogLikelihood.apply(theta, points, z, family, alpha, tol_fact, tol_peel, o)
