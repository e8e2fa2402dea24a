"""The batched-GEMM engines behind the solves and the peeling (Sec. 2.3.2
applies and solves, Sec. 3 products), checked element by element through
the C ABI (rsf_selftest_gemm) against NumPy's fp64 product.

Engines 1 and 3 multiply df64 operands on the tensor cores from exact bf16
slices (seven per operand, exact fp32 accumulation per diagonal of slice
products; engine 1 slices every operand once into work buffers with one
power of two per row and superblock of 384 terms, engine 3 slices inside the
GEMM per K-block of 64).  Their results must match the exact product to the df64
rounding of the operands: each operand is rounded to a 48-bit significand
(relative 2^-48 = 3.6e-15) and the slices keep 7 x 7 bits below the block's
largest power of two, so |C - AB| <= 1e-13 sum_k |A_ik||B_kj| + the same
bound on the beta C term (measured 1.6e-15 to 1e-14).  Engine 2 (df64 on
the CUDA cores) accumulates its rounding errors in one fp32 word, so its
bar is 5e-13 (measured up to 1.8e-13 at k = 1000); engine 0 (fp64) meets the
classical k u.  Shapes span several tiles with ragged
tails in m, n and k, more than one K-block, transposed operands, and rows
and columns whose magnitudes differ by up to 1e6 (one power of two per row
and K-block must still leave every element its full precision relative to
the largest one).
"""
import numpy as np
import pytest

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


def _mats(m, n, k, ta, tb, seed, spread):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, k)) * 10.0 ** rng.uniform(-spread, spread, (m, 1))
    Bm = rng.standard_normal((k, n)) * 10.0 ** rng.uniform(-spread, spread, (1, n))
    C = rng.standard_normal((m, n))
    return (A.T.copy() if ta else A), (Bm.T.copy() if tb else Bm), C, A, Bm


# (m, n, k) of C = op(A) op(B); the library sees the column-major transpose,
# whose row count is n: n >= 64 runs on the tensor cores, n < 64 on engine 2.
SHAPES = [(128, 64, 32), (200, 70, 45), (129, 33, 1), (300, 130, 1000), (1000, 257, 384), (64, 200, 17),
          (513, 64, 385), (40, 100, 50), (20, 150, 64)]


@pytest.mark.parametrize("engine", [1, 3, 2, 0])
@pytest.mark.parametrize("shape", SHAPES)
def test_engine_matches_numpy(B, engine, shape):
    m, n, k = shape
    for ta, tb, alpha, beta, spread in ((0, 0, 1.0, 0.0, 0.0), (1, 0, -1.0, 1.0, 3.0), (0, 1, 0.5, 1.0, 3.0),
                                        (1, 1, 1.0, -2.0, 1.0)):
        Aop, Bop, C, A, Bm = _mats(m, n, k, ta, tb, 1000 * m + 10 * n + k + 3 * ta + tb, spread)
        T = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")  # noqa: E731
        got = B.selftest_gemm(engine, T(Aop), T(Bop), T(C), bool(ta), bool(tb), alpha, beta).cpu().numpy()
        ref = alpha * (A @ Bm) + beta * C
        bound = abs(alpha) * (np.abs(A) @ np.abs(Bm)) + abs(beta) * np.abs(C)
        err = np.max(np.abs(got - ref) / bound)
        print(f"engine {engine} {shape} ta={ta} tb={tb}: max |err| / (|A||B| + |C|) = {err:.3e}")
        # fp64: k u (the classical bound); tensor cores: 1e-13 (exact within a
        # K-block, one df64 addition per block); df64 on the CUDA cores: its
        # fp32 error accumulator grows with k (measured up to 1.8e-13)
        bar = {0: 2.3e-16 * max(k, 2), 1: 1e-13, 2: 5e-13, 3: 1e-13}[engine]
        assert err <= bar


@pytest.mark.parametrize("engine", [1, 3, 2, 0])
def test_engine_without_k_terms_scales_c(B, engine):
    # K = 0 through the C ABI: nothing to multiply, C = beta C (df64 engines:
    # to the rounding of C to a df64 pair)
    import ctypes
    m, n = 200, 130
    rng = np.random.default_rng(7)
    C0 = rng.standard_normal((n, m))   # row-major n x m = column-major m x n
    A = torch.zeros(m, dtype=torch.float64, device="cuda")   # lda = m, no columns read
    Bb = torch.zeros(n, dtype=torch.float64, device="cuda")  # ldb = 1, k = 0 rows per column
    for beta in (0.0, 0.5, -2.0):
        C = torch.tensor(C0, dtype=torch.float64, device="cuda")
        st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        assert B.lib().rsf_selftest_gemm(engine, m, n, 0, 0, 0, 1.0, A.data_ptr(), m, Bb.data_ptr(), 1, beta,
                                         C.data_ptr(), m, st) == 0
        got = C.cpu().numpy()
        assert np.all(np.abs(got - beta * C0) <= 1e-14 * np.abs(C0))
