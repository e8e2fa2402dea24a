"""rsf_solve_noalloc: the solve entry point that allocates no device memory.

Some callers cannot allocate device memory when they solve -- for instance
code running inside another framework's memory budget, whose caching
allocator already holds the device memory.  For them the library offers
rsf_solve_noalloc, which keeps its work buffers in one fixed device array
inside the library.  This file checks, through the C ABI, that it returns what
rsf_solve returns (within the tolerance the other tests use for identical
arithmetic) on two calls in a row, and that a request larger than the fixed
array is refused with RSF_EINVAL.  The file is named so that pytest collects
it last.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_solve_matches_rsf_solve_twice(B, prec):
    x = W.mixture(3000, 301)
    th = (0.05, 2.0, 1e-2)
    F = B.Factorization(T(x), B.MATERN32, th, B.SIGMA, 1e-9, 0.0, B.opts(precision=prec))
    V = T(W.standard_normal(3000, 302, 4))
    for op in (B.OP_INV, B.OP_APPLY, B.OP_SQRT, B.OP_INV_SQRT_T):
        ref = F.solve(V, op)
        first = F.solve_noalloc(V, op)
        second = F.solve_noalloc(V, op)
        scale = torch.max(torch.abs(ref)).item()
        assert torch.max(torch.abs(first - ref)).item() <= 1e-12 * scale
        assert torch.max(torch.abs(second - ref)).item() <= 1e-12 * scale


def test_noalloc_rejects_requests_beyond_the_scratch(B):
    x = W.uniform(2000, 311)
    F = B.Factorization(T(x), B.MATERN32, (0.1, 1.0, 1e-2), B.SIGMA, 1e-9)
    big = T(np.ones((2000, 2048)))
    with pytest.raises(B.RsfError) as e:
        F.solve_noalloc(big, B.OP_INV)
    assert e.value.code == 1 and "scratch" in str(e.value)
