"""rsf_set_allocator: the library's device memory from PyTorch's caching allocator.

The hook has no counterpart in the paper; it lets the library live inside a
PyTorch program's memory pool.  Checked through the C ABI: with the hook
installed every buffer comes from the torch pool (its allocation counter
grows, a live factorization holds torch memory and returns it when
destroyed) and the results are bitwise those of the default allocator (the
arithmetic does not depend on where the buffers live).
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


def test_torch_allocator_backs_the_library(B):
    x = T(W.mixture(3000, 401))
    z = T(W.standard_normal(3000, 402))
    th = (0.05, 2.0, 1e-2)
    ll0, g0, t0 = B.loglik_and_score(x, z, B.MATERN32, th, 1e-9, 1e-6)
    torch.cuda.synchronize()
    count0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    B.use_torch_allocator(True)
    try:
        ll1, g1, t1 = B.loglik_and_score(x, z, B.MATERN32, th, 1e-9, 1e-6)
        torch.cuda.synchronize()
        base = torch.cuda.memory_allocated()
        F = B.Factorization(x, B.MATERN32, th, B.SIGMA, 1e-9)
        torch.cuda.synchronize()
        held = torch.cuda.memory_allocated()
        y = F.solve(z.reshape(-1, 1), B.OP_INV)
        del F
        torch.cuda.synchronize()
        after = torch.cuda.memory_allocated() - y.numel() * 8
    finally:
        B.use_torch_allocator(False)
    count1 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    assert count1 > count0 + 100
    assert held > base
    assert after <= base
    assert ll1 == ll0
    assert torch.equal(g1, g0) and torch.equal(t1, t0)


def test_allocator_hook_arguments(B):
    # one of the two functions missing: RSF_EINVAL, the setting is unchanged
    keep = B._ALLOC_FN(lambda n, s, c: None)
    assert B.lib().rsf_set_allocator(keep, B._FREE_FN(), None) == 1


def test_failing_hook_reports_enomem(B):
    keep = (B._ALLOC_FN(lambda n, s, c: None), B._FREE_FN(lambda p, n, s, c: None))
    B._check(B.lib().rsf_set_allocator(keep[0], keep[1], None))
    try:
        with pytest.raises(B.RsfError) as e:
            B.Factorization(T(W.uniform(500, 403)), B.MATERN32, (0.1, 1.0, 1e-2))
        assert e.value.code == 2
    finally:
        B.use_torch_allocator(False)
