"""Failure detection without a GPU fault: bounded device waits.

Every device-side wait of the library is bounded.  The grid barrier of the
persistent pivoted-QR kernel gives up after a few seconds and records
RSF_ETIMEOUT in the status word that the host reads after the launch.
rsf_selftest_wait_limit runs that barrier with one participant more than it
launches, so nothing can end the wait: the test checks that the call
returns in bounded time with the timeout reported, and that the CUDA
context is still usable afterwards (a factorization and solve succeed).
"""
import time

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


def test_bounded_wait_gives_up_and_reports(B):
    t0 = time.time()
    B.selftest_wait_limit()
    assert time.time() - t0 < 60.0
    x = torch.tensor(W.uniform(800, 11), dtype=torch.float64, device="cuda")
    F = B.Factorization(x, B.MATERN32, (0.1, 1.0, 1e-2), B.SIGMA, 1e-9)
    v = torch.tensor(W.standard_normal(800, 12, 2), dtype=torch.float64, device="cuda")
    r = F.solve(F.solve(v, B.OP_APPLY), B.OP_INV)
    assert torch.max(torch.abs(r - v)).item() <= 1e-8 * torch.max(torch.abs(v)).item()
    assert np.isfinite(F.logdet())
