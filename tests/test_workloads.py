"""The seeded workload descriptions (random draws and layouts only): every
named workload builds its point set with the stated size, and the paper's
gridded experiments (Sec. 5.1) are sqrt(n) x sqrt(n) grids of [0, 100]^2 with
the anisotropic theta = (l1, s2, nug, l2) = (10, 1, 1e-4, 7)."""
import numpy as np
import pytest

from paper_1603_08057_gb300 import workloads as W


@pytest.mark.parametrize("name", sorted(W.WORKLOADS))
def test_workload_points(name):
    wl = W.WORKLOADS[name]
    n = 4096 if wl["points"] != "grid" else 64 * 64
    x = W.make_points(wl["points"], n, wl["seed_points"])
    assert x.shape == (n, 2) and np.all(np.isfinite(x))
    assert len(wl["theta"]) in (3, 4)


def test_grid_workloads_are_the_papers():
    for name in ("matern32_grid_aniso_n262144", "rq_half_grid_aniso_n262144"):
        wl = W.WORKLOADS[name]
        assert wl["n"] == 512 * 512 and wl["theta"] == (10.0, 1.0, 1e-4, 7.0)
        assert wl["tol_fact"] == pytest.approx(wl["tol_peel"] / 1000, rel=1e-12)
    x = W.make_points("grid", 64 * 64, 0)
    assert x.min() > 0.0 and x.max() < 100.0
    assert len(np.unique(x[:, 0])) == 64 and len(np.unique(x[:, 1])) == 64
    with pytest.raises(ValueError):
        W.make_points("grid", 1000, 0)
