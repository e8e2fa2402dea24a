"""The staged-tolerance driver (dynamic tolerances, Sec. 6) on CPU: with the
per-stage L-BFGS stubbed, the stages run in order at their tolerances, each
starts from the previous stage's theta, and the totals add up."""
import pytest

pytest.importorskip("torch")


def test_stages_chain_and_tighten(monkeypatch):
    from paper_1603_08057_gb300 import mle
    calls = []

    def fake_fit(points, z, family, theta, alpha, tol_fact, tol_peel, o, max_iter, history_size):
        calls.append((tuple(theta), tol_fact, tol_peel, max_iter))
        new = [t * 0.5 for t in theta]
        return new, {"evals": max_iter + 1, "seconds": 0.25, "loglik": -1.0 / tol_peel, "trace": []}

    monkeypatch.setattr(mle, "fit", fake_fit)
    th, info = mle.fit_staged(None, None, 0, (0.2, 0.5, 0.1))
    assert [c[1:] for c in calls] == [s for s in mle.DEFAULT_STAGES]
    assert calls[0][0] == (0.2, 0.5, 0.1)
    assert calls[1][0] == pytest.approx((0.1, 0.25, 0.05)) and calls[2][0] == pytest.approx((0.05, 0.125, 0.025))
    assert th == pytest.approx([0.025, 0.0625, 0.0125])
    assert info["evals"] == sum(s[2] + 1 for s in mle.DEFAULT_STAGES) and info["seconds"] == pytest.approx(0.75)
    assert info["loglik"] == pytest.approx(-1e6)
    assert [s["tol_peel"] for s in info["stages"]] == [1e-4, 1e-5, 1e-6]
    # tolerances only tighten, ending at the paper's pairing
    tf = [s[0] for s in mle.DEFAULT_STAGES]
    assert tf == sorted(tf, reverse=True) and mle.DEFAULT_STAGES[-1][:2] == (1e-9, 1e-6)
