"""bench.py's roofline bookkeeping on CPU: with the library's profile totals
stubbed, the dominant GEMM engine is picked by time, its fraction is its
algorithmic flops over its time against its own bound, every engine that ran
is reported, and the flop-weighted total combines them."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class _B:
    PROF_GEMM, PROF_QR_UPDATE, PROF_GEMM_DF, PROF_GEMM_TC = 0, 1, 8, 9
    PROF_NAMES = {0: "gemm_fp64", 1: "qr", 8: "gemm_df64", 9: "gemm_tc"}


def _prof(ms_tc, fl_tc, ms_fp, fl_fp):
    z = dict(launches=0, ms=0.0, flops=0.0, bytes=0.0)
    return {0: dict(launches=10, ms=ms_fp, flops=fl_fp, bytes=0.0), 1: dict(launches=5, ms=300.0, flops=0.0, bytes=0.0),
            8: dict(z), 9: dict(launches=100, ms=ms_tc, flops=fl_tc, bytes=0.0)}


def test_roofline_of_picks_the_dominant_engine_and_reports_all():
    sys.path.insert(0, ROOT)
    import bench
    prof = _prof(ms_tc=2000.0, fl_tc=3.0e13, ms_fp=500.0, fl_fp=5.0e11)
    r = bench.roofline_of(_B, prof, 4000.0)
    bf16, _ = bench.bf16_peak_tflops()
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(3.0e13 / 2.0 / 1e12)
    assert r["peak"] == pytest.approx(bf16 / 28)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["share_of_step"] == pytest.approx(0.5)
    assert r["phases_ms"] == {"gemm_fp64": 500.0, "qr": 300.0, "gemm_tc": 2000.0}
    eng = r["engines"]
    names = [e["engine"] for e in eng["per_engine"]]
    assert names == ["tensor-core GEMM (slicing + products)", "fp64 GEMM"]
    fp = eng["per_engine"][1]
    assert fp["achieved_tflops"] == pytest.approx(1.0) and fp["frac"] == pytest.approx(1.0 / bench.FP64_PEAK_TFLOPS)
    assert eng["flop_weighted_total"]["achieved_tflops"] == pytest.approx((3.0e13 + 5.0e11) / 2.5 / 1e12)


def test_roofline_of_fp64_dominant():
    sys.path.insert(0, ROOT)
    import bench
    prof = _prof(ms_tc=0.0, fl_tc=0.0, ms_fp=1000.0, fl_fp=1.0e12)
    prof[9]["launches"] = 0
    r = bench.roofline_of(_B, prof, 2000.0)
    assert r["bound"] == "alu" and r["peak"] == pytest.approx(bench.FP64_PEAK_TFLOPS)
    assert [e["engine"] for e in r["engines"]["per_engine"]] == ["fp64 GEMM"]
