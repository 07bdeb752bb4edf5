"""The roofline entry bench.py prints (no GPU): the keys of the JSON contract
and its arithmetic, achieved = algorithmic bytes per step / time per step,
frac = achieved / peak, with the FP64-pipe and oracle-flop sides beside it."""
import os
import sys

import pytest

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), ".."))
import bench  # noqa: E402


@pytest.fixture
def peaks(monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: {"hbm_gbs": 6775.3})


def test_fp64_fused_entry(peaks):
    sites, step_s = 2048 * 8192, 2.7e-3
    r = bench.roofline_of("fused", step_s, sites, "fp64", traffic=9.78e9)
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in r
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6775.3
    gbs = 592 * sites / step_s / 1e9
    assert r["achieved"] == pytest.approx(gbs, abs=0.05)
    assert r["frac"] == pytest.approx(gbs / 6775.3, abs=1e-4)
    assert r["algorithmic_bytes_per_launch"] == 592 * sites
    fp = r["fp64_pipe"]
    assert fp["inst_per_site"] == bench.FP64_PIPE_INST_PER_SITE
    assert fp["achieved"] == pytest.approx(bench.FP64_PIPE_INST_PER_SITE * sites / step_s / 1e9, abs=0.01)
    assert fp["peak"] == pytest.approx(2 * 152 * 2.07, abs=0.01)
    assert r["oracle_flops"]["tensor_form_flops_per_site"] == bench.ORACLE_FLOPS_PER_SITE
    assert r["oracle_flops"]["contracted_flops_per_site"] == bench.ORACLE_CONTRACTED_FLOPS_PER_SITE
    # both terms of min(HBM / bytes, FP64 peak / flops)
    b = r["bounds"]
    assert b["hbm_gsites_per_s"] == pytest.approx(6775.3 / 592, abs=1e-3)
    flop = 2 * 2 * 152 * 2.07e9 / bench.ORACLE_CONTRACTED_FLOPS_PER_SITE / 1e9
    assert b["fp64_flop_gsites_per_s"] == pytest.approx(flop, abs=1e-4)
    assert b["min_gsites_per_s"] == pytest.approx(min(6775.3 / 592, flop), abs=1e-4)
    assert b["achieved_gsites_per_s"] == pytest.approx(sites / step_s / 1e9, abs=1e-4)


def test_fp32_entry_has_no_fp64_sides(peaks):
    r = bench.roofline_of("fused", 1e-3, 1000, "fp32-df")
    assert r["achieved"] == pytest.approx(296 * 1000 / 1e-3 / 1e9, abs=0.05)
    assert "fp64_pipe" not in r and "oracle_flops" not in r and r["traffic"] is None


def test_without_measured_peaks(monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: {})
    r = bench.roofline_of("fused", 1e-3, 1000, "fp64")
    assert r["peak"] is None and r["frac"] is None


def test_whole_job_rate():
    # sites x ranks x steps / seconds, in millions
    assert bench.whole_job_mlups(1000, 4, 10, 2.0) == pytest.approx(1000 * 4 * 10 / 2e-3 / 1e6)
