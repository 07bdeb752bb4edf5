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


def test_oracle_errors_metric():
    """bench.oracle_errors: per field max |a - b| / max |b| over the stored sites
    and the row and column means (u over both components), and the relative L2
    error over the stored sites, on a made-up state and stored summary."""
    import numpy as np
    rng = np.random.default_rng(5)
    Lx, Ly, n = 6, 10, 7
    ref = {"rho": rng.uniform(0.5, 2.0, (Lx, Ly)), "ux": rng.normal(0, 1e-2, (Lx, Ly)),
           "uy": rng.normal(0, 1e-2, (Lx, Ly)), "T": rng.uniform(0.5, 1.5, (Lx, Ly))}
    sx, sy = np.array([0, 5, 2, 3]), np.array([9, 0, 4, 4])
    z = {"sample_x": sx, "sample_y": sy,
         "n7_max_abs": np.array([np.abs(ref["rho"]).max(), max(np.abs(ref["ux"]).max(), np.abs(ref["uy"]).max()),
                                 np.abs(ref["T"]).max()])}
    for k, v in ref.items():
        z["n7_%s_sample" % k], z["n7_%s_rowmean" % k], z["n7_%s_colmean" % k] = v[sx, sy], v.mean(0), v.mean(1)
    got = {k: v.copy() for k, v in ref.items()}
    got["T"][2, 4] += 1e-9  # a stored site
    got["uy"][1, 1] += 3e-9  # seen only through its row and column means
    e = bench.oracle_errors(got["rho"], np.stack([got["ux"], got["uy"]]), got["T"], z, n)
    assert e["max_rel"]["rho"] == 0.0
    assert e["max_rel"]["T"] == pytest.approx(1e-9 / z["n7_max_abs"][2], rel=1e-6)
    assert e["max_rel"]["u"] == pytest.approx(3e-9 / Lx / z["n7_max_abs"][1], rel=1e-6)  # the row mean
    t = ref["T"][sx, sy]
    assert e["rel_l2_sample"]["T"] == pytest.approx(1e-9 / np.sqrt((t ** 2).sum()), rel=1e-6)
    assert e["rel_l2_sample"]["u"] == 0.0
