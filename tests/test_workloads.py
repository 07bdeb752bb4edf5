"""The seeded workload generators (no GPU): the batched 64-lattice workload
and the serving traces match the recipes the benchmark states, and are
reproducible from their master seed."""
import numpy as np

from paper_1703_00185_gb300 import workloads


def test_batched_lattices_recipe():
    jobs = workloads.batched_lattices(1, 64)
    assert len(jobs) == 64
    assert sum(j["Lx"] * j["Ly"] for j in jobs) == 42_270_720  # the batched workload's site count
    assert {j["Lx"] for j in jobs} <= set(range(128, 1025, 128))
    assert {j["Ly"] for j in jobs} <= set(range(256, 2049, 256))
    assert all(1.2 <= j["T_bot"] < 1.8 for j in jobs)
    assert len({j["seed"] for j in jobs}) == 64
    assert jobs == workloads.batched_lattices(1, 64)
    assert jobs != workloads.batched_lattices(2, 64)


def test_serving_trace_recipe():
    trace = workloads.serving_trace(1, rate=50.0, n_jobs=2000)
    t = np.array([j["arrival"] for j in trace])
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0)
    # Poisson arrivals: mean gap 1 / rate (2000 gaps: standard error ~2 %)
    assert abs(np.diff(t).mean() - 1 / 50.0) < 0.1 / 50.0
    Lx = np.array([j["Lx"] for j in trace])
    Ly = np.array([j["Ly"] for j in trace])
    assert np.all(Lx % 8 == 0) and np.all(Ly % 8 == 0)
    assert Lx.min() >= 64 and Lx.max() <= 2048 and Ly.min() >= 64 and Ly.max() <= 4096
    # log-uniform: the median near the geometric mean of the range
    assert abs(np.log(np.median(Lx)) - 0.5 * np.log(64 * 2048)) < 0.15
    steps = np.array([j["steps"] for j in trace])
    assert steps.min() >= 100 and steps.max() <= 5000
    prec = [j["precision"] for j in trace]
    assert set(prec) == {"fp64", "fp32-df"} and abs(prec.count("fp64") / len(prec) - 0.5) < 0.05
    assert [j["id"] for j in trace] == list(range(2000))
    assert trace == workloads.serving_trace(1, rate=50.0, n_jobs=2000)


def test_serving_trace_size_scale():
    full = workloads.serving_trace(3, n_jobs=500)
    quarter = workloads.serving_trace(3, n_jobs=500, size_scale=0.25)
    ratio = np.median([q["Lx"] * q["Ly"] for q in quarter]) / np.median([f["Lx"] * f["Ly"] for f in full])
    assert 0.04 < ratio < 0.09  # sites scale by about 0.25^2
    assert all(q["Lx"] >= 8 and q["Lx"] % 8 == 0 for q in quarter)
