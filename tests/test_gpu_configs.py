"""The batched and served forms against the FP64 CPU oracle directly.

The other batched and serving tests hold every lattice's result bit-identical
to the same lattice stepped alone; here lattices drawn by the workload
generators themselves (the 64-lattice batch's sizes, seeds and bottom-wall
temperatures; a scaled-down serving trace) are run through the batched
single launch and through the server, and their fields are compared with the
oracle's: per field max |a - b| / max |b| <= 1e-12 (u over both components).
"""
import numpy as np
import pytest

import oracle
import paper_1703_00185_gb300 as lbm
from paper_1703_00185_gb300 import serving, workloads

pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_00185_gb300 import _build
    _build.build()
    lbm.load_library()


def rel_field_errors(a, b):
    return tuple(float(np.max(np.abs(x - y)) / np.max(np.abs(y))) for x, y in zip(a, b))


def oracle_fields(Lx, Ly, seed, T_bot, steps):
    o = oracle.Lattice(Lx, Ly, tau=0.8, g0=1e-4, T_top=0.5, T_bot=T_bot)
    o.init_rayleigh_taylor(seed)
    o.run(steps)
    return o.fields()


def test_batched_workload_lattices_against_oracle():
    """The three smallest lattices of the 64-lattice workload, advanced 100 steps
    together by the split single launch (one kernel per step)."""
    import torch
    jobs = sorted(workloads.batched_lattices(1, 64), key=lambda j: j["Lx"] * j["Ly"])[:3]
    lats = []
    for j in jobs:
        lat = lbm.Lattice(j["Lx"], j["Ly"], tau=0.8, g0=1e-4, T_top=0.5, T_bot=j["T_bot"], device="cuda:0")
        lat.init_rayleigh_taylor(j["seed"])
        lats.append(lat)
    b = lbm.Batch(lats, stream=torch.cuda.Stream(device="cuda:0"))
    b.set_config(256, 0)
    b.step(100)
    b.synchronize()
    assert b.launch_count == 100
    b.close()
    for j, lat in zip(jobs, lats):
        errs = rel_field_errors(lat.fields(), oracle_fields(j["Lx"], j["Ly"], j["seed"], j["T_bot"], 100))
        assert max(errs) <= FIELD_TOL, (j, errs)


def test_served_jobs_against_oracle():
    """FP64 jobs of a scaled-down serving trace (sizes / 8, 100-300 steps),
    served side by side with FP32-storage jobs under a budget that makes jobs
    queue, each compared with the oracle."""
    trace = workloads.serving_trace(4, rate=200.0, n_jobs=10, size_scale=0.125, steps=(100, 300))
    need = max(lbm.lbm_required_bytes(j["Lx"], j["Ly"], lbm.lbm_default_params()) for j in trace)
    summary, results = serving.run_trace(trace, budget_bytes=4 * need, max_steps_per_tick=16, keep_results=True)
    assert summary["completed"] == len(trace)
    checked = 0
    for j in trace:
        if j["precision"] != "fp64":
            continue
        errs = rel_field_errors(results[j["id"]], oracle_fields(j["Lx"], j["Ly"], j["seed"], j["T_bot"], j["steps"]))
        assert max(errs) <= FIELD_TOL, (j, errs)
        checked += 1
    assert checked >= 2
