"""GPU checks of the continuous-batching server (lbm_server_* through the C
ABI): a job's result is the same alone and in a mix of jobs of other sizes,
precisions and step counts that arrive while others are running, admission
respects the memory budget, and bad jobs are rejected."""
import numpy as np
import pytest

import paper_1703_00185_gb300 as lbm
from paper_1703_00185_gb300 import serving

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_00185_gb300 import _build
    _build.build()
    lbm.load_library()


def small_trace(n=12, seed=3):
    rng = np.random.default_rng(seed)
    return [{"id": i, "arrival": 0.02 * i, "Lx": int(rng.integers(3, 40) * 4), "Ly": int(rng.integers(2, 30) * 8),
             "steps": int(rng.integers(0, 60)), "precision": ["fp64", "fp32-df", "fp32"][i % 3],
             "seed": int(rng.integers(1, 1000)), "T_bot": float(rng.uniform(1.2, 1.8))} for i in range(n)]


def alone(job):
    lat = lbm.Lattice(job["Lx"], job["Ly"], T_bot=job["T_bot"], precision=job["precision"], device="cuda:0")
    lat.init_rayleigh_taylor(job["seed"])
    lat.step(job["steps"])
    return lat.fields()


def test_results_same_alone_and_in_mix():
    trace = small_trace()
    # a budget for a few jobs at a time: later arrivals wait for memory to free
    need = max(lbm.lbm_required_bytes(j["Lx"], j["Ly"], _params(j)) for j in trace)
    summary, results = serving.run_trace(trace, budget_bytes=3 * need + (1 << 20), max_steps_per_tick=7,
                                         keep_results=True)
    assert summary["completed"] == len(trace) and summary["rejected"] == 0
    for j in trace:
        ref = alone(j)
        for a, b in zip(results[j["id"]], ref):
            assert np.array_equal(a, b), j


def _params(j):
    p = lbm.lbm_default_params()
    p.precision = lbm.PRECISIONS[j["precision"]]
    return p


def test_budget_and_rejection():
    srv = serving.Server(budget_bytes=64 << 20, max_steps_per_tick=4)
    with pytest.raises(lbm.LBMError) as e:
        srv.submit(2048, 2048, 10)  # needs ~2.5 GB
    assert e.value.code == lbm.LBM_ENOMEM
    with pytest.raises(lbm.LBMError):
        srv.submit(2, 64, 10)
    ids = [srv.submit(96, 96, 5 + i, "fp64" if i % 2 else "fp32-df", seed=i) for i in range(8)]
    seen_in_use = []
    while srv.stats()["completed"] < len(ids):
        srv.tick()
        st = srv.stats()
        seen_in_use.append(st["bytes_in_use"])
        assert st["bytes_in_use"] <= st["budget_bytes"]
    done = []
    while True:
        got = srv.poll()
        if not got:
            break
        done += got
    assert sorted(done) == ids
    for jid in ids:
        assert srv.state(jid)[0] == lbm.JOB_DONE
        rho, u, T = srv.fetch(jid)
        assert np.isfinite(rho).all()
    assert srv.stats()["bytes_in_use"] == 0
    srv.close()
