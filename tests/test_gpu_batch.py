"""GPU checks of batched stepping (many lattices, one launch per step, or one
launch per lattice in concurrent branches), through the C ABI: each
lattice's result is bit-identical to the same lattice stepped alone, for
every launch shape, and autotuning leaves the state alone."""
import numpy as np
import pytest

import paper_1703_00185_gb300 as lbm

pytestmark = pytest.mark.gpu

SIZES = [(128, 256), (37, 61), (256, 128), (5, 6), (300, 40)]


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_00185_gb300 import _build
    _build.build()
    lbm.load_library()


def make(precision, periodic_last=True, shared_tau=False):
    """Lattices of different sizes and wall temperatures; with shared_tau all
    have tau 0.8 and g0 1e-4 (the FP64 batch then takes the collision
    constants as one kernel argument), else tau differs per lattice."""
    lats = []
    for i, (Lx, Ly) in enumerate(SIZES):
        tau = 0.8 if shared_tau else 0.7 + 0.05 * i
        lat = lbm.Lattice(Lx, Ly, T_bot=1.2 + 0.1 * i, tau=tau, precision=precision, device="cuda:0",
                          periodic_y=(periodic_last and i == len(SIZES) - 1))
        lat.init_rayleigh_taylor(10 + i)
        lats.append(lat)
    return lats


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32-df"])
@pytest.mark.parametrize("config", [(128, 0), (64, 2), (256, 1), (0, 0)])
@pytest.mark.parametrize("shared_tau", [False, True])
def test_batch_equals_alone(precision, config, shared_tau):
    alone, batched = make(precision, shared_tau=shared_tau), make(precision, shared_tau=shared_tau)
    for lat in alone:
        lat.step(7)
    b = lbm.Batch(batched)
    b.set_config(*config)
    b.step(7)
    b.synchronize()
    # block_y 0: each lattice's fused step, in FP64 two kernels with walls (sites, wall bands)
    per_step = 1 if config[0] else sum(2 if precision == "fp64" and not lat.params.periodic_y else 1
                                       for lat in batched)
    assert b.launch_count == 7 * per_step
    for a, c in zip(alone, batched):
        assert np.array_equal(a.populations(), c.populations())
    # and the lattices continue correctly on their own handles afterwards
    b.close()
    for lat in alone + batched:
        lat.step(3)
    for a, c in zip(alone, batched):
        assert np.array_equal(a.populations(), c.populations())


@pytest.mark.parametrize("block_y", [64, 128, 256])
def test_split_single_launch_equals_alone(block_y):
    """FP64 lattices with walls and one tau and g: one block per tile runs the
    split form (site tiles and wall tiles in one launch), one kernel per step,
    and each lattice's result is bit-identical to the lattice stepped alone."""
    alone = make("fp64", periodic_last=False, shared_tau=True)
    batched = make("fp64", periodic_last=False, shared_tau=True)
    for lat in alone:
        lat.step(9)
    b = lbm.Batch(batched)
    b.set_config(block_y, 0)
    b.step(9)  # one direct step, then replays of the captured two-step graph
    b.synchronize()
    assert b.launch_count == 9
    for a, c in zip(alone, batched):
        assert np.array_equal(a.populations(), c.populations())
    b.close()


def test_autotune_keeps_state(tmp_path, monkeypatch):
    monkeypatch.setenv("D2Q37_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    lats = make("fp64")
    before = [lat.populations() for lat in lats]
    b = lbm.Batch(lats)
    res = b.autotune(trial_steps=2)
    assert res["block_y"] in (64, 128, 256) and res["ms_per_step"] > 0 and not res["cached"]
    b.synchronize()
    for lat, f in zip(lats, before):
        assert np.array_equal(lat.populations(), f)
    again = b.autotune(trial_steps=2)
    assert again["cached"] and (again["block_y"], again["blocks_per_sm"]) == (res["block_y"], res["blocks_per_sm"])
    assert b.config() == (res["block_y"], res["blocks_per_sm"])


def test_batch_rejects_bad_input():
    a = lbm.Lattice(16, 16, device="cuda:0")
    a.init_rayleigh_taylor(1)
    c = lbm.Lattice(16, 16, precision="fp32", device="cuda:0")
    c.init_rayleigh_taylor(1)
    with pytest.raises(lbm.LBMError):
        lbm.Batch([a, c])
    d = lbm.Lattice(16, 16, device="cuda:0")  # no state yet
    with pytest.raises(lbm.LBMError) as e:
        lbm.Batch([a, d])
    assert e.value.code == lbm.LBM_ESTATE
    b = lbm.Batch([a])
    with pytest.raises(lbm.LBMError):
        b.set_config(96, 0)
    with pytest.raises(lbm.LBMError):
        b.set_config(0, 1)  # the per-lattice form has no persistent grid
