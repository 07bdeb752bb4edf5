"""GPU test of lbm_batch_step_static: the batched step for callers that cannot
call cudaMalloc (device memory owned by a caching allocator or a registered
pool, loops that must not synchronise the device).  Through the C ABI, two
calls in a row must give the same populations as the allocating batched entry
point (lbm_batch_*), bit for bit as the other batched tests require, while the
device's free memory stays the same; a call with more lattices than the fixed
table holds, and a call on a stream that is capturing, must be refused.

Kept in a file of its own, collected last."""
import numpy as np
import pytest

import paper_1703_00185_gb300 as lbm

pytestmark = pytest.mark.gpu

SIZES = [(64, 96), (37, 61), (130, 40), (5, 6)]


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_00185_gb300 import _build
    _build.build()
    lbm.load_library()


def make(precision):
    lats = []
    for i, (Lx, Ly) in enumerate(SIZES):
        lat = lbm.Lattice(Lx, Ly, T_bot=1.3 + 0.1 * i, tau=0.75 + 0.05 * i, precision=precision, device="cuda:0")
        lat.init_rayleigh_taylor(20 + i)
        lats.append(lat)
    return lats


@pytest.mark.parametrize("precision", ["fp64", "fp32-df"])
def test_static_batch_matches_allocating_batch(precision):
    import torch
    ref, stat = make(precision), make(precision)
    batch = lbm.Batch(ref)  # allocates its tile table with cudaMalloc
    stream = torch.cuda.Stream(device="cuda:0")
    for steps in (3, 4):  # two calls in a row, reusing the static table
        batch.step(steps)
        batch.synchronize()
        for lat in stat:
            lat.synchronize()
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info(0)[0]
        lbm.lbm_batch_step_static([lat._h for lat in stat], steps, stream.cuda_stream)
        stream.synchronize()
        assert torch.cuda.mem_get_info(0)[0] == free0  # nothing allocated on the device
        for a, b in zip(ref, stat):
            assert np.array_equal(a.populations(), b.populations())
    batch.close()


def test_static_batch_refuses_too_many_lattices():
    import torch
    lat = lbm.Lattice(16, 16, device="cuda:0")
    lat.init_rayleigh_taylor(1)
    before = lat.populations()
    stream = torch.cuda.Stream(device="cuda:0")
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_batch_step_static([lat._h] * (lbm.LBM_STATIC_BATCH_MAX + 1), 2, stream.cuda_stream)
    assert e.value.code == lbm.LBM_ETOOBIG
    assert "static table" in lbm.lbm_strerror(lbm.LBM_ETOOBIG)
    assert np.array_equal(lat.populations(), before)


@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")
def test_static_batch_refuses_a_capturing_stream():
    import torch
    lat = lbm.Lattice(16, 16, device="cuda:0")
    lat.init_rayleigh_taylor(1)
    lat.synchronize()
    before = lat.populations()
    stream = torch.cuda.Stream(device="cuda:0")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        with pytest.raises(lbm.LBMError) as e:
            lbm.lbm_batch_step_static([lat._h], 2, stream.cuda_stream)
    assert e.value.code == lbm.LBM_EINVAL
    assert np.array_equal(lat.populations(), before)
