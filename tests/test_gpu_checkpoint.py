"""Checkpoint / resume through the C ABI: populations read with
lbm_get_populations and written into a fresh lattice with
lbm_set_populations continue bit for bit like the uninterrupted run."""
import numpy as np
import pytest

import paper_1703_00185_gb300 as lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_00185_gb300 import _build
    _build.build()
    lbm.load_library()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32-df"])
@pytest.mark.parametrize("kernel", ["fused", "separate"])
def test_resume_is_bit_identical(precision, kernel):
    kw = dict(tau=0.9, g0=2e-4, T_bot=1.4, precision=precision, kernel=kernel, device="cuda:0")
    a = lbm.Lattice(90, 70, **kw)
    a.init_rayleigh_taylor(5)
    a.step(10)
    b = lbm.Lattice(90, 70, **kw)
    b.init_rayleigh_taylor(5)
    b.step(4)
    snapshot = b.populations()
    b.close()
    c = lbm.Lattice(90, 70, **kw)
    c.set_populations(snapshot)
    c.step(6)
    assert np.array_equal(a.populations(), c.populations())
    for x, y in zip(a.fields(), c.fields()):
        assert np.array_equal(x, y)
