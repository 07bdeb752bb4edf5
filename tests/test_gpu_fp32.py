"""GPU checks of the FP32 deviation storage forms (populations stored as
d_l = f_l - w_l in FP32; rho, u, T and the temperature-dependent equilibrium
terms in FP64 or in double-float), through the C ABI.

Propagation only moves stored values, so it stays exact; whole steps carry
the FP32 storage rounding (2^-24 relative per stored value and step) and are
compared with the FP64 oracle by relative L2 error per field.
"""
import numpy as np
import pytest

import oracle
import paper_1703_00185_gb300 as lbm
from tests import synthetic

pytestmark = pytest.mark.gpu

FORMS = ["fp32", "fp32-df"]


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_00185_gb300 import _build
    _build.build()
    lbm.load_library()


@pytest.fixture(scope="module")
def perm():
    cx, cy = lbm.lbm_velocity_set()
    ocx, ocy = oracle.velocity_set()
    idx = {(a, b): i for i, (a, b) in enumerate(zip(ocx.tolist(), ocy.tolist()))}
    return np.array([idx[(a, b)] for a, b in zip(cx.tolist(), cy.tolist())])


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("precision", FORMS)
def test_fp32_propagate_is_exact_permutation(precision):
    Lx, Ly = 19, 37
    g = lbm.Lattice(Lx, Ly, periodic_y=True, precision=precision, device="cuda:0")
    _, w = lbm.lbm_quadrature()
    g.set_populations(synthetic.random_populations(w, Lx, Ly, 5, rel_noise=0.2))
    f0 = g.populations()  # w + the stored FP32 deviations
    cx, cy = lbm.lbm_velocity_set()
    for k in range(1, 3):
        g.run_phases(1, lbm.PHASE_PROPAGATE)
        f = g.populations()
        for l in range(37):
            assert np.array_equal(f[l], np.roll(f0[l], (k * cx[l], k * cy[l]), axis=(0, 1)))


@pytest.mark.parametrize("precision", FORMS)
def test_fp32_storage_round_trip(precision):
    Lx, Ly = 24, 20
    g = lbm.Lattice(Lx, Ly, precision=precision, device="cuda:0")
    _, w = lbm.lbm_quadrature()
    f = synthetic.random_populations(w * 1.3, Lx, Ly, 6, rel_noise=0.2)
    g.set_populations(f)
    back = g.populations()
    d = f - w[:, None, None]
    # one FP32 rounding of the deviation
    assert np.all(np.abs(back - f) <= np.abs(d) * 2.0 ** -24 + 1e-18)


@pytest.mark.parametrize("precision", FORMS)
def test_fp32_fused_equals_separate(precision):
    a = lbm.Lattice(128, 96, kernel="separate", precision=precision, device="cuda:0")
    b = lbm.Lattice(128, 96, kernel="fused", precision=precision, device="cuda:0")
    for x in (a, b):
        x.init_rayleigh_taylor(2)
        x.step(20)
    assert np.array_equal(a.populations(), b.populations())


@pytest.fixture(scope="module")
def oracle_1000():
    """256 x 128 Rayleigh-Taylor, seed 1: oracle fields after 100 and 1000 steps."""
    o = oracle.Lattice(256, 128)
    o.init_rayleigh_taylor(1)
    o.run(100)
    f100 = o.fields()
    o.run(900)
    return {100: f100, 1000: o.fields()}


# Bars: measured errors times ~3.
ACC_BARS = {100: (2e-7, 5e-5, 2e-7), 1000: (1e-6, 1e-4, 1e-6)}


@pytest.mark.parametrize("precision", FORMS)
@pytest.mark.parametrize("steps", [100, 1000])
def test_fp32_accuracy_vs_fp64_oracle(precision, steps, oracle_1000):
    g = lbm.Lattice(256, 128, precision=precision, device="cuda:0")
    g.init_rayleigh_taylor(1)
    g.step(steps)
    errs = [rel_l2(a, b) for a, b in zip(g.fields(), oracle_1000[steps])]
    assert all(e <= bar for e, bar in zip(errs, ACC_BARS[steps])), (precision, steps, errs)


def test_fp32_wide_forms_agree():
    a = lbm.Lattice(200, 64, precision="fp32", device="cuda:0")
    b = lbm.Lattice(200, 64, precision="fp32-df", device="cuda:0")
    for x in (a, b):
        x.init_rayleigh_taylor(3)
        x.step(50)
    errs = [rel_l2(p, q) for p, q in zip(a.fields(), b.fields())]
    assert max(errs) < 1e-5, errs


@pytest.mark.parametrize("precision", FORMS)
def test_fp32_collide_near_oracle(precision, perm):
    """One collision from random near-equilibrium states: the FP32 result is
    within a few FP32 roundings of the FP64 oracle, per population plane."""
    Lx, Ly = 37, 45
    o = oracle.Lattice(Lx, Ly, tau=0.8, g0=1e-3)
    rho, ux, uy, T = synthetic.random_fields(Lx, Ly, 11)
    o.set_equilibrium(rho, ux, uy, T)
    f = o.populations() * (1.0 + 0.02 * (2.0 * np.random.default_rng(3).random((37, Lx, Ly)) - 1.0))
    g = lbm.Lattice(Lx, Ly, tau=0.8, g0=1e-3, precision=precision, device="cuda:0")
    g.set_populations(f[perm])
    o.set_populations(g.populations()[np.argsort(perm)])  # the same FP32-rounded input
    o.run(1, oracle.PHASE_COLLIDE)
    g.run_phases(1, lbm.PHASE_COLLIDE)
    a, b = g.populations(), o.populations()[perm]
    err = np.max(np.abs(a - b).reshape(37, -1), axis=1) / np.max(np.abs(b).reshape(37, -1), axis=1)
    assert err.max() < 1e-6, err.max()


@pytest.mark.parametrize("precision", FORMS)
def test_fp32_full_size_mass(precision):
    """2048 x 8192 in the bench schedule: 10 steps, global mass kept to FP32
    storage accuracy."""
    g = lbm.Lattice(2048, 8192, precision=precision, device="cuda:0")
    g.init_rayleigh_taylor(1)
    m0 = g.fields()[0].sum()
    g.step(10)
    rho, u, T = g.fields()
    assert np.isfinite(rho).all() and np.isfinite(u).all() and np.isfinite(T).all()
    assert abs(rho.sum() / m0 - 1.0) < 1e-7
