"""Lattice-level pins of the oracle: propagate (P5), rest state (P6), mass with
walls and gravity (P7), mirror symmetry (P8), shear-wave viscosity (P10 i) and
brute force against the independent naive formulation (P10 ii)."""
import numpy as np
import pytest

import oracle
from oracle import naive
from tests import synthetic

Q = 37


def _naive_order(m):
    cx, cy = oracle.velocity_set()
    return np.array([list(zip(m.cx, m.cy)).index((a, b)) for a, b in zip(cx, cy)])


def _random_state(Lx, Ly, seed):
    _, w = oracle.scale_and_weights()
    return synthetic.random_populations(w, Lx, Ly, seed, rel_noise=0.1)


def test_propagate_periodic_is_roll():
    Lx, Ly = 11, 9
    f = _random_state(Lx, Ly, 1)
    lat = oracle.Lattice(Lx, Ly, periodic_y=True)
    lat.set_populations(f)
    lat.run(1, oracle.PHASE_PROPAGATE)
    g = lat.populations()
    cx, cy = oracle.velocity_set()
    for l in range(Q):
        assert np.array_equal(g[l], np.roll(f[l], (cx[l], cy[l]), axis=(0, 1)))
        assert np.array_equal(np.sort(g[l].ravel()), np.sort(f[l].ravel()))


def test_propagate_with_walls_leaves_missing_zero():
    Lx, Ly = 7, 10
    f = _random_state(Lx, Ly, 2)
    lat = oracle.Lattice(Lx, Ly)
    lat.set_populations(f)
    lat.run(1, oracle.PHASE_PROPAGATE)
    g = lat.populations()
    cx, cy = oracle.velocity_set()
    for l in range(Q):
        rolled = np.roll(f[l], cx[l], axis=0)
        for y in range(Ly):
            ys = y - cy[l]
            expect = rolled[:, ys] if 0 <= ys < Ly else np.zeros(Lx)
            assert np.array_equal(g[l, :, y], expect)


@pytest.mark.parametrize("Lx,Ly,periodic_y", [(8, 8, False), (16, 12, False), (8, 8, True), (5, 7, True)])
@pytest.mark.parametrize("phases", [1, 3, 4, 7])
def test_brute_force_against_naive(Lx, Ly, periodic_y, phases):
    m = naive.Model()
    order = _naive_order(m)
    inv = np.argsort(order)
    f0 = _random_state(Lx, Ly, 3)
    kw = dict(tau=0.7, g0=1e-3, T_top=0.6, T_bot=1.4)
    lat = oracle.Lattice(Lx, Ly, periodic_y=periodic_y, **kw)
    lat.set_populations(f0)
    fn = f0[inv]
    for _ in range(3):
        lat.run(1, phases)
        fn = m.step(fn, kw["tau"], kw["g0"], kw["T_top"], kw["T_bot"], periodic_y, phases)
    got = lat.populations()
    np.testing.assert_allclose(got, fn[order], rtol=1e-13, atol=1e-16)


def test_rest_state_stays_at_rest():
    Lx, Ly, T = 12, 16, 0.9
    lat = oracle.Lattice(Lx, Ly, tau=0.8, g0=0.0, T_top=T, T_bot=T)
    feq = oracle.equilibrium(1.3, 0.0, 0.0, T)
    f0 = np.repeat(np.repeat(feq[:, None, None], Lx, 1), Ly, 2)
    lat.set_populations(f0)
    lat.run(50)
    # FP64-rounded weights satisfy the moment conditions only to ~1e-16, so
    # every collision shifts rho and T by a systematic ~1e-16: allow 50 x 2e-15
    np.testing.assert_allclose(lat.populations(), f0, rtol=1e-13, atol=0)
    rho, u, Tf = lat.fields()
    assert np.abs(u).max() < 1e-15


def test_mass_conserved_with_walls_and_gravity():
    lat = oracle.Lattice(32, 24, tau=0.8, g0=1e-4)
    lat.init_rayleigh_taylor(5)
    m0 = lat.fields()[0].sum()
    lat.run(100)
    rho, u, T = lat.fields()
    # systematic ~1e-16 per collision from the rounded weights (see the rest-state test)
    assert abs(rho.sum() - m0) / m0 < 1e-13
    assert np.isfinite(u).all() and np.abs(u).max() > 0


def test_mirror_symmetry():
    Lx, Ly = 10, 12
    x = np.arange(Lx)[:, None] + 0.5
    y = np.arange(Ly)[None, :] + 0.5
    rho = 1.0 + 0.2 * np.cos(2 * np.pi * x / Lx) * np.sin(np.pi * y / Ly)
    ux = 0.02 * np.sin(2 * np.pi * x / Lx) * np.ones_like(y)
    uy = 0.01 * np.cos(2 * np.pi * x / Lx) * np.cos(np.pi * y / Ly)
    T = 1.0 + 0.1 * np.cos(4 * np.pi * x / Lx) * np.ones_like(y)
    f = np.zeros((Q, Lx, Ly))
    for i in range(Lx):
        for j in range(Ly):
            f[:, i, j] = oracle.equilibrium(rho[i, j], ux[i, j], uy[i, j], T[i, j])
    cx, cy = oracle.velocity_set()
    mirror = np.array([list(zip(cx, cy)).index((-a, b)) for a, b in zip(cx, cy)])
    # the initial state is mirror symmetric to round-off
    fm = f[mirror][:, ::-1, :]
    np.testing.assert_allclose(fm, f, rtol=1e-14)
    a, b = oracle.Lattice(Lx, Ly, g0=1e-3), oracle.Lattice(Lx, Ly, g0=1e-3)
    a.set_populations(f)
    b.set_populations(np.ascontiguousarray(fm))
    a.run(20)
    b.run(20)
    np.testing.assert_allclose(b.populations()[mirror][:, ::-1, :], a.populations(), rtol=1e-12, atol=1e-16)


def test_shear_wave_viscosity():
    """A small shear wave ux = A sin(k y) decays at nu k^2 with the BGK
    viscosity nu = c_s^2 (tau - 1/2), c_s^2 = T / s^2 in lattice units."""
    Lx, Ly, tau, T, A = 3, 128, 0.8, 1.0, 1e-5
    s, _ = oracle.scale_and_weights()
    y = np.arange(Ly) + 0.5
    k = 2 * np.pi / Ly
    ux = A * np.sin(k * y)
    f = np.zeros((Q, Lx, Ly))
    for j in range(Ly):
        f[:, :, j] = oracle.equilibrium(1.0, ux[j], 0.0, T)[:, None]
    lat = oracle.Lattice(Lx, Ly, tau=tau, g0=0.0, periodic_y=True)
    lat.set_populations(f)

    def amp():
        u = lat.fields()[1][0].mean(0)
        return 2.0 / Ly * np.sum(u * np.sin(k * y))

    lat.run(40)
    a1 = amp()
    lat.run(200)
    a2 = amp()
    nu_measured = -np.log(a2 / a1) / (200 * k * k)
    nu_theory = T / s ** 2 * (tau - 0.5)
    assert abs(nu_measured / nu_theory - 1.0) < 2e-3, (nu_measured, nu_theory)


def test_rt_temperature_recipe():
    Lx, Ly, seed = 64, 32, 9
    T = oracle.rt_temperature(Lx, Ly, seed, 0.5, 1.5)
    yi = 0.5 * Ly + Ly / 64.0 * np.sin(2 * np.pi * (np.arange(Lx) + 0.5) / Lx)
    hot = (np.arange(Ly)[None, :] + 0.5) < yi[:, None]
    T0 = np.where(hot, 1.5, 0.5)
    assert np.all(np.abs(T / T0 - 1.0) <= 1e-3)
    assert np.std(T / T0) > 1e-4
    # the perturbation is U(-1e-3, 1e-3) from splitmix64 at counter seed + x Ly + y
    x, yv = 3, 7
    U = (oracle.splitmix64(seed + x * Ly + yv) >> 11) * 2.0 ** -53
    assert T[x, yv] == T0[x, yv] * (1.0 + 1e-3 * (2.0 * U - 1.0))
    lat = oracle.Lattice(Lx, Ly)
    lat.init_rayleigh_taylor(seed)
    rho, u, Tf = lat.fields()
    np.testing.assert_allclose(Tf, T, rtol=1e-14)
    np.testing.assert_allclose(rho, 1.0 / T, rtol=1e-14)
    assert np.abs(u).max() < 1e-15


def test_bad_arguments():
    with pytest.raises(ValueError):
        oracle.Lattice(2, 8)
    with pytest.raises(ValueError):
        oracle.Lattice(8, 5)
    with pytest.raises(ValueError):
        oracle.Lattice(8, 8, tau=0.5)
    lat = oracle.Lattice(8, 8)
    with pytest.raises(ValueError):
        lat.run(1, oracle.PHASE_BC)
