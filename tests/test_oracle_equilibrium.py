"""Pins of the oracle's equilibrium and collision.

* P2: every moment of order <= 4 of f^eq(rho, u, T) equals the moment of the
  Maxwellian of Eq. MASTERSHIFT3, rho E[(u + sqrt(T) Z)^alpha] (closed form).
* P3: one collision with gravity changes mass by 0, momentum by rho g and
  energy sum |xi|^2 f by 2 rho u.g (follows from the shifts
  u_bar = u + tau g, T_bar = T - tau^2 g^2 / D of Eq. MASTERSHIFT3).
* P4: with g = 0 an equilibrium is a fixed point of collide; with tau = 1
  collide returns f^eq(rho, u_bar, T_bar) (Eq. discrete).
"""
from math import comb

import numpy as np
import pytest

import oracle
from oracle import naive, quadrature
from tests import synthetic

Q = 37


def gauss_shift_moment(k, u, T):
    """E[(u + sqrt(T) Z)^k], Z standard normal."""
    return sum(comb(k, m) * u ** (k - m) * T ** (m // 2) * quadrature.gaussian_moment(m)
               for m in range(0, k + 1, 2))


def moment_errors(feq_fn, cases, max_order=4):
    s, _ = oracle.scale_and_weights()
    cx, cy = oracle.velocity_set()
    xx, yy = s * cx, s * cy
    worst = 0.0
    for rho, ux, uy, T in cases:
        f = feq_fn(rho, ux, uy, T)
        for i in range(max_order + 1):
            for j in range(max_order + 1 - i):
                terms = f * xx ** i * yy ** j
                exact = rho * gauss_shift_moment(i, ux, T) * gauss_shift_moment(j, uy, T)
                scale = float(np.sum(np.abs(terms)))
                worst = max(worst, abs(float(np.sum(terms)) - exact) / scale)
    return worst


CASES = [(1.0, 0.0, 0.0, 1.0), (1.3, 0.05, -0.02, 0.7), (0.6, -0.2, 0.3, 1.4), (2.0, 0.1, 0.1, 0.5),
         (1.0, 0.4, -0.3, 1.1)]


def test_equilibrium_moments_to_order_4():
    assert moment_errors(oracle.equilibrium, CASES) < 5e-15


def test_equilibrium_misses_order_5():
    # the 4th-order truncation must not reproduce 5th-order moments at finite u
    s, _ = oracle.scale_and_weights()
    cx, cy = oracle.velocity_set()
    rho, ux, uy, T = 1.0, 0.4, -0.3, 1.1
    f = oracle.equilibrium(rho, ux, uy, T)
    q = float(np.sum(f * (s * cx) ** 5))
    assert abs(q - rho * gauss_shift_moment(5, ux, T)) > 1e-4


def test_equilibrium_at_reference_state_is_weights():
    _, w = oracle.scale_and_weights()
    assert np.array_equal(oracle.equilibrium(1.0, 0.0, 0.0, 1.0), w)
    np.testing.assert_allclose(oracle.equilibrium(1.7, 0.0, 0.0, 1.0), 1.7 * w, rtol=1e-15)


@pytest.mark.parametrize("mutation", ["drop_theta2", "flip_a3", "drop_q2", "x2_shift"])
def test_moment_pin_catches_planted_mistakes(mutation):
    """Plant a plausible mistake in a copy of the (naive) equilibrium and check
    that the order <= 4 moment pin fails; guards the pin's sensitivity."""
    m = naive.Model()

    def bad(rho, ux, uy, T):
        a = m.xix * ux + m.xiy * uy
        q = ux * ux + uy * uy
        th = T - 1.0
        x2 = m.x2
        t4 = 3.0 * th * th * (x2 * x2 - 8.0 * x2 + 8.0)
        t3 = a * (a * a - 3.0 * q + 3.0 * th * (x2 - 4.0)) / 6.0
        q2 = 3.0 * q * q
        t2 = (a * a - q + th * (x2 - 2.0)) / 2.0
        if mutation == "drop_theta2":
            t4 = 0.0
        if mutation == "flip_a3":
            t3 = -t3
        if mutation == "drop_q2":
            q2 = 0.0
        if mutation == "x2_shift":
            t2 = (a * a - q + th * (x2 - 3.0)) / 2.0
        P = 1.0 + a + t2 + t3 + (a ** 4 - 6.0 * a * a * q + q2 + 6.0 * th * (a * a * (x2 - 6.0) + q * (4.0 - x2))
                               + t4) / 24.0
        return m.w * rho * P

    # the mutated form uses quadrature order; map the C oracle's order onto it
    cx, cy = oracle.velocity_set()
    order = [list(zip(m.cx, m.cy)).index((a, b)) for a, b in zip(cx, cy)]
    assert moment_errors(lambda *a: bad(*a)[order], CASES) > 1e-6


def test_naive_equilibrium_equals_tensor_form():
    m = naive.Model()
    cx, cy = oracle.velocity_set()
    order = [list(zip(m.cx, m.cy)).index((a, b)) for a, b in zip(cx, cy)]
    for rho, ux, uy, T in CASES:
        np.testing.assert_allclose(m.feq(rho, ux, uy, T)[order], oracle.equilibrium(rho, ux, uy, T),
                                   rtol=2e-14, atol=1e-17)


def _random_f(seed):
    _, w = oracle.scale_and_weights()
    return synthetic.random_populations(w * 1.2, 1, 1, seed, rel_noise=0.1)[:, 0, 0]


@pytest.mark.parametrize("tau", [0.6, 0.8, 1.0, 1.5])
def test_collide_conservation_and_gravity_work(tau):
    s, _ = oracle.scale_and_weights()
    cx, cy = oracle.velocity_set()
    xx, yy = s * cx, s * cy
    gx, gy = 0.0, -1e-3
    for seed in range(5):
        f = _random_f(seed)
        out = oracle.collide_site(f, tau, gx, gy)
        rho, ux, uy, _ = oracle.site_moments(f)
        assert abs(out.sum() - f.sum()) < 1e-15 * rho
        assert abs((xx * out).sum() - (xx * f).sum() - rho * gx) < 2e-15
        assert abs((yy * out).sum() - (yy * f).sum() - rho * gy) < 2e-15
        e_in, e_out = ((xx ** 2 + yy ** 2) * f).sum(), ((xx ** 2 + yy ** 2) * out).sum()
        assert abs(e_out - e_in - 2.0 * rho * (ux * gx + uy * gy)) < 2e-14


def test_collide_equilibrium_fixed_point():
    for rho, ux, uy, T in CASES:
        feq = oracle.equilibrium(rho, ux, uy, T)
        out = oracle.collide_site(feq, 0.8, 0.0, 0.0)
        np.testing.assert_allclose(out, feq, rtol=1e-13, atol=1e-16)


def test_collide_tau_one_returns_shifted_equilibrium():
    gx, gy = 0.0, -2e-3
    for seed in range(3):
        f = _random_f(seed)
        rho, ux, uy, T = oracle.site_moments(f)
        out = oracle.collide_site(f, 1.0, gx, gy)
        ref = oracle.equilibrium(rho, ux + gx, uy + gy, T - (gx * gx + gy * gy) / 2.0)
        np.testing.assert_allclose(out, ref, rtol=1e-14, atol=1e-17)


def test_moments_definition():
    # D rho T = sum |xi - u|^2 f; checked against the expanded form
    s, _ = oracle.scale_and_weights()
    cx, cy = oracle.velocity_set()
    f = _random_f(7)
    rho, ux, uy, T = oracle.site_moments(f)
    e = ((s * cx) ** 2 + (s * cy) ** 2) @ f
    assert abs(2.0 * rho * T - (e - rho * (ux * ux + uy * uy))) < 1e-14
