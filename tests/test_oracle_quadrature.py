"""Pins of the oracle's velocity set and quadrature (reading of Sec. "Lattice
Boltzmann methods": the D2Q37 set and its weights are not printed)."""
import os
from decimal import Decimal

import numpy as np
import pytest

from oracle import quadrature
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split()
            out[k] = v
    return out


def test_velocity_set_matches_paper_counts():
    g = _golden("paper_counts.txt")
    vel = quadrature.velocity_set()
    assert len(vel) == int(g["populations"]) == 37
    assert len(set(vel)) == 37
    assert max(max(abs(a), abs(b)) for a, b in vel) == int(g["max_hop"])
    # populations that must be moved across one vertical boundary per site:
    # one strip per (population, halo column d) with c_x >= d
    crossing = sum(1 for cx, _ in vel for d in (1, 2, 3) if cx >= d)
    assert crossing == int(g["populations_crossing_one_boundary"])
    assert 2 * crossing == int(g["halo_exchange_operations"])
    # symmetric under c -> -c and x <-> y
    assert set(vel) == {(-a, -b) for a, b in vel} == {(b, a) for a, b in vel}
    sizes = [sum(1 for a, b in vel if a * a + b * b == c2) for c2 in quadrature.SHELL_C2]
    assert sizes == [1, 4, 4, 4, 8, 4, 4, 8]


def test_c_oracle_enumerates_same_set():
    cx, cy = oracle.velocity_set()
    assert sorted(zip(cx.tolist(), cy.tolist())) == sorted(quadrature.velocity_set())


def _dpow(x, n):
    return Decimal(1) if n == 0 else x ** n


def test_decimal_solution_residual():
    s, w = quadrature.solve_weights()
    vel = quadrature.velocity_set()
    for i, j in quadrature.MOMENT_ORDERS:
        acc = Decimal(0)
        for cx, cy in vel:
            k = quadrature.SHELL_C2.index(cx * cx + cy * cy)
            acc += w[k] * _dpow(s * cx, i) * _dpow(s * cy, j)
        exact = quadrature.gaussian_moment(i) * quadrature.gaussian_moment(j)
        assert abs(acc - exact) < Decimal(10) ** -35
    assert all(x > 0 for x in w)
    assert Decimal("0.3") < s < Decimal("2.5")


def test_gaussian_moments_all_monomials_up_to_degree_9():
    """Closed form: sum_l w_l xi_x^i xi_y^j = E[X^i] E[Y^j] for i + j <= 9,
    including odd and mixed monomials the solve never imposed directly."""
    s, w = oracle.scale_and_weights()
    cx, cy = oracle.velocity_set()
    xx, yy = s * cx, s * cy
    assert abs(w.sum() - 1.0) < 1e-15
    for i in range(10):
        for j in range(10 - i):
            terms = w * xx ** i * yy ** j
            q = float(np.sum(terms))
            exact = quadrature.gaussian_moment(i) * quadrature.gaussian_moment(j)
            # rounding bound of a 37-term FP64 sum, relative to the sum of |terms|
            assert abs(q - exact) <= 1e-15 * float(np.sum(np.abs(terms))), (i, j, q, exact)


def test_quadrature_not_exact_at_degree_10():
    # a degree-9 rule must miss some degree-10 moment; guards a test that passes trivially
    s, w = oracle.scale_and_weights()
    cx, cy = oracle.velocity_set()
    q = float(np.sum(w * (s * cx) ** 10))
    assert abs(q - quadrature.gaussian_moment(10)) > 1e-3


def test_independent_high_precision_solve():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    vel = quadrature.velocity_set()
    # eliminate the weights: for fixed s solve the 8 conditions other than (8, 0)
    # and bisect on the residual of (8, 0)
    rows = [ij for ij in quadrature.MOMENT_ORDERS if ij != (8, 0)]

    def weights_at(s):
        A = mp.matrix([[sum((s * a) ** i * (s * b) ** j for a, b in vel if a * a + b * b == c2)
                        for c2 in quadrature.SHELL_C2] for i, j in rows])
        rhs = mp.matrix([quadrature.gaussian_moment(i) * quadrature.gaussian_moment(j) for i, j in rows])
        return mp.lu_solve(A, rhs)

    def resid(s):
        w = weights_at(s)
        return sum(w[quadrature.SHELL_C2.index(a * a + b * b)] * (s * a) ** 8 for a, b in vel) - 105

    s_root = mp.findroot(resid, (mp.mpf("1.1"), mp.mpf("1.3")), solver="anderson")
    s, w = quadrature.weights_fp64()
    assert abs(float(s_root) - s) <= 2 * np.spacing(s)
    w_mp = weights_at(s_root)
    for k in range(8):
        assert abs(float(w_mp[k]) - w[k]) <= 2 * np.spacing(w[k])


def test_splitmix64_published_output():
    g = open(os.path.join(GOLDEN, "splitmix64.txt")).read().split("\n")
    for line in g:
        line = line.split("#")[0].strip()
        if line:
            state, out = (int(v, 16) for v in line.split())
            assert oracle.splitmix64(state) == out
