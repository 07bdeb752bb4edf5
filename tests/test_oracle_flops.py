"""The oracle's FP64 flop count per site collision (its counting build) and
the constants bench.py reports it with (the FP64-flop side of the roofline,
which bench.py may not compute itself: it only runs the oracle in its CPU
baseline)."""
import ast
import os
import shutil

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++ for the counting build")


def bench_constants():
    src = open(os.path.join(os.path.dirname(__file__), "..", "bench.py")).read()
    out = {}
    for node in ast.parse(src).body:
        if isinstance(node, ast.Assign) and isinstance(node.targets[0], ast.Name) and \
                node.targets[0].id.startswith("ORACLE_"):
            out[node.targets[0].id] = ast.literal_eval(node.value)
    return out


def test_counts_match_bench_constants():
    c = bench_constants()
    assert oracle.collide_flops_per_site() == c["ORACLE_FLOPS_PER_SITE"]
    assert oracle.collide_flops_per_site(nontrivial=True) == c["ORACLE_NONTRIVIAL_FLOPS_PER_SITE"]
    assert oracle.contracted_collide_flops_per_site() == c["ORACLE_CONTRACTED_FLOPS_PER_SITE"]


def test_contracted_form_is_the_same_collision():
    """The hand-contracted form whose operations the roofline counts computes
    the oracle's collision: on random near-equilibrium sites (rho 0.7..1.4,
    |u| < 0.1, T 0.5..1.5, populations perturbed by 2 %) both counted forms
    agree to rounding, and the contracted one equals the plain one of the
    oracle library."""
    rng = np.random.default_rng(7)
    worst = 0.0
    for _ in range(200):
        rho, T = rng.uniform(0.7, 1.4), rng.uniform(0.5, 1.5)
        ux, uy = rng.uniform(-0.07, 0.07, 2)
        f = oracle.equilibrium(rho, ux, uy, T) * (1.0 + 0.02 * rng.uniform(-1, 1, 37))
        tau, gy = rng.choice([0.6, 0.8, 1.5]), -rng.choice([0.0, 1e-4, 1e-2])
        a = oracle.counted_collide_values(f, tau, 0.0, gy, contracted=True)
        b = oracle.counted_collide_values(f, tau, 0.0, gy, contracted=False)
        c = oracle.collide_site(f, tau, 0.0, gy)
        assert np.array_equal(b, c)  # the counting type changes no arithmetic
        worst = max(worst, np.abs(a - b).max() / np.abs(b).max())
    assert worst < 1e-14, worst


def test_contracted_count_is_per_population_work():
    """The contracted form does O(50) operations per population, far fewer
    than the tensor form, and more than the moments alone."""
    n, nt = oracle.contracted_collide_flops_per_site(), oracle.contracted_collide_flops_per_site(nontrivial=True)
    assert 37 * 40 < nt <= n < oracle.collide_flops_per_site() / 10


def test_count_is_the_oracles_arithmetic():
    """Sanity: the tensor-form equilibrium dominates (more than 37 x 100
    operations), the non-trivial count is smaller, and the moments alone
    (4 sums of 37 terms) bound it from below."""
    n, nt = oracle.collide_flops_per_site(), oracle.collide_flops_per_site(nontrivial=True)
    assert 4 * 37 < nt < n
    assert n > 37 * 100
