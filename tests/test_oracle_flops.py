"""The oracle's FP64 flop count per site collision (its counting build) and
the constants bench.py reports it with (the FP64-flop side of the roofline,
which bench.py may not compute itself: it only runs the oracle in its CPU
baseline)."""
import ast
import os
import shutil

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


def test_count_is_the_oracles_arithmetic():
    """Sanity: the tensor-form equilibrium dominates (more than 37 x 100
    operations), the non-trivial count is smaller, and the moments alone
    (4 sums of 37 terms) bound it from below."""
    n, nt = oracle.collide_flops_per_site(), oracle.collide_flops_per_site(nontrivial=True)
    assert 4 * 37 < nt < n
    assert n > 37 * 100
