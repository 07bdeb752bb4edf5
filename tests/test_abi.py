"""CPU checks of the C ABI: the library loads, exports every entry point that
include/d2q37.h declares, and its host-side set-up (velocity set, quadrature
solved by its own double-double solver) agrees with the oracle.  No CUDA
call is made."""
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
import paper_1703_00185_gb300 as lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "d2q37.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1703_00185_gb300 import _build
    _build.build()
    return lbm.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", text)))


def test_header_declares_binding_names():
    assert declared_functions() == sorted(lbm.exported_symbols())


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lbm.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (lbm_[a-z_]+)\b", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    for f in declared_functions():
        assert hasattr(lib, f)


def test_velocity_set_is_the_oracle_set(lib):
    cx, cy = lbm.lbm_velocity_set()
    ocx, ocy = oracle.velocity_set()
    assert sorted(zip(cx.tolist(), cy.tolist())) == sorted(zip(ocx.tolist(), ocy.tolist()))
    # pairs (c, -c) are adjacent after the rest population
    assert (cx[0], cy[0]) == (0, 0)
    assert np.array_equal(cx[1::2], -cx[2::2]) and np.array_equal(cy[1::2], -cy[2::2])


def test_library_quadrature_matches_oracle_bitwise(lib):
    s, w = lbm.lbm_quadrature()
    so, wo = oracle.scale_and_weights()
    cx, cy = lbm.lbm_velocity_set()
    ocx, ocy = oracle.velocity_set()
    idx = {(a, b): i for i, (a, b) in enumerate(zip(ocx.tolist(), ocy.tolist()))}
    perm = [idx[(a, b)] for a, b in zip(cx.tolist(), cy.tolist())]
    assert s == so
    assert np.array_equal(w, wo[perm])


def test_params_validation_without_gpu(lib):
    p = lbm.lbm_default_params()
    assert (p.tau, p.g0, p.T_top, p.T_bot, p.kernel) == (0.8, 1e-4, 0.5, 1.5, lbm.KERNEL_FUSED)
    assert lbm.lbm_required_bytes(2048, 8192, p) > 2 * 37 * 2054 * 8224 * 8
    assert lbm.lbm_required_bytes(2, 8192, p) == 0
    assert lbm.lbm_required_bytes(8, 5, p) == 0
    p.tau = 0.5
    assert lbm.lbm_required_bytes(8, 8, p) == 0
    p.tau, p.kernel = 0.8, 7
    assert lbm.lbm_required_bytes(8, 8, p) == 0
    assert lbm.lbm_strerror(lbm.LBM_EINVAL) == "invalid argument"
