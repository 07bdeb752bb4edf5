"""Design check of the FP64 step's fixed-point arithmetic (no GPU).

The CUDA collision evaluates the equilibrium, and the site values it needs,
in 64-bit integers with a power-of-two scale per quantity, every product
being the high word of a 64 x 64-bit product: exact (floor), with the
low-by-low partial product left out (the per-pair products), or rounded (the
odd part); signed site values meet the shell constants shifted by 2^63, with
the offsets and rounding corrections in per-shell constants, and the
conversion sets the result's lowest bit.  This module restates those integer
operations in Python (exact integers, the same scales and the same order)
and checks them against exact rational arithmetic: no intermediate leaves its
64-bit format anywhere inside the fixed-point ranges (rho in (0, 4),
|u| < 0.35 per component, |T_bar - 1| < 1), and the results are better than
FP64 rounding.  It also recomputes the moment sums' floor compensation.  It is
a check of the formats, not of the kernel: the kernel itself is held to the
oracle by the GPU tests.
"""
import math
import os
import random
import re
import struct
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle

M64 = (1 << 64) - 1


def umulhi(a, b):
    assert 0 <= a <= M64 and 0 <= b <= M64
    return (a * b) >> 64


def mulhi_su(x, y):  # signed x, unsigned y: floor(x y 2^-64)
    assert -(1 << 63) <= x < (1 << 63) and 0 <= y <= M64
    return (x * y) >> 64


def umulhi_t(a, y):
    """High word of a y without the low-by-low partial product: three
    32 x 32 -> 64-bit multiply-adds, the floor or one below it."""
    assert 0 <= a <= M64 and 0 <= y <= M64
    al, ah, yl, yh = a & 0xFFFFFFFF, a >> 32, y & 0xFFFFFFFF, y >> 32
    lh = al * yh
    hl = ah * yl + (lh & 0xFFFFFFFF)
    assert hl <= M64
    r = ah * yh + (lh >> 32) + (hl >> 32)
    assert (a * y >> 64) - 1 <= r <= a * y >> 64
    return r


def mulhi_su_t(x, y):  # umulhi_t for signed x (mod 2^64, as the kernel's u64)
    assert -(1 << 63) <= x < (1 << 63) and 0 <= y <= M64
    return umulhi_t(x & M64, y) - (y if x < 0 else 0)


def flip(x):  # x + 2^63 as an unsigned operand: the sign bit flipped
    assert -(1 << 63) <= x < (1 << 63)
    return x + (1 << 63)


def fits(v, name):
    assert -(1 << 63) <= v < (1 << 63), name
    return v


@pytest.fixture(scope="module")
def quad():
    s, w = oracle.scale_and_weights()
    cx, cy = oracle.velocity_set()
    c2 = (np.asarray(cx) ** 2 + np.asarray(cy) ** 2).tolist()
    shells = sorted(set(c2))
    wk = [float(np.asarray(w)[c2.index(k)]) for k in shells]
    return float(s), shells, wk


def shell_consts(s, c2, w, omega):
    x2 = Fr(s) ** 2 * c2
    cw = Fr(omega) * Fr(w)
    E = math.frexp(float(cw))[1]
    c = cw / Fr(2) ** E
    C = dict(E=E, c60=round(c * 2**60), c62=round(c * 2**62), c64=round(c * 2**64),
             cx2_59=round(c * x2 * 2**59), cx2_60=round(c * x2 * 2**60), cx4_55=round(c * x2 * x2 * 2**55),
             c6=round(c / 6 * 2**64))
    assert C["c6"] == round(c / 24 * 2**66)  # the same integer serves R3 (Q61) and R4 (Q63)
    # y / 2 of each product with a flipped operand, less a rounding correction
    C["d0"] = 0 if c2 == 0 else (C["cx2_59"] >> 1) - 2
    C["d1"] = (C["c62"] >> 1) + (C["cx2_59"] >> 1) - 1
    C["d2"] = (C["c64"] >> 1) + (C["cx2_60"] >> 1) - 1
    return C


PAIRS = [(1, 0), (0, 1), (1, 1), (1, -1), (2, 0), (0, 2), (2, 1), (2, -1), (1, 2), (1, -2), (2, 2), (2, -2),
         (3, 0), (0, 3), (3, 1), (3, -1), (1, 3), (1, -3)]


def equilibrium_fixed(s, shells, wk, R, UX, UY, TH, omega):
    """The kernel's fixed-point equilibrium: omega w rho P for every velocity."""
    AUX, AUY = abs(UX), abs(UY)
    q = umulhi(AUX, AUX) + umulhi(AUY, AUY)
    q2 = umulhi(q, q)
    B1 = (1 << 62) - (q >> 3)
    B2 = (1 << 61) - (q >> 4)
    A0 = B1 + (q2 >> 5)
    S62 = round(Fr(s) * 2**62)
    SX, SY = mulhi_su(UX, S62), mulhi_su(UY, S62)
    rA0, rB1, rB2 = umulhi(R, A0), umulhi(R, B1), umulhi(R, B2)
    rth = fits((R * TH) >> 62, "rth")
    rth2 = fits((rth * TH) >> 62, "rth2")
    rthq = fits(mulhi_su(rth, q), "rthq")
    K0 = fits(rA0 - (rth >> 2) + (rthq >> 2) + (rth2 >> 2), "K0")
    K1 = fits((rth >> 2) - (rthq >> 3) - (rth2 >> 1), "K1")
    K2 = rth2
    L0 = fits(rB1 - (rth >> 1), "L0")
    M0 = fits(rB2 - (rth >> 2) - (rth >> 3), "M0")
    assert K0 > 0  # taken as an unsigned operand without the flip
    out = {}
    for k, c2 in enumerate(shells):
        C = shell_consts(s, c2, wk[k], omega)
        if c2 == 0:
            out[(0, 0)] = Fr(fits(umulhi(K0, C["c60"]) - C["d0"], "G0") | 1) * Fr(2) ** (C["E"] - 55)
            continue
        R0 = fits(umulhi(K0, C["c60"]) + umulhi(flip(K1), C["cx2_59"]) + umulhi(K2, C["cx4_55"]) - C["d0"],
                  "R0")
        R1 = fits(umulhi(flip(L0), C["c62"]) + umulhi(flip(rth), C["cx2_59"]) - C["d1"], "R1")
        R2 = fits(umulhi(flip(M0), C["c64"]) + umulhi(flip(rth), C["cx2_60"]) - C["d2"], "R2")
        R3 = fits(umulhi(R, C["c6"]), "R3")
        R4 = R3  # c rho / 24 at Q63
        for cx, cy in PAIRS:
            if cx * cx + cy * cy != c2:
                continue
            a = fits(cx * SX + cy * SY, "a")
            A = abs(a)
            b = umulhi_t(A, A)
            t = fits(R2 + umulhi_t(b, R4), "t")
            even = fits(R0 + mulhi_su_t(t, b), "even")
            sv = fits(R1 + umulhi_t(b, R3), "s")
            oa = (sv * A + (1 << 63)) >> 64  # rounded to nearest
            odd = -oa if a < 0 else oa
            # the conversion sets the lowest bit (never zero)
            out[(cx, cy)] = Fr(fits(even + odd, "G+") | 1) * Fr(2) ** (C["E"] - 55)
            out[(-cx, -cy)] = Fr(fits(even - odd, "G-") | 1) * Fr(2) ** (C["E"] - 55)
    return out


def equilibrium_exact(s, shells, wk, rho, ux, uy, th, omega):
    q = ux * ux + uy * uy
    out = {}
    for k, c2 in enumerate(shells):
        x2 = Fr(s) ** 2 * c2
        C0 = 1 - q / 2 + q * q / 8 + th * ((x2 - 2) / 2 + q * (4 - x2) / 4 + th * (x2 * x2 - 8 * x2 + 8) / 8)
        C1 = 1 - q / 2 + th * (x2 - 4) / 2
        C2 = Fr(1, 2) - q / 4 + th * (x2 - 6) / 4
        vs = [(0, 0)] if c2 == 0 else [v for cx, cy in PAIRS if cx * cx + cy * cy == c2 for v in ((cx, cy), (-cx, -cy))]
        for cx, cy in vs:
            a = Fr(s) * (cx * ux + cy * uy)
            out[(cx, cy)] = Fr(omega) * Fr(wk[k]) * rho * (C0 + a * C1 + a * a * C2 + a ** 3 / 6 + a ** 4 / 24)
    return out


STATES = [(3.999, 0.3499, -0.3499, 0.999, 1.9), (3.999, -0.3499, 0.3499, -0.999, 0.5), (0.5, 0.0, 0.0, 0.0, 1.25)]
_rng = random.Random(11)
STATES += [(_rng.uniform(0.3, 3.99), _rng.uniform(-0.349, 0.349), _rng.uniform(-0.349, 0.349), _rng.uniform(-0.99, 0.99),
            _rng.choice([0.6, 1.0, 1.25, 1.9])) for _ in range(40)]
STATES += [(_rng.uniform(0.6, 2.1), _rng.uniform(-0.05, 0.05), _rng.uniform(-0.05, 0.05), _rng.uniform(-0.55, 0.55),
            1.25) for _ in range(40)]


def test_equilibrium_formats_fit_and_beat_fp64(quad):
    """Every intermediate fits 64 bits at the range corners and inside; the
    error relative to omega w rho stays below 2^-50 (the FP64 evaluation of
    the same polynomial loses ~1e-14 near T = 0.5 for the outer shells)."""
    s, shells, wk = quad
    worst = 0.0
    for rho, ux, uy, th, omega in STATES:
        R, UX, UY, TH = round(Fr(rho) * 2**61), round(Fr(ux) * 2**64), round(Fr(uy) * 2**64), round(Fr(th) * 2**62)
        got = equilibrium_fixed(s, shells, wk, R, UX, UY, TH, omega)
        ref = equilibrium_exact(s, shells, wk, Fr(R, 2**61), Fr(UX, 2**64), Fr(UY, 2**64), Fr(TH, 2**62), omega)
        assert set(got) == set(ref) and len(got) == 37
        for key, v in got.items():
            c2 = key[0] ** 2 + key[1] ** 2
            scale = Fr(omega) * Fr(wk[shells.index(c2)]) * Fr(rho)
            worst = max(worst, float(abs(v - ref[key]) / scale))
    assert worst < 2.0 ** -50, worst


def site_values_fixed(s, r, jx, jy, e, emax, uy_shift, th_shift):
    """The kernel's rho (Q61), u_x, u_bar_y (Q64) and theta (Q62) from the
    exact moment sums on the grid 2^(emax - 1075); None outside the ranges."""
    if r <= 0 or e < 0 or 2 * abs(jx) >= r or 2 * abs(jy) >= r or e >= 3 * r:
        return None
    n = 64 - r.bit_length()
    rn = r << n
    rc = np.float32(1.0) / np.float32(rn >> 40)  # correctly rounded float reciprocal
    rb = struct.unpack("<I", struct.pack("<f", rc))[0]
    X = ((rb & 0x7FFFFF) | 0x800000) << (((rb >> 23) & 0xFF) - 64)
    for _ in range(2):
        X = (umulhi(X, (1 << 63) - umulhi(rn, X)) << 2) & M64
    S63, S2 = round(Fr(s) * 2**63), round(Fr(s) * Fr(s) * 2**63)
    ux61 = mulhi_su(mulhi_su(jx << n, X), S63)
    uy61 = mulhi_su(mulhi_su(jy << n, X), S63)
    if abs(ux61) >= 0x0B33333333333333:
        return None
    UX, UY0 = ux61 << 3, uy61 << 3
    UY = UY0 + round(Fr(uy_shift) * 2**64)
    if abs(UY) >= 0x5999999999999999:
        return None
    er = umulhi(e << (n - 2), X)
    th60 = umulhi(er, S2) - ((umulhi(abs(UX), abs(UX)) + umulhi(abs(UY0), abs(UY0))) >> 5) + round(Fr(th_shift) * 2**60)
    if abs(th60) >= 1 << 60:
        return None
    sR = emax - 1014
    if sR >= 0:
        if sR >= n:
            return None
        R = r << sR
    else:
        rs = min(-sR, 63)
        R = (r + (1 << (rs - 1))) >> rs
    if R == 0 or R >= 1 << 63:
        return None
    return R, UX, UY, th60 << 2


def test_site_values_from_sums(quad):
    """rho, u and theta from the integer sums: inside the ranges within
    1e-17 absolute (FP64 rounding of u and T is ~1e-17 to 1e-16); outside
    them (up to the last digit) rejected."""
    s = quad[0]
    rng = random.Random(5)
    tau, g0 = 0.8, 1e-4
    uy_shift, th_shift = -tau * g0, -(tau * g0) ** 2 / 2 - 1
    inside = 0
    for _ in range(600):
        emax = rng.randint(1015, 1024)
        rho, ux, uy, T = rng.uniform(0.05, 4.5), rng.uniform(-0.4, 0.4), rng.uniform(-0.4, 0.4), rng.uniform(0.02, 2.2)
        g = Fr(2) ** (emax - 1075)
        r = int(Fr(rho) / g)
        if r >= 37 * 2**53:
            continue
        jx, jy = int(Fr(rho * ux / s) / g), int(Fr(rho * uy / s) / g)
        e = int(Fr(rho * (2 * T + ux * ux + uy * uy) / (s * s)) / g)
        RHO, UXe, UY0e = Fr(r) * g, Fr(s) * jx / r, Fr(s) * jy / r
        THe = (Fr(s) * Fr(s) * e / r - UXe ** 2 - UY0e ** 2) / 2 + Fr(th_shift)
        UYe = UY0e + Fr(uy_shift)
        out = site_values_fixed(s, r, jx, jy, e, emax, uy_shift, th_shift)
        ok = 0 < RHO < 4 and abs(UXe) < Fr(35, 100) and abs(UYe) < Fr(35, 100) and abs(THe) < 1
        if out is None:
            margin = min(abs(RHO - 4), abs(abs(UXe) - Fr(35, 100)), abs(abs(UYe) - Fr(35, 100)), abs(abs(THe) - 1))
            assert not ok or margin < Fr(1, 10**12)
            continue
        inside += 1
        R, UX, UY, TH = out
        assert abs(Fr(R, 2**61) - RHO) < Fr(1, 10**17)
        assert abs(Fr(UX, 2**64) - UXe) < Fr(1, 10**17)
        assert abs(Fr(UY, 2**64) - UYe) < Fr(1, 10**17)
        assert abs(Fr(TH, 2**62) - THe) < Fr(1, 10**17)
    assert inside > 100


# The FP64 step's exact moment sums round every population down to the grid
# 2^(emax - 1075) of the site's largest exponent (a negative one through the
# one's complement of its magnitude) and give the mean deficit back as
# constants: kFloorR to r = sum f, kFloorE to e = sum |c|^2 f (jx, jy need
# none: sum c = 0).  The kernel's constants, read from its source:
_KSRC = open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", "paper_1703_00185_gb300", "csrc",
                          "d2q37_kernels.cu")).read()
FLOOR_R, FLOOR_E = (int(v) for v in re.search(r"kFloorR = (\d+), kFloorE = (\d+);", _KSRC).groups())


def floor_deficits(f, c2):
    """Per site (rows of f), the deficits sum_l (exact - floored) and
    sum_l |c_l|^2 (exact - floored) of the kernel's conversion, in grid units."""
    bits = f.view(np.int64)
    hi = bits >> 32
    e = (hi >> 20) & 0x7FF
    emax = ((hi & 0x7FFFFFFF) >> 20).max(axis=1, keepdims=True)
    mant = (bits & ((1 << 52) - 1)) | (1 << 52)
    sh = np.minimum(emax - e, 62)
    neg = hi < 0
    got = np.where(neg, ~mant, mant) >> sh  # the kernel's term
    # exact value on the grid: +-mant 2^-sh; the deficit is computed in two
    # integer parts so that no float rounding enters
    whole = np.where(neg, -((mant + (1 << sh) - 1) >> sh), mant >> sh)
    rem = np.where(neg, (-mant) & ((1 << sh) - 1), mant & ((1 << sh) - 1))
    deficit = (whole - got) + rem / np.exp2(sh.astype(float))
    return deficit.sum(axis=1), (deficit * np.asarray(c2)).sum(axis=1)


def test_moment_floor_compensation():
    """The constants are the mean deficits (to the nearest integer) over
    near-equilibrium sites: the oracle's equilibria over the step's range of
    states (including the cold ones with negative populations), perturbed by
    1 %.  Every single deficit stays within [0, 37] (r) and [0, 216] (e)."""
    cx, cy = oracle.velocity_set()
    c2 = (np.asarray(cx) ** 2 + np.asarray(cy) ** 2)
    rng = np.random.default_rng(17)
    n = 4000
    rho = rng.uniform(0.7, 1.4, n)
    ux, uy = rng.uniform(-0.1, 0.1, n), rng.uniform(-0.1, 0.1, n)
    T = rng.uniform(0.5, 1.5, n)
    f = np.stack([oracle.equilibrium(rho[i], ux[i], uy[i], T[i]) for i in range(n)])
    f = f * (1.0 + 0.01 * rng.standard_normal(f.shape))
    assert (f < 0).any(axis=1).mean() > 0.1  # cold sites with negative populations are in the sample
    dr, de = floor_deficits(np.ascontiguousarray(f), c2)
    assert dr.min() >= 0 and dr.max() <= 37 and de.min() >= 0 and de.max() <= c2.sum()
    assert abs(dr.mean() - FLOOR_R) <= 0.5, dr.mean()
    assert abs(de.mean() - FLOOR_E) <= 0.5, de.mean()
