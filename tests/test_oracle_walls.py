"""Pin: each wall imposes its own temperature on the fluid.

The paper's walls (Sec. "The propagate and bc Kernels") hold a constant
temperature and zero velocity on the rows next to them.  Without gravity, a
fluid at rest between a wall at T_bot (y = 0 side) and one at T_top
(y = Ly - 1 side) relaxes to steady heat conduction.  The pressure rho T is
then uniform, and the BGK heat conductivity is proportional to it, so the
steady temperature is linear in y.  It runs from T_bot at the bottom to T_top
at the top, up to the small temperature jumps of a kinetic wall (a few
percent of T_bot - T_top at tau = 0.8).

The checks fail for a wall that injects its equilibrium at the wrong
temperature with the right mass (flat or offset profile), for swapped wall
temperatures (wrong sign of the slope and wrong end values), and for a missing
wall term in the energy balance (nonlinear profile).  Mirror symmetry of the
velocity set adds an exact check: swapping T_bot and T_top mirrors the steady
profile in y.
"""
import numpy as np
import pytest

import oracle

LX, LY, STEPS = 3, 24, 3000  # converged to < 1e-8 (checked by the test)


@pytest.fixture(scope="module", autouse=True)
def one_thread():
    n = oracle.threads()
    oracle.set_threads(1)  # a 3 x 24 lattice: threads only add overhead
    yield
    oracle.set_threads(n)


def steady_profile(T_bot, T_top):
    """Mean over x of T(y) after STEPS steps from rest at the mean wall
    temperature (g = 0), and the largest change of it over 200 more steps."""
    o = oracle.Lattice(LX, LY, tau=0.8, g0=0.0, T_top=T_top, T_bot=T_bot)
    o.set_equilibrium(1.0, 0.0, 0.0, 0.5 * (T_bot + T_top))
    o.run(STEPS)
    T = o.fields()[2].mean(axis=0)
    o.run(200)
    return T, float(np.abs(o.fields()[2].mean(axis=0) - T).max())


def conduction_errors(T, T_bot, T_top):
    """Deviations from steady conduction between walls at T_bot and T_top,
    each relative to |T_bot - T_top|: fit residual of the bulk (rows 4..Ly-5),
    slope ratio to the ideal -(T_bot - T_top)/Ly, and the fitted line's values
    at the walls (y = -1/2 and y = Ly - 1/2) minus the wall temperatures."""
    dT = T_bot - T_top
    y = np.arange(LY, dtype=float)
    b = slice(4, LY - 4)
    A = np.vstack([y[b], np.ones(LY - 8)]).T
    (slope, icpt), *_ = np.linalg.lstsq(A, T[b], rcond=None)
    resid = float(np.abs(A @ np.array([slope, icpt]) - T[b]).max() / abs(dT))
    ratio = float(slope / (-dT / LY))
    jump_bot = float((icpt - 0.5 * slope - T_bot) / dT)
    jump_top = float((icpt + (LY - 0.5) * slope - T_top) / dT)
    return resid, ratio, jump_bot, jump_top


def is_conduction(T, T_bot, T_top):
    resid, ratio, jb, jt = conduction_errors(T, T_bot, T_top)
    return resid < 3e-3 and 0.93 < ratio <= 1.0 and abs(jb) < 0.03 and abs(jt) < 0.03


@pytest.mark.parametrize("T_bot,T_top", [(1.5, 0.5), (1.3, 0.9), (0.8, 1.2)])
def test_walls_impose_their_own_temperature(T_bot, T_top):
    T, change = steady_profile(T_bot, T_top)
    assert change < 1e-7  # steady
    resid, ratio, jb, jt = conduction_errors(T, T_bot, T_top)
    assert resid < 3e-3, resid       # linear in the bulk
    assert 0.93 < ratio <= 1.0, ratio  # slope: sign and size set by the two walls
    assert abs(jb) < 0.03 and abs(jt) < 0.03, (jb, jt)  # each wall at its own temperature
    # the fluid's mean temperature lies midway between the walls
    assert abs(T.mean() - 0.5 * (T_bot + T_top)) < 0.01 * abs(T_bot - T_top)


def test_swapped_walls_mirror_the_profile():
    """Exchanging T_bot and T_top mirrors the steady state in y exactly (the
    velocity set is symmetric under cy -> -cy), so the top wall acts with
    T_top as the bottom one does with T_bot."""
    a, _ = steady_profile(1.3, 0.9)
    b, _ = steady_profile(0.9, 1.3)
    assert np.abs(a - b[::-1]).max() < 1e-12


def test_checks_reject_wrong_wall_temperatures():
    """Planted mistakes, made by running the oracle with the walls a faulty bc
    would produce: swapped temperatures, both walls at the mean temperature
    (right mass, wrong temperature), and both at one wall's temperature."""
    T_bot, T_top = 1.3, 0.9
    good, _ = steady_profile(T_bot, T_top)
    assert is_conduction(good, T_bot, T_top)
    for wrong in [(T_top, T_bot), (1.1, 1.1), (T_bot, T_bot), (T_top, T_top)]:
        T, _ = steady_profile(*wrong)
        assert not is_conduction(T, T_bot, T_top), wrong
