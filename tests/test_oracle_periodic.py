"""Pins of the periodic-source oracle (Sect. 3.5: eq. (split2) and the
neighbouring-frequency step eq. (4diff) of Fig. alg:spl1) against the
exact solution of eq. (ode) and against what the paper's argument needs."""
import math

import numpy as np
import pytest

import scenario as S
from oracle import exact, periodic, yee


def _case(cfg):
    if cfg == "2d":
        sc = S.config_2d(n=10, ndisks=2)
    else:
        sc = S.config_3d(n=8, fill=0.25)
    sc.g = S.masked_random_vector(sc.grid, 31)
    op = yee.Operator(sc.grid, sc.eps_cell)
    return sc, op.matrix()


@pytest.mark.parametrize("cfg", ["2d", "3d"])
@pytest.mark.parametrize("periods", [1, 2])
def test_split2_equals_exact(cfg, periods):
    """Whole periods per subinterval: the restarted result is y(T) (with a
    shorter last subinterval when T is not a multiple of dT)."""
    sc, A = _case(cfg)
    W = 1.07
    T = 37.0
    dT = periodic.period_multiple(W, T, periods)
    assert T / dT > 2 and abs(T / dT - round(T / dT)) > 0.05
    ref = exact.y_plain(A, sc.g, W, T)
    got = periodic.split2(A, sc.g, W, T, dT)
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


def test_split2_needs_whole_periods():
    """The reuse of w2 rests on the source having the same phase at every
    subinterval start: a subinterval of 0.7 periods breaks the identity."""
    sc, A = _case("2d")
    W = 1.07
    T = 37.0
    ref = exact.y_plain(A, sc.g, W, T)
    bad = periodic.split2(A, sc.g, W, T, 0.7 * 2 * math.pi / W)
    assert np.linalg.norm(bad - ref) > 1e-2 * np.linalg.norm(ref)


@pytest.mark.parametrize("cfg", ["2d", "3d"])
def test_neighbouring_frequency_steps_equal_exact(cfg):
    """Fig. alg:spl1 steps 4-6 reproduce every frequency's exact response."""
    sc, A = _case(cfg)
    oms = [0.9, 0.93, 0.96, 0.99]
    T = 25.0
    ys, dn, zn = periodic.split1_next(A, sc.g, oms, T)
    for y, W in zip(ys, oms):
        ref = exact.y_plain(A, sc.g, W, T)
        assert np.linalg.norm(y - ref) <= 1e-10 * np.linalg.norm(ref)
    # each difference problem starts from the previous frequency (step 6)
    zs = [exact.z_stat(A, sc.g, W) for W in oms]
    for j in range(1, len(oms)):
        want = np.linalg.norm(np.imag(zs[j]) - np.imag(zs[j - 1]))
        assert abs(dn[j - 1] - want) <= 1e-12 * want


def test_difference_problem_is_smaller_for_close_frequencies():
    """The premise of eq. (4diff): for neighbouring frequencies the
    difference initial value is smaller than Im z itself, and shrinks with
    the frequency step (the paper's experiments step by 0.001)."""
    sc, A = _case("2d")
    T = 25.0
    _, dn1, zn1 = periodic.split1_next(A, sc.g, [1.0, 1.001], T)
    _, dn2, zn2 = periodic.split1_next(A, sc.g, [1.0, 1.01], T)
    assert dn1[0] < 0.1 * zn1[0]
    assert dn1[0] < 0.2 * dn2[0]
