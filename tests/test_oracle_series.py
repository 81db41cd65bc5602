"""Pins of the oracle's time-varying inflow: hourly targets of wind speed and
direction with an interpolation interval between them (Sec. 2.2, the
boundary velocity is moved gradually to the next magnitude and direction;
Sec. 2.4 step 1 and Sec. 3, one target per hour of measurements).

The schedule is checked against values worked out by hand from that reading;
the stepping under it against the steady solver (a constant series, a jump)
and against the rotational symmetry of D3Q19 about z (a series turned by 90
degrees gives the turned flow)."""
import math

import numpy as np
import pytest

VEL, OUT, BB, FS = 0, 1, 2, 3
SPEED = [1.0, 1.4, 0.8]
DIRS = [0.0, 30.0, -20.0]


@pytest.mark.parametrize("m,want", [
    (0, (1.0, 0.0)), (9, (1.0, 0.0)), (10, (1.0, 0.0)),       # target 0; level 10 starts the move
    (11, (1.1, 7.5)), (12, (1.2, 15.0)), (14, (1.4, 30.0)),   # lam = 1/4, 1/2, 1
    (19, (1.4, 30.0)), (20, (1.4, 30.0)),                       # hold of target 1
    (21, (1.25, 17.5)), (23, (0.95, -7.5)), (24, (0.8, -20.0)),
    (30, (0.8, -20.0)), (10 ** 6, (0.8, -20.0)),                # after the last target
])
def test_schedule_hand_values(O, m, want):
    s, d = O.series_at(SPEED, DIRS, 10, 4, m)
    assert abs(s - want[0]) < 1e-15 and abs(d - want[1]) < 1e-13


def test_schedule_jump_without_interval(O):
    assert O.series_at(SPEED, DIRS, 10, 0, 9) == (1.0, 0.0)
    assert O.series_at(SPEED, DIRS, 10, 0, 10) == (1.4, 30.0)
    assert O.series_at(SPEED, DIRS, 10, 0, 20) == (0.8, -20.0)


def unit(d):
    return np.array([math.cos(math.radians(d)), math.sin(math.radians(d))])


@pytest.mark.parametrize("dirs,mid", [((350.0, 10.0), 0.0), ((10.0, 350.0), 0.0),
                                      ((170.0, -170.0), 180.0), ((0.0, 180.0), -90.0),
                                      ((0.0, 90.0), 45.0)])
def test_direction_takes_the_shorter_arc(O, dirs, mid):
    """Midway through the move the direction is the arc's midpoint (a half
    turn goes clockwise); the hold afterwards points at the target."""
    _, d = O.series_at([1.0, 1.0], list(dirs), 4, 4, 6)
    np.testing.assert_allclose(unit(d), unit(mid), atol=1e-15)
    _, d = O.series_at([1.0, 1.0], list(dirs), 4, 4, 100)
    np.testing.assert_allclose(unit(d), unit(dirs[1]), atol=1e-15)


def channel(O, nx, ny, nz, bc, ramp):
    p = O.params(nx, ny, nz, bc, 0.56, 0.14, ramp)
    flags = np.zeros(nx * ny * nz, np.uint8)
    return p, flags


def series_inflow(O, p, u_ref, alpha, H, theta, series):
    speed, dirs, per, interp = series

    def at(m):
        s, d = O.series_at(speed, dirs, per, interp, m)
        return O.ramp(p.ramp_steps, m) * O.inflow(p.nz, u_ref * s, 0.0, alpha, H, theta + d)
    return at


def test_constant_series_equals_the_steady_run(O):
    """Targets that never change (a full turn included) give the steady
    inflow at u_ref * s and theta + delta, ramp and all."""
    nx, ny, nz = 10, 8, 6
    p, flags = channel(O, nx, ny, nz, [VEL, OUT, VEL, VEL, BB, FS], 6)
    series = ([1.3, 1.3, 1.3], [25.0, 25.0, 385.0], 7, 3)
    f1 = O.init_equilibrium(p, flags)
    O.run_series(p, flags, f1, 0, 30, series_inflow(O, p, 0.05, 0.25, nz, 5.0, series))
    f2 = O.init_equilibrium(p, flags)
    O.run(p, flags, O.inflow(nz, 0.05 * 1.3, 0.0, 0.25, nz, 30.0), f2, 0, 30)
    np.testing.assert_allclose(f1, f2, rtol=0, atol=2e-15)


def test_jump_equals_two_steady_segments(O):
    """Without an interval target 1 drives every arrival level from
    steps_per_target on: the run equals steady target 0 up to level P - 1,
    then steady target 1."""
    nx, ny, nz = 10, 8, 6
    P = 12
    p, flags = channel(O, nx, ny, nz, [VEL, OUT, VEL, VEL, BB, FS], 4)
    series = ([1.0, 0.7], [0.0, -35.0], P, 0)
    f1 = O.init_equilibrium(p, flags)
    O.run_series(p, flags, f1, 0, 30, series_inflow(O, p, 0.05, 0.25, nz, 10.0, series))
    f2 = O.init_equilibrium(p, flags)
    O.run(p, flags, O.inflow(nz, 0.05, 0.0, 0.25, nz, 10.0), f2, 0, P - 1)
    O.run(p, flags, O.inflow(nz, 0.035, 0.0, 0.25, nz, -25.0), f2, P - 1, 30 - (P - 1))
    np.testing.assert_allclose(f1, f2, rtol=0, atol=2e-15)
    # and it differs from holding target 0 throughout
    f3 = O.init_equilibrium(p, flags)
    O.run(p, flags, O.inflow(nz, 0.05, 0.0, 0.25, nz, 10.0), f3, 0, 30)
    assert np.max(np.abs(f1 - f3)) > 1e-4


def test_turned_series_gives_the_turned_flow(O):
    """Square domain with inflow on all four sides: the series turned by 90
    degrees (every target) gives the flow of the original series turned by
    90 degrees about z, cell by cell, during the interpolation interval."""
    N, nz = 10, 6
    p, flags = channel(O, N, N, nz, [VEL, VEL, VEL, VEL, BB, FS], 3)
    A = ([1.0, 1.25], [0.0, 40.0], 8, 6)
    B = ([1.0, 1.25], [90.0, 130.0], 8, 6)
    fa = O.init_equilibrium(p, flags)
    O.run_series(p, flags, fa, 0, 12, series_inflow(O, p, 0.05, 0.25, nz, 0.0, A))
    fb = O.init_equilibrium(p, flags)
    O.run_series(p, flags, fb, 0, 12, series_inflow(O, p, 0.05, 0.25, nz, 0.0, B))
    _, ua = O.macros(p, flags, fa)
    _, ub = O.macros(p, flags, fb)
    ua = ua.reshape(3, nz, N, N)     # [comp][z][y][x]
    ub = ub.reshape(3, nz, N, N)
    # u_B(i, j) = R u_A(j, N - 1 - i), R (ux, uy) = (-uy, ux); arrays indexed [y][x]
    src = np.empty_like(ua)
    for y in range(N):
        for x in range(N):
            src[:, :, y, x] = ua[:, :, N - 1 - x, y]
    turned = np.stack([-src[1], src[0], src[2]])
    np.testing.assert_allclose(ub, turned, rtol=0, atol=1e-14)
    assert np.max(np.abs(ub - ua)) > 1e-3   # the two flows do differ
