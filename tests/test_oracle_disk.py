"""Pins of the oracle's circular domain: the paper's cylinder of radius R
whose mantle carries a local velocity boundary (Sec. 2.2 boundary list,
Sec. 3 domain).  Columns whose centre lies beyond R from the axis are flag 2;
a link from a fluid cell into them takes the moving-wall velocity rule.

Checked against row counts worked out by hand, the area of the disk, the
exactness of the velocity rule for a uniform equilibrium flow (every
population is then reproduced), and the 90-degree symmetry of D3Q19."""
import math

import numpy as np
import pytest

VEL, OUT, BB, FS = 0, 1, 2, 3


def test_mantle_rows_hand_worked(O):
    """R = 4 on 10 x 10: row y has centre offset dy = y - 4.5; a cell is
    inside when dx^2 <= 16 - dy^2 with dx in +-0.5, +-1.5, ...:
    |dy| = 4.5 -> none; 3.5 -> |dx| <= 1.94 (4 cells); 2.5 -> 3.12 (6);
    1.5 and 0.5 -> 3.71 and 3.97 (8)."""
    f = O.geometry(10, 10, 3, disk_radius=4.0).reshape(3, 10, 10)
    for z in range(3):
        inside = (f[z] == 0).sum(axis=1)
        assert list(inside) == [0, 4, 6, 8, 8, 8, 8, 6, 4, 0]
        assert set(np.unique(f[z])) == {0, 2}


def test_mantle_area_and_symmetry(O):
    N, R = 64, 27.3
    f = O.geometry(N, N, 1, disk_radius=R).reshape(N, N)
    inside = f == 0
    assert abs(inside.sum() - math.pi * R * R) < 2 * math.pi * R
    for g in (inside.T, inside[::-1], inside[:, ::-1], np.rot90(inside)):
        assert np.array_equal(g, inside)


def test_buildings_inside_stay_solid(O):
    f = O.geometry(20, 20, 6, boxes=[[8, 8, 0, 12, 12, 3], [0, 0, 0, 3, 3, 6]], disk_radius=9.0)
    f = f.reshape(6, 20, 20)
    assert (f[:3, 8:12, 8:12] == 1).all()         # the centred block
    assert (f[:, 0:3, 0:3] == 2).all()            # a block beyond the mantle is outside


def disk_case(O, N, nz, R, alpha, theta, ramp, boxes=None):
    p = O.params(N, N, nz, [VEL, VEL, VEL, VEL, FS, FS], 0.6, 0.0, ramp)
    flags = O.geometry(N, N, nz, boxes=boxes, disk_radius=R)
    uin = O.inflow(nz, 0.04, 0.0, alpha, nz, theta)
    return p, flags, uin


def test_uniform_flow_is_kept_exactly(O):
    """A uniform equilibrium flow at the mantle's velocity is a steady state:
    bounce-back plus 6 w_i (c_i . u) turns f_eq,opp(i) into f_eq,i exactly,
    and free-slip lids reflect a horizontal flow onto itself."""
    N, nz = 20, 6
    p, flags, uin = disk_case(O, N, nz, 9.0, 0.0, 30.0, 0)
    u = np.zeros((3, N * N * nz))
    u[0], u[1] = uin[0, 0], uin[0, 1]
    f0 = O.init_equilibrium(p, flags, None, u)
    f = f0.copy()
    O.run(p, flags, uin, f, 0, 40)
    assert np.max(np.abs(f - f0)) < 1e-14   # rounding of 40 steps
    # the same flow against walls instead of the mantle's velocity rule decays
    p2 = O.params(N, N, nz, [VEL, VEL, VEL, VEL, FS, FS], 0.6, 0.0, 0)
    solid = np.where(flags == 2, 1, flags).astype(np.uint8)
    fw = O.init_equilibrium(p2, solid, None, u)
    O.run(p2, solid, uin, fw, 0, 40)
    assert np.max(np.abs(fw - f0)) > 1e-3


def test_turned_inflow_gives_the_turned_flow(O):
    """Centred square block: the inflow turned by 90 degrees gives the flow
    turned by 90 degrees about the axis, cell by cell."""
    N, nz = 20, 6
    box = [[8, 8, 0, 12, 12, 3]]
    pa, flags, ua = disk_case(O, N, nz, 9.0, 0.25, 10.0, 5, box)
    _, _, ub = disk_case(O, N, nz, 9.0, 0.25, 100.0, 5, box)
    fa = O.init_equilibrium(pa, flags)
    O.run(pa, flags, ua, fa, 0, 30)
    fb = O.init_equilibrium(pa, flags)
    O.run(pa, flags, ub, fb, 0, 30)
    va = O.macros(pa, flags, fa)[1].reshape(3, nz, N, N)
    vb = O.macros(pa, flags, fb)[1].reshape(3, nz, N, N)
    src = np.empty_like(va)
    for y in range(N):
        for x in range(N):
            src[:, :, y, x] = va[:, :, N - 1 - x, y]
    np.testing.assert_allclose(vb, np.stack([-src[1], src[0], src[2]]), rtol=0, atol=1e-14)
    assert np.max(np.abs(vb - va)) > 1e-3


@pytest.mark.parametrize("theta", [0.0, 35.0, 130.0])
def test_mantle_drives_the_flow_along_the_wind(O, theta):
    """Fluid at rest, an empty disk: the mantle's velocity boundary sets the
    whole disk moving along the wind direction (mean direction in the
    central region within 2 degrees, speed approaching the inflow's)."""
    N, nz = 24, 4
    p, flags, uin = disk_case(O, N, nz, 11.0, 0.0, theta, 20)
    f = O.init_equilibrium(p, flags)
    O.run(p, flags, uin, f, 0, 400)
    u = O.macros(p, flags, f)[1].reshape(3, nz, N, N)
    c = u[:, :, 8:16, 8:16].reshape(3, -1).mean(axis=1)
    ang = math.degrees(math.atan2(c[1], c[0]))
    assert abs((ang - theta + 180.0) % 360.0 - 180.0) < 2.0
    assert 0.5 * 0.04 < math.hypot(c[0], c[1]) < 1.1 * 0.04
