"""Pins for the oracle's seeded geometry, probes and inflow table.

SplitMix64 is checked against its published reference outputs; the building
generator against the properties its definition fixes; the power-law inflow
against its closed form.
"""
import math

import numpy as np

from conftest import golden


def test_splitmix64_reference_vectors(O):
    by_seed = {}
    for seed, k, v in golden("splitmix64.txt"):
        by_seed.setdefault(int(seed), {})[int(k)] = int(v)
    for seed, outs in by_seed.items():
        got = O.splitmix64(seed, max(outs))
        for k, v in outs.items():
            assert int(got[k - 1]) == v


def test_explicit_cube(O):
    nx, ny, nz = 48, 24, 24
    flags = O.geometry(nx, ny, nz, boxes=[[12, 8, 0, 20, 16, 12]])
    F = flags.reshape(nz, ny, nx)
    assert F.sum() == 8 * 8 * 12
    assert F[0:12, 8:16, 12:20].all()
    assert F[12, 8, 12] == 0 and F[0, 7, 12] == 0 and F[0, 8, 20] == 0


def test_seeded_buildings_properties(O):
    nx, ny, nz = 256, 128, 64
    flags = O.geometry(nx, ny, nz, 2025, 24, 8, 24, 10, 40)
    F = flags.reshape(nz, ny, nx).astype(bool)
    # ground footprint is the union of at most 24 rectangles inside the bounds
    foot = F[0]
    assert foot.any()
    assert not foot[:, : nx // 8].any() and not foot[:, nx - nx // 8:].any()
    assert not foot[:2].any() and not foot[ny - 2:].any()
    # buildings are vertical prisms from the ground, at most min(40, nz-4) tall
    for z in range(1, nz):
        assert not (F[z] & ~F[z - 1]).any()
    assert F[9].sum() == foot.sum()            # every height >= 10
    assert not F[40].any() and F[:40].any()
    # solid fraction plausible for 24 blocks of 8..24 cells footprint
    frac = F.mean()
    assert 0.005 < frac < 0.3
    # determinism and seed dependence
    assert np.array_equal(flags, O.geometry(nx, ny, nz, 2025, 24, 8, 24, 10, 40))
    assert not np.array_equal(flags, O.geometry(nx, ny, nz, 2026, 24, 8, 24, 10, 40))


def test_probe_columns_and_points(O):
    nx, ny, nz = 256, 128, 64
    flags = O.geometry(nx, ny, nz, 2025, 24, 8, 24, 10, 40)
    F = flags.reshape(nz, ny, nx)
    xy = O.probe_columns(nx, ny, nz, 2025, flags, 4)
    assert len({tuple(v) for v in xy}) == 4
    for x, y in xy:
        assert nx // 8 <= x < nx and 0 <= y < ny and F[0, y, x] == 0
    pts = O.probe_points(nx, ny, nz, 7, flags, 16)
    assert len({tuple(v) for v in pts}) == 16
    for x, y, z in pts:
        assert nx // 8 <= x < nx and 0 <= y < ny and 0 <= z <= nz - 3 and F[z, y, x] == 0


def test_power_law_inflow(O):
    nz, H = 24, 24.0
    uin = O.inflow(nz, 0.05, 0.1, 0.25, H, 30.0)
    for k in range(nz):
        mag = 0.05 * 1.1 * ((k + 0.5) / H) ** 0.25
        assert abs(uin[k, 0] - mag * math.cos(math.pi / 6)) < 1e-16
        assert abs(uin[k, 1] - mag * 0.5) < 1e-16
        assert uin[k, 2] == 0.0
    # monotone in height, speed at the reference height equals u_ref (1 + xi)
    assert np.all(np.diff(np.hypot(uin[:, 0], uin[:, 1])) > 0)
