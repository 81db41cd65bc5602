"""Pins of the oracle's Q-criterion (the vortex identification of the
paper's Q-criterion figures): solid-body rotation Q = Omega^2, pure strain
Q = -a^2, simple shear Q = 0 (central and one-sided differences are exact on
linear fields, also next to solid cells), and a periodic sinusoidal vortex
field against the closed form of its central differences."""
import math

import numpy as np

PER, BB = 4, 2


def grid(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.reshape(-1).astype(float), y.reshape(-1).astype(float), z.reshape(-1).astype(float)


def test_linear_fields(O):
    nx, ny, nz = 9, 7, 5
    x, y, z = grid(nx, ny, nz)
    flags = np.zeros(nx * ny * nz, np.uint8)
    bc = [BB] * 6
    W, a, g = 0.03, 0.02, 0.05
    q = O.qcriterion(np.stack([-W * y, W * x, 0 * x]), flags, nx, ny, nz, bc)
    np.testing.assert_allclose(q, W * W, rtol=1e-12)
    q = O.qcriterion(np.stack([a * x, -a * y, 0 * x]), flags, nx, ny, nz, bc)
    np.testing.assert_allclose(q, -a * a, rtol=1e-12)
    q = O.qcriterion(np.stack([g * y, 0 * x, 0 * x]), flags, nx, ny, nz, bc)
    assert np.max(np.abs(q)) < 1e-18


def test_linear_field_next_to_solids(O):
    nx, ny, nz = 10, 8, 6
    x, y, z = grid(nx, ny, nz)
    flags = ((x >= 3) & (x < 5) & (y >= 2) & (y < 4) & (z < 3)).astype(np.uint8)
    W = 0.04
    q = O.qcriterion(np.stack([-W * y, W * x, 0 * x]), flags, nx, ny, nz, [BB] * 6)
    fl = flags == 0
    np.testing.assert_allclose(q[fl], W * W, rtol=1e-12)
    assert np.all(q[~fl] == 0)


def test_periodic_wrap(O):
    nx, ny, nz = 16, 12, 3
    x, y, z = grid(nx, ny, nz)
    kx, ky = 2 * math.pi / nx, 2 * math.pi / ny
    u = np.stack([-np.sin(ky * y), np.sin(kx * x), 0 * x])
    q = O.qcriterion(u, np.zeros(x.size, np.uint8), nx, ny, nz, [PER] * 6)
    # central differences: d/dy sin(ky y) -> cos(ky y) sin(ky), d/dx sin(kx x) -> cos(kx x) sin(kx)
    jxy = -np.cos(ky * y) * math.sin(ky)
    jyx = np.cos(kx * x) * math.sin(kx)
    np.testing.assert_allclose(q, -jxy * jyx, atol=1e-15)


def test_time_average_is_the_mean_of_snapshots(O):
    """The per-node time average equals the mean of |u| fields of separate
    runs stopped at the sampling levels."""
    VEL, OUT = 0, 1
    p = O.params(12, 6, 5, [VEL, OUT, BB, BB, BB, BB], 0.6, 0.0, 0)
    flags = np.zeros(12 * 6 * 5, np.uint8)
    Z, a = O.quadrature(0, 1, 2, [-0.1], [0.1])
    A = O.ensemble_time_average(p, flags, Z, [0], 0.05, 0.25, 0.0, 5, 20, 3, 7)
    snaps = [O.ensemble(p, flags, Z, [0], 0.05, 0.25, 0.0, 5, n) for n in (20, 27, 34)]
    np.testing.assert_allclose(A, sum(snaps) / 3, rtol=1e-14, atol=1e-18)
