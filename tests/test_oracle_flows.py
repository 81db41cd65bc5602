"""Physics pins for the oracle's lattice Boltzmann solver (Sec. 2.2).

Analytic flows and exact invariants that the discrete method must reproduce:
Couette (linear profile, exact for half-way walls), force-driven Poiseuille
(parabola; exact at the BGK 'magic' relaxation time, second order otherwise),
Taylor-Green decay (viscosity nu = (tau - 1/2)/3), uniform equilibrium flow as
a fixed point of every boundary kind, mass / momentum conservation and mirror
symmetry.
"""
import math

import numpy as np
import pytest

VEL, OUT, BB, FS, PER = 0, 1, 2, 3, 4


def _column_run(O, nz, tau, bc_lo, bc_hi, steps, U=0.0, force=(0, 0, 0)):
    p = O.params(1, 1, nz, [PER, PER, PER, PER, bc_lo, bc_hi], tau, 0.0, 0, force)
    flags = np.zeros(nz, np.uint8)
    uin = np.zeros((nz, 3))
    uin[:, 0] = U
    f = O.init_equilibrium(p, flags)
    O.run(p, flags, uin, f, 0, steps)
    cx = np.array(O.lattice()[0], float)
    rho = f.sum(0)
    ux = (cx @ f + 0.5 * force[0]) / rho
    return ux


def test_couette_linear_profile(O):
    nz, U, tau = 16, 0.02, 0.8
    ux = _column_run(O, nz, tau, BB, VEL, 9000, U=U)
    h = np.arange(nz) + 0.5
    exact = U * h / nz          # walls half-way: z = -1/2 (rest) and nz - 1/2 (moving)
    assert np.max(np.abs(ux - exact)) < 1e-12 * U / 1e-2


def _poiseuille_err(O, nz, tau, F=1e-6):
    nu = (tau - 0.5) / 3.0
    steps = int(40 * nz * nz / (math.pi ** 2 * nu)) + 200
    ux = _column_run(O, nz, tau, BB, BB, steps, force=(F, 0, 0))
    h = np.arange(nz) + 0.5
    exact = F / (2.0 * nu) * h * (nz - h)
    return np.max(np.abs(ux - exact)) / np.max(exact)


def test_poiseuille_magic_tau_exact(O):
    tau = 0.5 + math.sqrt(3.0 / 16.0)
    assert _poiseuille_err(O, 12, tau) < 1e-9


def test_poiseuille_second_order(O):
    e8 = _poiseuille_err(O, 8, 0.6)
    e16 = _poiseuille_err(O, 16, 0.6)
    e32 = _poiseuille_err(O, 32, 0.6)
    assert e16 < 0.05
    assert 3.5 < e8 / e16 < 4.5
    assert 3.5 < e16 / e32 < 4.5


def _tg_rate(O, N, tau, t1, t2, U=0.01):
    p = O.params(N, N, 1, [PER] * 6, tau, 0.0)
    flags = np.zeros(N * N, np.uint8)
    k = 2 * math.pi / N
    x, y = np.meshgrid(np.arange(N), np.arange(N), indexing="xy")
    u = np.zeros((3, N * N))
    u[0] = (-U * np.cos(k * x) * np.sin(k * y)).reshape(-1)
    u[1] = (U * np.sin(k * x) * np.cos(k * y)).reshape(-1)
    f = O.init_equilibrium(p, flags, None, u)
    uin = np.zeros((1, 3))
    O.run(p, flags, uin, f, 0, t1)
    r1, u1 = O.macros(p, flags, f)
    E1 = np.sum(r1 * (u1 ** 2).sum(0))
    O.run(p, flags, uin, f, t1, t2 - t1)
    r2, u2 = O.macros(p, flags, f)
    E2 = np.sum(r2 * (u2 ** 2).sum(0))
    rate = -math.log(E2 / E1) / (t2 - t1)
    nu = (tau - 0.5) / 3.0
    return rate, 4.0 * nu * k * k


def test_taylor_green_decay(O):
    tau = 0.8
    r32, e32 = _tg_rate(O, 32, tau, 60, 300)
    r64, e64 = _tg_rate(O, 64, tau, 240, 1200)
    err32 = abs(r32 / e32 - 1.0)
    err64 = abs(r64 / e64 - 1.0)
    assert err64 < 0.01
    assert 3.0 < err32 / err64 < 5.0


def test_uniform_flow_is_fixed_point_of_all_boundaries(O):
    """f^eq(1, U) is reproduced exactly by velocity faces (moving-wall term),
    the outflow copy and specular free-slip reflection, at any flow angle."""
    nx, ny, nz = 12, 8, 6
    th = math.radians(10.0)
    Uv = np.array([0.04 * math.cos(th), 0.04 * math.sin(th), 0.0])
    p = O.params(nx, ny, nz, [VEL, OUT, VEL, VEL, FS, FS], 0.6, 0.14)
    flags = np.zeros(nx * ny * nz, np.uint8)
    n = flags.size
    u = np.repeat(Uv[:, None], n, 1)
    f = O.init_equilibrium(p, flags, None, u)
    f0 = f.copy()
    uin = np.repeat(Uv[None, :], nz, 0)
    O.run(p, flags, uin, f, 0, 40)
    assert np.max(np.abs(f - f0)) < 1e-15


def test_wrong_boundary_breaks_fixed_point(O):
    """Control for the fixed-point pin: a no-slip ground is not a fixed point."""
    nx, ny, nz = 12, 8, 6
    Uv = np.array([0.04, 0.0, 0.0])
    p = O.params(nx, ny, nz, [VEL, OUT, VEL, VEL, BB, FS], 0.6, 0.0)
    flags = np.zeros(nx * ny * nz, np.uint8)
    f = O.init_equilibrium(p, flags, None, np.repeat(Uv[:, None], flags.size, 1))
    f0 = f.copy()
    O.run(p, flags, np.repeat(Uv[None, :], nz, 0), f, 0, 5)
    assert np.max(np.abs(f - f0)) > 1e-6


def _perturbed_state(O, p, flags, seed, amp=0.02):
    rng = np.random.default_rng(seed)
    n = flags.size
    rho = 1.0 + 0.01 * rng.standard_normal(n)
    u = 0.03 * rng.standard_normal((3, n))
    f = O.init_equilibrium(p, flags, rho, u)
    f *= 1.0 + amp * rng.standard_normal(f.shape)
    f[:, flags != 0] = 0.0
    return f


def test_closed_box_conserves_mass(O):
    nx, ny, nz = 14, 10, 9
    # buildings, one of them touching the free-slip lid (fallback links)
    flags = O.geometry(nx, ny, nz, boxes=[[3, 2, 0, 6, 5, 4], [8, 4, 0, 11, 8, 9]])
    p = O.params(nx, ny, nz, [BB, BB, BB, BB, BB, FS], 0.55, 0.14)
    f = _perturbed_state(O, p, flags, 5)
    m0 = f.sum()
    O.run(p, flags, np.zeros((nz, 3)), f, 0, 30)
    assert abs(f.sum() - m0) < 1e-12 * m0


def test_periodic_box_conserves_mass_and_momentum(O):
    nx, ny, nz = 10, 8, 6
    flags = np.zeros(nx * ny * nz, np.uint8)
    p = O.params(nx, ny, nz, [PER] * 6, 0.52, 0.2)
    f = _perturbed_state(O, p, flags, 6)
    cx, cy, cz, w, opp = O.lattice()
    c = np.stack([cx, cy, cz], 1).astype(float)
    m0, j0 = f.sum(), c.T @ f.sum(1)
    O.run(p, flags, np.zeros((nz, 3)), f, 0, 25)
    assert abs(f.sum() - m0) < 1e-12 * m0
    assert np.allclose(c.T @ f.sum(1), j0, atol=1e-13)


def test_mirror_symmetry_in_y(O):
    """A y-symmetric domain with a y-symmetric inflow gives a y-symmetric flow
    (u_x even, u_y odd): catches index and sign slips in y."""
    nx, ny, nz = 20, 10, 8
    flags = O.geometry(nx, ny, nz, boxes=[[6, 3, 0, 9, 7, 4], [12, 0, 0, 14, 2, 3],
                                          [12, 8, 0, 14, 10, 3]])
    p = O.params(nx, ny, nz, [VEL, OUT, VEL, VEL, BB, FS], 0.56, 0.14, 20)
    uin = O.inflow(nz, 0.05, 0.0, 0.25, nz, 0.0)
    f = O.init_equilibrium(p, flags)
    O.run(p, flags, uin, f, 0, 60)
    _, u = O.macros(p, flags, f)
    U = u.reshape(3, nz, ny, nx)
    assert np.max(np.abs(U[0])) > 1e-3
    assert np.max(np.abs(U[0] - U[0][:, ::-1, :])) < 1e-14
    assert np.max(np.abs(U[1] + U[1][:, ::-1, :])) < 1e-14
    assert np.max(np.abs(U[2] - U[2][:, ::-1, :])) < 1e-14


def test_outflow_is_zero_gradient(O):
    """Outflow face: every incoming population at an outlet cell equals the one
    its upstream neighbour (x = nx - 2) receives from the same source, i.e. a
    zero normal gradient, whenever that source cell is fluid."""
    nx, ny, nz = 16, 9, 7
    flags = O.geometry(nx, ny, nz, boxes=[[4, 2, 0, 7, 5, 4], [14, 6, 0, 16, 9, 3]])
    p = O.params(nx, ny, nz, [VEL, OUT, VEL, VEL, BB, FS], 0.56, 0.14)
    f = _perturbed_state(O, p, flags, 8)
    uin = O.inflow(nz, 0.05, 0.0, 0.25, nz, 15.0)
    O.run(p, flags, uin, f, 0, 9)
    F = flags.reshape(nz, ny, nx)
    cx, cy, cz, w, opp = O.lattice()
    checked = 0
    for z in range(nz):
        for y in range(ny):
            if F[z, y, nx - 1] or F[z, y, nx - 2]:
                continue
            for i in range(19):
                if cx[i] != -1:
                    continue
                sy, sz = y - cy[i], z - cz[i]
                if not (0 <= sy < ny and 0 <= sz < nz) or F[sz, sy, nx - 1]:
                    continue
                a = f[i, (nx - 1) + nx * (y + ny * z)]
                b = f[i, (nx - 2) + nx * (y + ny * z)]
                assert a == b
                checked += 1
    assert checked > 100


def test_free_slip_equals_mirror_extension(O):
    """Specular free-slip at the lid z = nz - 1/2 must reproduce the lower half
    of the domain mirrored in z (height 2 nz, geometry and inflow mirrored,
    a wall at both ends)."""
    nx, ny, nz = 14, 8, 5
    boxes = [[4, 2, 0, 7, 5, 3], [9, 4, 0, 11, 8, 5]]      # one block reaches the lid
    flagsA = O.geometry(nx, ny, nz, boxes=boxes)
    mirrored = boxes + [[b[0], b[1], 2 * nz - b[5], b[3], b[4], 2 * nz - b[2]] for b in boxes]
    flagsB = O.geometry(nx, ny, 2 * nz, boxes=mirrored)
    pA = O.params(nx, ny, nz, [VEL, OUT, VEL, VEL, BB, FS], 0.57, 0.14, 10)
    pB = O.params(nx, ny, 2 * nz, [VEL, OUT, VEL, VEL, BB, BB], 0.57, 0.14, 10)
    uA = O.inflow(nz, 0.05, 0.05, 0.3, nz, 8.0)
    uB = np.concatenate([uA, uA[::-1]])
    fA = O.init_equilibrium(pA, flagsA)
    fB = O.init_equilibrium(pB, flagsB)
    O.run(pA, flagsA, uA, fA, 0, 40)
    O.run(pB, flagsB, uB, fB, 0, 40)
    _, vA = O.macros(pA, flagsA, fA)
    _, vB = O.macros(pB, flagsB, fB)
    VA = vA.reshape(3, nz, ny, nx)
    VB = vB.reshape(3, 2 * nz, ny, nx)
    assert np.max(np.abs(VA[0])) > 1e-3
    assert np.max(np.abs(VA - VB[:, :nz])) < 1e-14
