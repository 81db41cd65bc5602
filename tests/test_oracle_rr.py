"""Pins of the oracle's recursive regularized collision (Sec. 2.2, Eq.
deterministicLBE with the regularized non-equilibrium and the third-order
equilibrium, Eq. hermiteCoeff).

A D3Q19 state is fixed by its 19 moments.  The model fixes them as follows
(checked here from the definitions of the Hermite polynomials, not from the
oracle's formulas):
  - equilibrium: density rho, momentum rho u, second-order Hermite moments
    rho u_a u_b, and for the six third-order combinations D3Q19 carries
    (H_xxy +- H_yzz, H_xzz +- H_xyy, H_yyz +- H_xxz) the matching
    combinations of rho u_a u_b u_g; its three remaining (ghost) moments are
    those of the projection and nothing else;
  - after collision: the same density and momentum, second-order moments
    rho u u + (1 - 1/tau) a2 with a2 the non-equilibrium stress of the
    incoming state, third-order combinations of rho u u u + (1 - 1/tau) a3
    with a3_abg = u_a a2_bg + u_b a2_ag + u_g a2_ab (the recursion), and the
    ghost moments of the equilibrium.
"""
import itertools
import math

import numpy as np
import pytest

PER = 4
CS2 = 1.0 / 3.0
TRIPLES = [((0, 0, 1), (1, 2, 2)), ((0, 2, 2), (0, 1, 1)), ((1, 1, 2), (0, 0, 2))]


@pytest.fixture(scope="module")
def lat(O):
    cx, cy, cz, w, _ = O.lattice()
    c = np.stack([cx, cy, cz], 1).astype(float)
    return c, np.asarray(w, float)


def h2(c, a, b):
    return c[:, a] * c[:, b] - (CS2 if a == b else 0.0)


def h3(c, a, b, g):
    d = lambda i, j: 1.0 if i == j else 0.0
    return c[:, a] * c[:, b] * c[:, g] - CS2 * (c[:, a] * d(b, g) + c[:, b] * d(a, g) + c[:, g] * d(a, b))


def combos(c):
    """The six third-order combinations as polynomials of c (sums, then differences)."""
    out = []
    for sign in (1.0, -1.0):
        for t0, t1 in TRIPLES:
            out.append(h3(c, *t0) + sign * h3(c, *t1))
    return out


def tensor_combos(T3):
    out = []
    for sign in (1.0, -1.0):
        for t0, t1 in TRIPLES:
            out.append(T3[t0] + sign * T3[t1])
    return np.array(out)


def ghost_basis(c, w):
    """Polynomials orthogonal (under the weights) to 1, c, H2 and the six
    third-order combinations: the three ghost moments of D3Q19."""
    cols = [np.ones(19)] + [c[:, a] for a in range(3)]
    cols += [h2(c, a, b) for a in range(3) for b in range(a, 3)]
    cols += combos(c)
    M = np.stack(cols, 1) * np.sqrt(w)[:, None]
    u, s, _ = np.linalg.svd(M, full_matrices=True)
    rank = int(np.sum(s > 1e-12))
    assert rank == 16
    return u[:, rank:] / np.sqrt(w)[:, None]   # columns: ghost polynomials at c_i


def moments_ok(c, f, rho, u, a2, a3, keep):
    assert abs(f.sum() - rho) < 1e-14
    np.testing.assert_allclose(c.T @ f, rho * u, atol=1e-15)
    for a in range(3):
        for b in range(3):
            assert abs(h2(c, a, b) @ f - (rho * u[a] * u[b] + keep * a2[a, b])) < 1e-15
    want = tensor_combos(rho * np.einsum("a,b,g->abg", u, u, u) + keep * a3)
    got = np.array([hk @ f for hk in combos(c)])
    np.testing.assert_allclose(got, want, atol=1e-16)


def test_third_order_equilibrium_moments(O, lat):
    c, w = lat
    rng = np.random.default_rng(5)
    G = ghost_basis(c, w)
    for _ in range(20):
        rho = 1.0 + 0.05 * rng.standard_normal()
        u = 0.1 * rng.standard_normal(3)
        feq = O.equilibrium3(rho, u)
        moments_ok(c, feq, rho, u, np.zeros((3, 3)), np.zeros((3, 3, 3)), 0.0)
        # the third-order terms touch no moment of order <= 2 and no ghost
        d = feq - O.equilibrium(rho, u)
        assert abs(d.sum()) < 1e-16 and np.max(np.abs(c.T @ d)) < 1e-16
        assert max(abs(h2(c, a, b) @ d) for a in range(3) for b in range(3)) < 1e-16
        assert np.max(np.abs(G.T @ d)) < 1e-16


@pytest.mark.parametrize("csmag", [0.0, 0.14, 0.25])
def test_regularized_collision_moments(O, lat, csmag):
    c, w = lat
    G = ghost_basis(c, w)
    rng = np.random.default_rng(11)
    tau0 = 0.62
    p = O.params(1, 1, 1, [PER] * 6, tau0, csmag, collision=O.RR)
    for _ in range(20):
        rho0 = 1.0 + 0.05 * rng.standard_normal()
        u0 = 0.08 * rng.standard_normal(3)
        f = O.equilibrium3(rho0, u0) + 1e-3 * w * rng.standard_normal(19)   # every moment disturbed
        fpost, tau = O.collide_cell(p, f)
        rho = f.sum()
        u = c.T @ f / rho
        a2 = np.array([[h2(c, a, b) @ f - rho * u[a] * u[b] for b in range(3)] for a in range(3)])
        a3 = (np.einsum("a,bg->abg", u, a2) + np.einsum("b,ag->abg", u, a2)
              + np.einsum("g,ab->abg", u, a2))
        want_tau = tau0
        if csmag:
            want_tau = 0.5 * (tau0 + math.sqrt(tau0 ** 2 + 18 * csmag ** 2 * math.sqrt(2 * np.sum(a2 * a2)) / rho))
        assert abs(tau - want_tau) < 1e-14
        moments_ok(c, fpost, rho, u, a2, a3, 1.0 - 1.0 / tau)
        # ghosts are those of the equilibrium: regularization removes them
        assert np.max(np.abs(G.T @ (fpost - O.equilibrium3(rho, u)))) < 1e-15
        assert np.max(np.abs(G.T @ (f - O.equilibrium3(rho, u)))) > 1e-5  # the input had some


def test_regularized_equals_bgk_for_a_second_order_state_at_rest(O, lat):
    """At u = 0 a state whose non-equilibrium is a pure second-order Hermite
    mode is already regular: both collision forms give the same result."""
    c, w = lat
    rng = np.random.default_rng(3)
    for _ in range(10):
        Pi = rng.standard_normal((3, 3)) * 1e-3
        Pi = Pi + Pi.T
        f = O.equilibrium(1.02, np.zeros(3)) + w * 4.5 * sum(h2(c, a, b) * Pi[a, b]
                                                             for a in range(3) for b in range(3))
        for cs in (0.0, 0.2):
            fr, tr = O.collide_cell(O.params(1, 1, 1, [PER] * 6, 0.7, cs, collision=O.RR), f)
            fb, tb = O.collide_cell(O.params(1, 1, 1, [PER] * 6, 0.7, cs, collision=O.BGK), f)
            assert abs(tr - tb) < 1e-15
            np.testing.assert_allclose(fr, fb, atol=1e-16)


def _tg_rate_rr(O, N, tau, t1, t2, U=0.01):
    p = O.params(N, N, 1, [PER] * 6, tau, 0.0, collision=O.RR)
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
    O.run(p, flags, uin, f, t1, t2 - t1)
    r2, u2 = O.macros(p, flags, f)
    rate = -math.log(np.sum(r2 * (u2 ** 2).sum(0)) / np.sum(r1 * (u1 ** 2).sum(0))) / (t2 - t1)
    return rate, 4.0 * (tau - 0.5) / 3.0 * k * k


def test_regularized_taylor_green_viscosity(O):
    """The regularized model keeps nu = (tau - 1/2)/3: Taylor-Green energy
    decays at 4 nu k^2 within 1% at N = 64, converging at second order."""
    r32, e32 = _tg_rate_rr(O, 32, 0.8, 60, 300)
    r64, e64 = _tg_rate_rr(O, 64, 0.8, 240, 1200)
    err32, err64 = abs(r32 / e32 - 1.0), abs(r64 / e64 - 1.0)
    assert err64 < 0.01
    assert 3.0 < err32 / err64 < 5.0


def test_regularized_rejects_body_force(O):
    p = O.params(1, 1, 1, [PER] * 6, 0.7, 0.0, force=(1e-6, 0, 0), collision=O.RR)
    with pytest.raises(Exception):
        O.collide_cell(p, O.equilibrium(1.0, np.zeros(3)))
