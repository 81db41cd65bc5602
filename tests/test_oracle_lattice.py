"""Pins for the oracle's lattice, equilibrium and collision (Sec. 2.2).

Each check is fixed by the mathematics of D3Q19 / BGK, not by re-running the
oracle's own formula: lattice isotropy, the moments of the equilibrium, mass
and momentum conservation of the collision, BGK relaxation of the
non-equilibrium stress, and the implicit Smagorinsky relation of Eqs. tauEff
and turbVisc.
"""
import itertools
import math

import numpy as np


def test_velocity_set_and_weights(O):
    cx, cy, cz, w, opp = O.lattice()
    c = np.stack([cx, cy, cz], 1)
    # 19 distinct velocities: rest, 6 axis, 12 face diagonals (Fig. 1)
    assert len({tuple(v) for v in c}) == 19
    norms = (c ** 2).sum(1)
    assert sorted(norms.tolist()) == [0] + [1] * 6 + [2] * 12
    assert np.all(c[opp] == -c)
    assert np.all(opp[opp] == np.arange(19))
    # isotropy up to 4th order with cs^2 = 1/3
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(w @ c, 0.0, atol=1e-16)
    M2 = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.allclose(M2, np.eye(3) / 3.0, atol=1e-15)
    M3 = np.einsum("i,ia,ib,ic->abc", w, c, c, c)
    assert np.allclose(M3, 0.0, atol=1e-16)
    M4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9.0
    assert np.allclose(M4, iso, atol=1e-15)


def test_equilibrium_moments(O):
    cx, cy, cz, w, opp = O.lattice()
    c = np.stack([cx, cy, cz], 1).astype(float)
    rng = np.random.default_rng(1)
    for _ in range(20):
        rho = 1.0 + 0.2 * rng.standard_normal()
        u = 0.1 * rng.standard_normal(3)
        feq = O.equilibrium(rho, u)
        assert abs(feq.sum() - rho) < 1e-14
        assert np.allclose(c.T @ feq, rho * u, atol=1e-15)
        # second moment of the D3Q19 second-order equilibrium is exact
        P = np.einsum("i,ia,ib->ab", feq, c, c)
        assert np.allclose(P, rho / 3.0 * np.eye(3) + rho * np.outer(u, u), atol=1e-14)


def _random_f(O, rng, amp=0.02):
    feq = O.equilibrium(1.0 + 0.05 * rng.standard_normal(), 0.05 * rng.standard_normal(3))
    return feq * (1.0 + amp * rng.standard_normal(19))


def test_collision_conserves_and_relaxes(O):
    cx, cy, cz, w, opp = O.lattice()
    c = np.stack([cx, cy, cz], 1).astype(float)
    rng = np.random.default_rng(2)
    for tau0 in (0.51, 0.6, 1.3):
        p = O.params(1, 1, 1, [4] * 6, tau0, 0.0)
        for _ in range(10):
            f = _random_f(O, rng)
            fp, tau = O.collide_cell(p, f)
            assert tau == tau0
            assert abs(fp.sum() - f.sum()) < 1e-15
            assert np.allclose(c.T @ fp, c.T @ f, atol=1e-16)
            rho = f.sum()
            u = c.T @ f / rho
            feq = O.equilibrium(rho, u)
            # BGK: f* - f^eq = (1 - 1/tau)(f - f^eq), component by component
            assert np.allclose(fp - feq, (1.0 - 1.0 / tau0) * (f - feq), atol=1e-16)


def test_smagorinsky_implicit_relation(O):
    """tau_eff must satisfy Eq. tauEff with nu_turb of Eq. turbVisc, where the
    strain rate is recovered from the non-equilibrium stress of the same
    collision, S = -Pi / (2 rho cs^2 tau_eff), |S| = sqrt(2 S:S)."""
    cx, cy, cz, w, opp = O.lattice()
    c = np.stack([cx, cy, cz], 1).astype(float)
    rng = np.random.default_rng(3)
    for tau0, cs in itertools.product((0.5005, 0.55, 0.8), (0.1, 0.14, 0.25)):
        p = O.params(1, 1, 1, [4] * 6, tau0, cs)
        f = _random_f(O, rng, amp=0.05)
        fp, tau = O.collide_cell(p, f)
        rho = f.sum()
        u = c.T @ f / rho
        Pi = np.einsum("i,ia,ib->ab", f - O.equilibrium(rho, u), c, c)
        S = -Pi / (2.0 * rho * (1.0 / 3.0) * tau)
        Snorm = math.sqrt(2.0 * np.sum(S * S))
        nu0 = (tau0 - 0.5) / 3.0
        nu_eff = nu0 + (cs * 1.0) ** 2 * Snorm
        assert abs(tau - (3.0 * nu_eff + 0.5)) < 1e-12 * tau
        assert tau > tau0
        # collision is still mass/momentum conserving
        assert abs(fp.sum() - rho) < 1e-15
        assert np.allclose(c.T @ fp, rho * u, atol=1e-16)


def test_ramp_shape(O):
    assert O.ramp(0, 1) == 1.0
    assert O.ramp(0, 10 ** 6) == 1.0
    Tr = 1000
    assert O.ramp(Tr, 0) == 0.0
    assert abs(O.ramp(Tr, Tr // 2) - 0.5) < 1e-15
    assert O.ramp(Tr, Tr) == 1.0 and O.ramp(Tr, 5 * Tr) == 1.0
    vals = [O.ramp(Tr, m) for m in range(Tr + 1)]
    assert all(b >= a for a, b in zip(vals, vals[1:]))
