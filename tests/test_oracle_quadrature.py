"""Pins for the oracle's quadrature rules, moments and gPC projection
(Sec. 2.3, Eqs. gPC, coef_discrete, quad_moments).

Fixed from outside the oracle: Abramowitz & Stegun's Gauss-Legendre table,
Clenshaw-Curtis rational weights, published sparse-grid point counts,
polynomial exactness against closed-form moments of the uniform law, the
Gauss-Legendre remainder bound for exp, and closed-form gPC coefficients.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

from conftest import golden


def _mono_moment(k):
    """E[x^k] for x ~ U(-1, 1)."""
    return 0.0 if k % 2 else 1.0 / (k + 1)


def test_gauss_legendre_matches_abramowitz_stegun(O):
    table = {}
    for n, x, w in golden("gauss_legendre_as.txt"):
        table.setdefault(int(n), []).append((float(x), float(w)))
    for n, rows in table.items():
        Z, a = O.quadrature(0, 1, n, [-1.0], [1.0])
        x = Z[:, 0]
        assert np.all(np.diff(x) > 0)
        for xt, wt in rows:
            k = int(np.argmin(np.abs(x - xt)))
            assert abs(x[k] - xt) < 1e-15
            assert abs(2.0 * a[k] - wt) < 1e-15
            k2 = int(np.argmin(np.abs(x + xt)))   # mirrored node, same weight
            assert x[k2] == -x[k] and a[k2] == a[k]


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_gauss_legendre_exactness(O, n):
    Z, a = O.quadrature(0, 1, n, [-1.0], [1.0])
    x = Z[:, 0]
    for k in range(2 * n):
        assert abs(a @ x ** k - _mono_moment(k)) < 1e-15
    assert abs(a @ x ** (2 * n) - _mono_moment(2 * n)) > 1e-6


def test_clenshaw_curtis_rational_weights(O):
    want = {}
    for m, k, num, den in golden("clenshaw_curtis_rational.txt"):
        want.setdefault(int(m), {})[int(k)] = Fraction(int(num), int(den))
    level = {3: 2, 5: 3}
    for m, wk in want.items():
        Z, a = O.quadrature(1, 1, level[m], [-1.0], [1.0])
        assert len(a) == m
        for k, fr in wk.items():
            assert abs(2.0 * a[k] - float(fr)) < 4e-16
            assert abs(Z[k, 0] + math.cos(k * math.pi / (m - 1))) < 1e-15


@pytest.mark.parametrize("level", [1, 2, 3, 4, 5])
def test_clenshaw_curtis_exactness(O, level):
    Z, a = O.quadrature(1, 1, level, [-1.0], [1.0])
    x = Z[:, 0]
    m = len(x)
    deg = m - 1 if m % 2 == 0 else m
    for k in range(deg + 1):
        assert abs(a @ x ** k - _mono_moment(k)) < 1e-14


def test_smolyak_point_counts(O):
    for d, L, cnt in golden("smolyak_cc_counts.txt"):
        d, L, cnt = int(d), int(L), int(cnt)
        Z, a = O.quadrature(1, d, L, [-1.0] * d, [1.0] * d)
        assert len(a) == cnt
        assert abs(a.sum() - 1.0) < 1e-14
        assert len({tuple(z) for z in Z}) == cnt


def _largest_exact_total_degree(Z, a, d, maxdeg=14):
    best = -1
    for D in range(maxdeg + 1):
        ok = True
        for alpha in itertools.product(range(D + 1), repeat=d):
            if sum(alpha) != D:
                continue
            q = a @ np.prod([Z[:, t] ** alpha[t] for t in range(d)], axis=0)
            exact = np.prod([_mono_moment(k) for k in alpha])
            if abs(q - exact) > 1e-13:
                ok = False
                break
        if not ok:
            break
        best = D
    return best


@pytest.mark.parametrize("d,L", [(2, 2), (2, 3), (2, 4), (3, 2), (3, 3), (3, 4)])
def test_smolyak_polynomial_exactness(O, d, L):
    Z, a = O.quadrature(1, d, L, [-1.0] * d, [1.0] * d)
    D = _largest_exact_total_degree(Z, a, d)
    # Novak & Ritter: level L integrates total degree 2L - 1 exactly
    assert D >= 2 * L - 1


def test_gauss_legendre_exp_within_remainder_bound(O):
    """E[exp(c xi)], xi ~ U(-h, h), against sinh(ch)/(ch); the n-point error is
    bounded by the Gauss-Legendre remainder (b-a)^(2n+1)(n!)^4 / ((2n+1)((2n)!)^3)
    max|f^(2n)|, divided by b - a for the probability measure."""
    for n in (2, 3, 4, 5):
        for c, h in ((3.0, 0.1), (2.0, 0.5), (1.0, 1.0)):
            Z, a = O.quadrature(0, 1, n, [-h], [h])
            q = a @ np.exp(c * Z[:, 0])
            exact = math.sinh(c * h) / (c * h)
            L = 2 * h
            bound = (L ** (2 * n + 1) * math.factorial(n) ** 4
                     / ((2 * n + 1) * math.factorial(2 * n) ** 3)
                     * c ** (2 * n) * math.exp(c * h)) / L
            assert abs(q - exact) <= bound + 1e-15


def test_smolyak_exp_product(O):
    """E[exp(c1 x1 + c2 x2 + c3 x3)] for independent uniforms is a product of
    sinh(c h)/(c h); the sparse grid converges to it spectrally."""
    lo = np.array([-0.15, 0.15, -10.0])
    hi = np.array([0.15, 0.35, 10.0])
    c = np.array([2.0, 1.5, 0.02])
    mid, half = (lo + hi) / 2, (hi - lo) / 2
    exact = np.prod(np.exp(c * mid) * np.sinh(c * half) / (c * half))
    errs = []
    for L in (2, 3, 4, 5):
        Z, a = O.quadrature(1, 3, L, lo, hi)
        errs.append(abs(a @ np.exp(Z @ c) - exact) / exact)
    assert errs[-1] < 1e-9
    assert errs[2] < errs[0]


def test_two_pass_moments_closed_form(O):
    """Eq. quad_moments on Q(xi) = 1 + 2 xi + 3 xi^2 with a rule exact to
    degree >= 4: E and Var match the moments of U(-1, 1)."""
    Z, a = O.quadrature(0, 1, 3, [-1.0], [1.0])
    x = Z[:, 0]
    Qv = np.ascontiguousarray(np.stack([1 + 2 * x + 3 * x ** 2, 0 * x + 7.0, x], 1))  # 3 "cells"
    mean, std, ncl = O.moments_two_pass(a, Qv)
    e = 1 + 3 * (1 / 3)
    # E[Q^2] = E[1 + 4x + 10x^2 + 12x^3 + 9x^4] = 1 + 10/3 + 9/5
    var = 1 + 10 / 3 + 9 / 5 - e * e
    assert abs(mean[0] - e) < 1e-15 and abs(std[0] - math.sqrt(var)) < 1e-15
    assert mean[1] == 7.0 and std[1] == 0.0
    assert abs(mean[2]) < 1e-16 and abs(std[2] - math.sqrt(1 / 3)) < 1e-15
    assert ncl == 0


def test_negative_weight_variance_is_clamped(O):
    a = np.array([1.5, -0.5])
    Qv = np.array([[0.0], [1.0]])      # E = -0.5, sum a (Q - E)^2 = 1.5*.25 - .5*2.25 < 0
    mean, std, ncl = O.moments_two_pass(a, Qv)
    assert mean[0] == -0.5 and std[0] == 0.0 and ncl == 1


def test_profiles_band(O):
    rng = np.random.default_rng(4)
    nx, ny, nz, nq = 5, 4, 6, 7
    Qv = rng.random((nq, nx * ny * nz))
    Z, a = O.quadrature(0, 1, 5, [-1.0], [1.0])
    a = np.concatenate([a, [0.0, 0.0]])
    xy = np.array([[1, 2], [4, 0]], np.int32)
    prof, pn = O.profiles(a, Qv, nx, ny, nz, xy)
    for p, (x, y) in enumerate(xy):
        for z in range(nz):
            v = Qv[:, x + nx * (y + ny * z)]
            assert np.array_equal(pn[p, :, z], v)
            e = a @ v
            s = math.sqrt(a @ (v - e) ** 2)
            assert abs(prof[p, z, 0] - e) < 1e-15 and abs(prof[p, z, 1] - s) < 1e-15
            assert abs(prof[p, z, 2] - (e - 1.959963984540054 * s)) < 1e-15
            assert abs(prof[p, z, 3] - (e + 1.959963984540054 * s)) < 1e-15


def test_profiles_band_factor_is_the_normal_quantile(O):
    """The 95% band half-width is Phi^-1(0.975) std: the factor the oracle
    applies, recovered from its output, equals the standard normal quantile
    computed here independently (statistics.NormalDist)."""
    from statistics import NormalDist
    z975 = NormalDist().inv_cdf(0.975)
    a = np.array([0.5, 0.5])
    Qv = np.array([[1.0], [3.0]])          # mean 2, std 1 exactly
    prof, _ = O.profiles(a, Qv, 1, 1, 1, np.array([[0, 0]], np.int32))
    assert prof[0, 0, 0] == 2.0 and prof[0, 0, 1] == 1.0
    assert abs((prof[0, 0, 3] - prof[0, 0, 0]) - z975) < 1e-12
    assert abs((prof[0, 0, 0] - prof[0, 0, 2]) - z975) < 1e-12


def test_profiles_pick_the_probe_column(O):
    """Hand-worked field: Q_0(x, y, z) = x + 10 y + 100 z, Q_1 = Q_0 + 4 with
    weights (1/4, 3/4), so at every cell mean = Q_0 + 3 and
    var = (1/4) 9 + (3/4) 1 = 3.  The profile of column (x, y) = (2, 1) on a
    3 x 2 x 4 grid is then mean 2 + 10 + 3 + 100 z = 15 + 100 z and std
    sqrt(3) in every layer; a transposed index (x <-> y) or a wrong layer
    stride would give other numbers."""
    nx, ny, nz = 3, 2, 4
    x, y, z = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    q0 = np.zeros(nx * ny * nz)
    q0[(x + nx * (y + ny * z)).ravel()] = (x + 10 * y + 100 * z).ravel()
    Qv = np.stack([q0, q0 + 4.0])
    a = np.array([0.25, 0.75])
    prof, pn = O.profiles(a, Qv, nx, ny, nz, np.array([[2, 1]], np.int32))
    for k in range(nz):
        assert prof[0, k, 0] == 15.0 + 100.0 * k
        assert abs(prof[0, k, 1] - math.sqrt(3.0)) < 1e-14
        assert pn[0, 0, k] == 12.0 + 100.0 * k and pn[0, 1, k] == 16.0 + 100.0 * k


def test_node_inflow_params_maps_inputs_by_kind(O):
    """A node's coordinates replace the speed error, exponent and angle by
    input kind, in the order the configuration lists the inputs; the others
    keep the nominal values."""
    Zj = np.array([0.07, 0.31, -4.0])
    kinds = [O.IN_SPEED_REL, O.IN_ALPHA, O.IN_ANGLE_DEG]
    assert O.node_inflow_params(Zj, kinds, 0.05, 0.25, 10.0) == (0.07, 0.31, -4.0)
    assert O.node_inflow_params(Zj, kinds[::-1], 0.05, 0.25, 10.0) == (-4.0, 0.31, 0.07)
    assert O.node_inflow_params(Zj[:1], [O.IN_ALPHA], 0.05, 0.25, 10.0) == (0.0, 0.07, 10.0)
    assert O.node_inflow_params(Zj[:0], [], 0.05, 0.25, 10.0) == (0.0, 0.25, 10.0)


def test_gpc_closed_form_coefficients_1d(O):
    """s^2 = (1/3) Phi_0 + 2/(3 sqrt 5) Phi_2 for orthonormal Legendre Phi."""
    lo, hi = [-0.1], [0.1]
    Z, a = O.quadrature(0, 1, 5, lo, hi)
    s = O.legendre_s(Z, lo, hi)
    phi = O.gpc_basis(1, 4, s)
    Qv = np.ascontiguousarray((s[:, 0] ** 2)[:, None])
    coef = O.gpc_project(a, Qv, phi)[:, 0]
    want = [1 / 3, 0.0, 2 / (3 * math.sqrt(5)), 0.0, 0.0]
    assert np.allclose(coef, want, atol=1e-15)
    # mean = coef_0 and Var = sum_{alpha>0} coef^2 = E[s^4] - E[s^2]^2 = 4/45
    assert abs((coef[1:] ** 2).sum() - 4 / 45) < 1e-15


def test_gpc_closed_form_coefficients_2d_sparse(O):
    """Q = s1 s2 + s1^2 on the level-3 Smolyak grid (exact to total degree 5):
    graded basis order (0,0),(1,0),(0,1),(2,0),(1,1),(0,2)."""
    lo, hi = [-0.15, 0.15], [0.15, 0.35]
    Z, a = O.quadrature(1, 2, 3, lo, hi)
    s = O.legendre_s(Z, lo, hi)
    phi = O.gpc_basis(2, 2, s)
    assert phi.shape == (13, 6)
    Qv = np.ascontiguousarray((s[:, 0] * s[:, 1] + s[:, 0] ** 2)[:, None])
    coef = O.gpc_project(a, Qv, phi)[:, 0]
    want = [1 / 3, 0, 0, 2 / (3 * math.sqrt(5)), 1 / 3, 0]
    assert np.allclose(coef, want, atol=1e-14)


def test_gpc_mean_variance_of_exp(O):
    """gPC mean and variance of Q = exp(c xi), xi ~ U(-h, h), against
    sinh(ch)/(ch) and sinh(2ch)/(2ch) - mean^2."""
    c, h = 3.0, 0.15
    Z, a = O.quadrature(0, 1, 5, [-h], [h])
    s = O.legendre_s(Z, [-h], [h])
    phi = O.gpc_basis(1, 4, s)
    Qv = np.ascontiguousarray(np.exp(c * Z))
    coef = O.gpc_project(a, Qv, phi)[:, 0]
    mean = math.sinh(c * h) / (c * h)
    var = math.sinh(2 * c * h) / (2 * c * h) - mean ** 2
    assert abs(coef[0] - mean) < 1e-12
    assert abs((coef[1:] ** 2).sum() - var) / var < 1e-6
