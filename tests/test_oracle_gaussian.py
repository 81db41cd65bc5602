"""Pins of the oracle's Gaussian input model (Sec. 2.1 Eq. mult_noise, Sec.
2.4 steps 2-3, Sec. 3): the tensor Gauss-Hermite rule, the orthonormal
probabilists' Hermite gPC basis and the logarithmic wind profile.

The rule is pinned by the moments of the normal distribution (an n-point
Gauss rule integrates every polynomial of degree <= 2n - 1 exactly, which
fixes its n nodes and n weights) and by numpy's hermegauss; the basis by its
orthonormality and the closed-form Hermite coefficients of x^2 and exp(a x);
the profile by its value at the reference height and the log-law ratios.
"""
import math

import numpy as np
import pytest
from numpy.polynomial import hermite_e as HE

GH = 2


def normal_moment(m):
    """E[x^m] for x ~ N(0, 1): (m - 1)!! for even m, 0 for odd m."""
    if m % 2:
        return 0.0
    return float(np.prod(np.arange(m - 1, 0, -2))) if m > 0 else 1.0


@pytest.mark.parametrize("n", list(range(1, 13)) + [20, 30, 40])
def test_gauss_hermite_matches_numpy(O, n):
    Z, w = O.quadrature(GH, 1, n, [0.0], [1.0])
    x, wr = HE.hermegauss(n)
    wr = wr / math.sqrt(2.0 * math.pi)
    assert np.max(np.abs(Z[:, 0] - x)) < 1e-13
    assert np.max(np.abs(w - wr) / wr) < 1e-12


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 11])
def test_gauss_hermite_exact_to_degree_2n_minus_1(O, n):
    Z, w = O.quadrature(GH, 1, n, [0.0], [1.0])
    x = Z[:, 0]
    for m in range(2 * n):
        got = float(np.sum(w * x ** m))
        want = normal_moment(m)
        scale = float(np.sum(w * np.abs(x) ** m))  # size of the terms summed
        assert abs(got - want) <= 1e-13 * max(1.0, scale), (n, m, got, want)
    # and not beyond: degree 2n differs from the normal moment
    assert abs(float(np.sum(w * x ** (2 * n))) - normal_moment(2 * n)) > 1e-6


def test_tensor_rule_normal_inputs(O):
    """11 x 11 rule on (zeta_1 - 1, zeta_2) ~ N(0, 0.1^2) x N(0, 6^2): 121
    nodes in lexicographic order, means, variances and covariance exact."""
    Z, w = O.quadrature(GH, 2, 11, [0.0, 0.0], [0.1, 6.0])
    assert Z.shape == (121, 2)
    assert abs(w.sum() - 1.0) < 1e-14
    assert np.all(np.diff(Z[::11, 0]) > 0) and np.all(np.diff(Z[:11, 1]) > 0)
    assert abs(w @ Z[:, 0]) < 1e-16 and abs(w @ Z[:, 1]) < 1e-13
    assert abs(w @ Z[:, 0] ** 2 - 0.01) < 1e-15 and abs(w @ Z[:, 1] ** 2 - 36.0) < 1e-12
    assert abs(w @ (Z[:, 0] * Z[:, 1])) < 1e-15
    assert abs(w @ (Z[:, 0] ** 2 * Z[:, 1] ** 2) - 0.36) < 1e-12
    Z2, w2 = O.quadrature(GH, 1, 5, [1.0], [0.1])
    assert abs(w2 @ Z2[:, 0] - 1.0) < 1e-15


def test_hermite_basis_orthonormal(O):
    Z, w = O.quadrature(GH, 2, 8, [0.0, 0.0], [1.0, 1.0])
    phi = O.gpc_basis_family(2, 4, O.HERMITE, Z)
    G = phi.T @ (w[:, None] * phi)
    assert np.max(np.abs(G - np.eye(G.shape[0]))) < 1e-12


def test_hermite_coefficients_closed_forms(O):
    """x^2 = He_0 + sqrt(2) (He_2 / sqrt(2)); exp(a x) has coefficients
    a^n exp(a^2 / 2) / sqrt(n!) in the orthonormal basis."""
    Z, w = O.quadrature(GH, 1, 30, [0.0], [1.0])
    x = Z[:, 0]
    phi = O.gpc_basis_family(1, 6, O.HERMITE, Z)
    c = O.gpc_project(w, (x ** 2)[:, None], phi)[:, 0]
    np.testing.assert_allclose(c, [1.0, 0.0, math.sqrt(2.0), 0.0, 0.0, 0.0, 0.0], atol=1e-13)
    a = 0.7
    c = O.gpc_project(w, np.exp(a * x)[:, None], phi)[:, 0]
    want = [a ** n * math.exp(a * a / 2) / math.sqrt(math.factorial(n)) for n in range(7)]
    np.testing.assert_allclose(c, want, rtol=1e-12)
    # two inputs, graded order (1, s1, s2, s1^2, s1 s2, s2^2): Q = x1 x2
    Z2, w2 = O.quadrature(GH, 2, 6, [0.0, 0.0], [1.0, 1.0])
    phi2 = O.gpc_basis_family(2, 2, O.HERMITE, Z2)
    c2 = O.gpc_project(w2, (Z2[:, 0] * Z2[:, 1])[:, None], phi2)[:, 0]
    np.testing.assert_allclose(c2, [0, 0, 0, 0, 1, 0], atol=1e-13)


def test_log_profile(O):
    """Sec. 3: u_ref (1 + xi) ln((h + z0)/z0) / ln((H + z0)/z0) at h = k + 1/2.
    With H at the top cell centre the top value is u_ref (1 + xi); velocity
    differences between heights follow the log law; a huge roughness length
    turns the profile linear; the angle rotates the horizontal direction."""
    nz, z0 = 8, 0.1
    H = nz - 0.5
    u = O.inflow_log(nz, 0.05, 0.1, z0, H, 0.0)
    assert abs(u[-1, 0] - 0.055) < 1e-15
    assert np.all(u[:, 1:] == 0) and np.all(np.diff(u[:, 0]) > 0)
    h = np.arange(nz) + 0.5
    r = (u[5, 0] - u[3, 0]) / (u[3, 0] - u[1, 0])
    assert abs(r - math.log((h[5] + z0) / (h[3] + z0)) / math.log((h[3] + z0) / (h[1] + z0))) < 1e-12
    ul = O.inflow_log(nz, 0.05, 0.0, 1e7, H, 0.0)
    np.testing.assert_allclose(ul[:, 0] / ul[-1, 0], h / H, rtol=1e-5)
    ur = O.inflow_log(nz, 0.05, 0.0, z0, H, 30.0)
    np.testing.assert_allclose(ur[:, 0], u[:, 0] / 1.1 * math.cos(math.pi / 6), rtol=1e-14)
    np.testing.assert_allclose(ur[:, 1], u[:, 0] / 1.1 * 0.5, rtol=1e-14)
    with pytest.raises(ValueError):
        O.inflow_log(nz, 0.05, 0.0, 0.0, H, 0.0)
