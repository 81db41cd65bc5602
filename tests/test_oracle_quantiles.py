"""Pins of the oracle's confidence bounds from the gPC surrogate (Sec. 2.4
step 7: confidence intervals from the expansion coefficients; Sec. 4 profile
bands): empirical quantiles of the surrogate evaluated at given input
samples, the k-th smallest value with k = ceil(q M).

Checked against order statistics worked out in closed form for surrogates
whose distribution is known: linear in a uniform input (rising and falling),
the square of a uniform input, and linear in a normal input, where the band
must approach the Gaussian mean +- 1.96 std."""
import math

import numpy as np
import pytest

Q = [0.025, 0.5, 0.975]


def midpoints(M):
    return -1.0 + (2.0 * np.arange(M) + 1.0) / M


@pytest.mark.parametrize("b", [0.7, -0.7])
def test_linear_uniform_surrogate(O, b):
    """Q(s) = a + b s with Legendre coefficients (a, b / sqrt 3) at the M
    midpoints s_m = -1 + (2m + 1)/M: the k-th smallest value is
    a + |b| (-1 + (2k - 1)/M) whatever the sign of b."""
    M, a = 4000, 0.3
    phi = O.gpc_basis_family(1, 1, O.LEGENDRE, midpoints(M))
    coef = np.array([[a], [b / math.sqrt(3.0)]])
    got = O.gpc_quantiles(coef, phi, Q)[:, 0]
    for qq, g in zip(Q, got):
        k = math.ceil(qq * M)
        assert abs(g - (a + abs(b) * (-1.0 + (2 * k - 1) / M))) < 1e-14


def test_square_of_uniform(O):
    """Q = s^2 has coefficients (1/3, 0, 2/(3 sqrt 5)); for s uniform on
    [-1, 1], P(s^2 <= t) = sqrt t, so the q-quantile is q^2 (the midpoint
    samples put it within 2/M)."""
    M = 6000
    phi = O.gpc_basis_family(1, 2, O.LEGENDRE, midpoints(M))
    coef = np.array([[1.0 / 3.0], [0.0], [2.0 / (3.0 * math.sqrt(5.0))]])
    got = O.gpc_quantiles(coef, phi, Q)[:, 0]
    for qq, g in zip(Q, got):
        assert abs(g - qq * qq) < 2.0 / M


def test_linear_normal_surrogate_gives_the_gaussian_band(O):
    """Q = m + s sd He_1(s) with s standard normal: mean m, std sd, and the
    2.5/97.5% quantiles m -+ 1.959964 sd (to sampling accuracy)."""
    rng = np.random.default_rng(17)
    M, m, sd = 200000, 0.04, 0.006
    s = rng.standard_normal(M)
    phi = O.gpc_basis_family(1, 1, O.HERMITE, s)
    coef = np.array([[m], [sd]])
    lo, med, hi = O.gpc_quantiles(coef, phi, Q)[:, 0]
    assert abs(lo - (m - O.Z95 * sd)) < 0.02 * sd
    assert abs(hi - (m + O.Z95 * sd)) < 0.02 * sd
    assert abs(med - m) < 0.01 * sd


def test_cells_are_independent_and_k_is_clamped(O):
    M = 10
    phi = O.gpc_basis_family(1, 1, O.LEGENDRE, midpoints(M))
    coef = np.array([[0.0, 1.0], [1.0, -2.0]])
    got = O.gpc_quantiles(coef, phi, [0.0, 1.0])
    vals = phi @ coef
    np.testing.assert_array_equal(got[0], vals.min(axis=0))    # q = 0 -> k = 1
    np.testing.assert_array_equal(got[1], vals.max(axis=0))    # q = 1 -> k = M
