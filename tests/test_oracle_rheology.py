"""Pins for the oracle's strain rate and viscosity (Sec. II, Sec. III B).

Each check is fixed by the paper or by mathematics, not by re-typing the
oracle's formula: extended-precision evaluation, the limits of Eqs. 22/24, the
unregularised models of Eqs. 6, 8, 10, and exact central differences of linear
fields."""

import mpmath
import numpy as np
import pytest

from oracle.grid import Grid
from oracle.rheology import regularised_inverse, strain_rate_norm, viscosity

mpmath.mp.dps = 50


def _F_mp(g, m):
    g = mpmath.mpf(g)
    if g == 0:
        return mpmath.mpf(m)
    return (1 - mpmath.exp(-mpmath.mpf(m) * g)) / g


@pytest.mark.parametrize("m", [1.0, 400.0, 1e4, 1e5])
def test_regularised_inverse_matches_extended_precision(m):
    rng = np.random.default_rng(1)
    # both branches: x = m g across [1e-9, 1e3] plus the series threshold band
    x = np.concatenate([10.0 ** rng.uniform(-9, 3, 400), rng.uniform(0.5e-3, 2e-3, 100)])
    g = x / m
    F = regularised_inverse(g, m)
    ref = np.array([float(_F_mp(gi, m)) for gi in g])
    assert np.max(np.abs(F - ref) / ref) <= 1e-14


def test_zero_strain_limits():
    # Eq. 22: F -> 1/eps = m; Eq. 24: eta(0) = tau_0 / (2 eps) = tau_y m / 2
    for m in (400.0, 1e4):
        assert regularised_inverse(np.array([0.0]), m)[0] == m
        for n in (0.5, 1.0, 1.5):
            assert viscosity(np.array([0.0]), 0.7, n, 3.0, m)[0] == pytest.approx(1.5 * m, rel=1e-15)


@pytest.mark.parametrize("n", [0.3, 0.5, 1.0, 1.5, 2.0])
def test_large_strain_recovers_herschel_bulkley(n):
    # m g >> 1: the regularisation factor is 1 to double precision and Eq. 23
    # reduces to Eq. 10: eta = 2^(n-1) K g^(n-1) + tau_y / (2 g)
    K, tau, m = 0.37, 2.5, 1e4
    g = np.array([0.05, 0.3, 1.0, 7.0, 100.0])
    eta = viscosity(g, K, n, tau, m)
    hb = 2.0 ** (n - 1) * K * g ** (n - 1) + tau / (2 * g)
    np.testing.assert_allclose(eta, hb, rtol=1e-14)


def test_bingham_and_power_law_special_cases():
    g = np.array([0.1, 1.0, 10.0])
    m = 1e5
    # Eq. 8 (n = 1): eta = mu + tau_0 / (2 g)
    np.testing.assert_allclose(viscosity(g, 2.0, 1.0, 3.0, m), 2.0 + 3.0 / (2 * g), rtol=1e-14)
    # Eq. 6 (tau_0 = 0): eta = 2^(n-1) mu g^(n-1)
    np.testing.assert_allclose(viscosity(g, 2.0, 0.5, 0.0, m), 2.0 ** -0.5 * 2.0 * g ** -0.5, rtol=1e-14)


def test_newtonian_fixed_point_without_power_regularisation():
    # tau_y = 0, n = 1 with only the yield term regularised: eta = mu exactly (Eq. 3)
    g = np.array([0.0, 1e-12, 1e-3, 1.0, 1e3])
    assert np.all(viscosity(g, 0.8, 1.0, 0.0, 1e4, reg_power=False) == 0.8)


def test_paper_form_regularises_power_term_too():
    # Eq. 23 multiplies the whole bracket by (1 - e^{-g/eps}); at tau_y = 0, n = 1
    # this gives mu (1 - e^{-m g}), not mu
    g = np.array([1e-4, 1e-2])
    np.testing.assert_allclose(viscosity(g, 1.0, 1.0, 0.0, 1e2), -np.expm1(-1e2 * g), rtol=1e-14)


@pytest.mark.parametrize("d", [2, 3])
def test_strain_rate_norm_of_linear_field(d):
    # u_j = sum_i B_ij x_i has (grad u)_ij = du_j/dx_i = B_ij; central differences
    # are exact away from walls.  |gamma_dot| = sqrt(1/2 sum D_ij^2), D = (B + B^T)/2
    rng = np.random.default_rng(d)
    n = (6,) * d
    h = 0.25
    B = rng.normal(size=(d, d))
    g = Grid(n, h)
    X = np.meshgrid(*[(np.arange(s) + 0.5) * h for s in n], indexing="ij")
    u = [sum(B[i, j] * X[i] for i in range(d)) for j in range(d)]
    s = strain_rate_norm(u, g)
    D = 0.5 * (B + B.T)
    expect = np.sqrt(0.5 * np.sum(D * D))
    inner = tuple(slice(1, -1) for _ in range(d))
    np.testing.assert_allclose(s[inner], expect, rtol=1e-13)


def test_simple_shear_norm_is_half_the_shear_rate():
    # u_x = gs * y: the scaled norm of Eq. 1 gives |gamma_dot| = gs / 2
    n = (6, 6)
    h = 0.2
    g = Grid(n, h)
    X = np.meshgrid(*[(np.arange(s) + 0.5) * h for s in n], indexing="ij")
    u = [3.0 * X[1], np.zeros(n)]
    np.testing.assert_allclose(strain_rate_norm(u, g)[1:-1, 1:-1], 1.5, rtol=1e-14)
