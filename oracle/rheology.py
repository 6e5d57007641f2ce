"""Strain rate and Papanastasiou-regularised Herschel-Bulkley viscosity.

Paper: Sec. II (Eq. 1 scaled Frobenius norm, the gradient/strain-rate
definitions), Sec. II B (Eqs. 9-10, Herschel-Bulkley), Sec. III B (Eqs. 21-24,
Papanastasiou regularisation).

Parameters follow the paper with mu -> K and 1/epsilon -> m:

    eta(g) = (2^(n-1) K g^n + tau_y / 2) * F(g),    F(g) = (1 - exp(-m g)) / g,

with g = |gamma_dot| = sqrt(1/2 tr(D D^T)) and F(0) = m (Eq. 22), so that
eta(0) = tau_y m / 2 (Eq. 24).  F is evaluated as -expm1(-m g)/g; for
x = m g < 1e-3 the Taylor series m (1 - x/2 + x^2/6 - x^3/24) of (1-e^-x)/x is
used (truncation below 1e-14 relative).

``reg_power=False`` regularises only the yield term,
eta = 2^(n-1) K g^(n-1) + (tau_y/2) F(g); with tau_y = 0, n = 1 this is the exact
Newtonian law (Eq. 3) used as a fixed point in the tests.
"""

import numpy as np

from .grid import pad_cells, velocity_wall_vals

SERIES_X = 1.0e-3


def regularised_inverse(g, m):
    """F(g) = (1 - e^{-m g}) / g, bounded with F(0) = m (Eqs. 21-22)."""
    g = np.asarray(g, dtype=np.float64)
    x = m * g
    small = x < SERIES_X
    with np.errstate(divide="ignore", invalid="ignore"):
        direct = -np.expm1(-x) / g
    series = m * (1.0 - x / 2.0 + x * x / 6.0 - x * x * x / 24.0)
    return np.where(small, series, direct)


def viscosity(g, K, n, tau_y, m, reg_power=True):
    """Apparent viscosity eta(|gamma_dot|) of Eq. 23 (Sec. III B)."""
    g = np.asarray(g, dtype=np.float64)
    F = regularised_inverse(g, m)
    if reg_power:
        return (2.0 ** (n - 1.0) * K * np.power(g, n) + 0.5 * tau_y) * F
    with np.errstate(divide="ignore"):
        return 2.0 ** (n - 1.0) * K * np.power(g, n - 1.0) + 0.5 * tau_y * F


def velocity_gradient(u, grid):
    """(grad u)_{ij} = d u_j / d x_i by central differences over two cells,
    with wall ghosts (odd reflection about the wall velocity) or periodic wrap.
    Returns ``G[i][j]`` arrays of cell shape."""
    d, h = grid.d, grid.h
    G = [[None] * d for _ in range(d)]
    for j in range(d):
        up = pad_cells(u[j], 1, grid, "dirichlet", velocity_wall_vals(grid, j))
        for i in range(d):
            lo = [slice(1, -1)] * d
            hi = [slice(1, -1)] * d
            lo[i] = slice(0, -2)
            hi[i] = slice(2, None)
            G[i][j] = (up[tuple(hi)] - up[tuple(lo)]) / (2.0 * h)
    return G


def strain_rate_norm(u, grid):
    """|gamma_dot| with gamma_dot = 1/2 (grad u + grad u^T) (Sec. II) and the
    scaled norm |A| = sqrt(1/2 tr(A A^T)) (Eq. 1)."""
    G = velocity_gradient(u, grid)
    d = grid.d
    s = np.zeros(grid.n)
    for i in range(d):
        for j in range(d):
            Dij = 0.5 * (G[i][j] + G[j][i])
            s += Dij * Dij
    return np.sqrt(0.5 * s)


def cell_viscosity(u, grid, rheo):
    """Cell-centred eta^m from u^m (first stage of the step, Sec. III A)."""
    g = strain_rate_norm(u, grid)
    return viscosity(g, rheo.K, rheo.n, rheo.tau_y, rheo.m, rheo.reg_power)
