"""Variable-density elliptic operators (oracle; test infrastructure only).

Pressure (Eq. VDINSE.Lrho, discrete form Eq. VDINSE.Lrho.num):

    L~_rho phi = sum_j D_j ( rho^-1 * D_j phi )

Viscous (Eq. VDINSE.zeta and the Crank--Nicolson predictor Eq. VDINSE.num.momentum.proj,
whose 1D Sc=1 form is Eq. VDINSE.Vrho):

    V~_rho u = u - (dt/2) zeta(rho, u)
             = u - a rho^-1 [ Lap u + Sc^-1 ( (u.grad) grad rho + (grad rho . grad) u ) ],

with a = dt / (2 Re) and, component by component,
    [(u.grad) grad rho]_i = sum_j u_j D_j D_i rho,   [(grad rho . grad) u]_i = sum_j (D_j rho)(D_j u_i).
The derivatives of rho are spectral derivatives of the grid density (reading: the paper
does not say how they are formed).  Vector fields are numpy arrays of shape (d, *grid.shape).
"""

from __future__ import annotations

import numpy as np

from .spectral import Grid, deriv, lap, precond_pressure, precond_velocity


def apply_pressure(rho: np.ndarray, phi: np.ndarray, grid: Grid) -> np.ndarray:
    """L~_rho phi = sum_j D_j(rho^-1 D_j phi)."""
    out = np.zeros(grid.shape)
    for j in range(grid.ndim):
        out = out + deriv(deriv(phi, grid, j) / rho, grid, j)
    return out


class RhoDerivs:
    """Spectral first and second derivatives of the density: D_j rho and D_i D_j rho."""

    def __init__(self, rho: np.ndarray, grid: Grid):
        d = grid.ndim
        self.rho = rho
        self.g = [deriv(rho, grid, j) for j in range(d)]
        self.h = [[deriv(self.g[i], grid, j) for j in range(d)] for i in range(d)]


def zeta_bracket(u: np.ndarray, rd: RhoDerivs, grid: Grid, inv_sc: float) -> np.ndarray:
    """Lap u + Sc^-1((u.grad) grad rho + (grad rho.grad) u), per component."""
    d = grid.ndim
    out = np.empty_like(u)
    for i in range(d):
        acc = lap(u[i], grid)
        t = np.zeros(grid.shape)
        for j in range(d):
            t = t + u[j] * rd.h[j][i] + rd.g[j] * deriv(u[i], grid, j)
        out[i] = acc + inv_sc * t
    return out


def apply_velocity(rho: np.ndarray, u: np.ndarray, grid: Grid, a: float, inv_sc: float,
                   rd: RhoDerivs | None = None) -> np.ndarray:
    """V~_rho u = u - a rho^-1 [Lap u + Sc^-1((u.grad)grad rho + (grad rho.grad)u)]."""
    if rd is None:
        rd = RhoDerivs(rho, grid)
    return u - a * zeta_bracket(u, rd, grid, inv_sc) / rho


def precond_velocity_vec(g: np.ndarray, grid: Grid, a: float) -> np.ndarray:
    """Block-diagonal (I - a Lap)^-1 applied to each component (Eq. VDINSE.V)."""
    return np.stack([precond_velocity(g[i], grid, a) for i in range(g.shape[0])])


def pressure_system(rho: np.ndarray, grid: Grid):
    """(A, M) callables for the pressure equation in physical space."""
    return (lambda v: apply_pressure(rho, v, grid)), (lambda v: precond_pressure(v, grid))


def velocity_system(rho: np.ndarray, grid: Grid, a: float, inv_sc: float):
    """(A, M) callables for the coupled velocity system in physical space."""
    rd = RhoDerivs(rho, grid)
    return ((lambda v: apply_velocity(rho, v, grid, a, inv_sc, rd)),
            (lambda v: precond_velocity_vec(v, grid, a)))
