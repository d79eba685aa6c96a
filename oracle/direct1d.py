"""Exact direct solve of the 1D periodic pressure equation (oracle; test infrastructure only).

The 1D form of Eq. VDINSE.Lrho is D(rho^-1 D p) = f with the Fourier derivative D
(Nyquist wavenumber zeroed).  It can be solved without iteration:

1. g = rho^-1 D p satisfies D g = f, so g = D+ f + c1 * 1 + c2 * s, where D+ is the
   pseudo-inverse of D (symbol 1/(i k~), 0 where k~ = 0) and {1, s_j = (-1)^j} span
   the null space of D;
2. D p = rho g must lie in the range of D (zero mean and zero Nyquist coefficient), which
   gives two linear equations for (c1, c2):
       sum rho (h + c1 + c2 s) = 0,   sum rho s (h + c1 + c2 s) = 0,   h = D+ f;
3. p = D+ (rho g) is the unique solution orthogonal to the null space.

It needs f in the range of the operator (zero mean, zero Nyquist coefficient) and is
exact up to rounding, so it pins every Krylov solution of the 1D problem.
"""

from __future__ import annotations

import numpy as np

from .spectral import Grid, fwd, inv, wavenumber_1d


def dplus(f: np.ndarray, grid: Grid) -> np.ndarray:
    """Pseudo-inverse of D: multiply by 1/(i k~) where k~ != 0, else 0."""
    k = wavenumber_1d(grid.n[0], grid.L[0])
    nz = k != 0.0
    sym = np.zeros_like(k, dtype=np.complex128)
    sym[nz] = 1.0 / (1j * k[nz])
    return np.real(inv(sym * fwd(f)))


def solve_pressure_1d(rho: np.ndarray, f: np.ndarray, grid: Grid) -> np.ndarray:
    if grid.ndim != 1:
        raise ValueError("1D only")
    n = grid.n[0]
    s = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    h = dplus(f, grid)
    m = np.array([[rho.sum(), (rho * s).sum()], [(rho * s).sum(), rho.sum()]])
    rhs = -np.array([(rho * h).sum(), (rho * s * h).sum()])
    c1, c2 = np.linalg.solve(m, rhs)
    g = h + c1 + c2 * s
    return dplus(rho * g, grid)
