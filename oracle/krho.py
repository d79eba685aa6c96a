"""The modified-Helmholtz form of the pressure equation (oracle; test infrastructure only).

Sec. 4.2 ("Pressure equation", Eq. VDINSE.Krho): with Phi = phi / sqrt(rho) the pressure
equation div(rho^-1 grad phi) = f becomes

    K_rho Phi = Lap Phi + ( Lap rho / (2 rho) - (3/4) |grad rho|^2 / rho^2 ) Phi = sqrt(rho) f,

preconditioned by the inverse Laplacian (the inverse of K_rho at constant density), with a
pseudo-inverse that removes the first spectral coefficient, so that Phi is zero-mean
(text before Table 2).  K_rho costs two transforms per apply instead of the 2d of L_rho.

Readings taken here (the paper discretises the periodic case without these details):

* The Laplacian of K_rho keeps the Nyquist wavenumber (symbol -|k|^2 with every k_j the full
  2 pi m / L_j): its null space is then the constants alone, and its pseudo-inverse removes
  exactly the first coefficient, as the paper states.  (The first-derivative operators of
  L_rho zero the Nyquist wavenumber; K_rho has no first derivative of Phi.)
* The coefficient is formed as c = -Lap(w) / w with w = rho^-1/2.  The identity
  Lap(rho^-1/2) = -rho^-3/2 Lap rho / 2 + 3 rho^-5/2 |grad rho|^2 / 4 shows that this is the
  paper's coefficient; formed this way, the discrete operator K~ = Lap + diag(c) keeps the
  continuous null vector exactly: K~ w = 0.  K~ is symmetric, so its range is the orthogonal
  complement of w; the right-hand side sqrt(rho) f is projected onto it (for zero-mean f,
  <sqrt(rho) f, w> = sum f = 0 already in the continuum).
* The solution is the zero-mean Phi; phi = sqrt(rho) Phi then solves the pressure equation
  up to the discretisation difference between K~ and L~ (spectrally small for smooth rho).
"""

from __future__ import annotations

import numpy as np

from .spectral import Grid, deriv, fwd, inv, wavenumber_1d
from . import solvers


def kfull(grid: Grid, j: int) -> np.ndarray:
    """k_j = 2 pi m / L_j (Nyquist kept) broadcast to the full-spectrum shape."""
    k = wavenumber_1d(grid.n[j], grid.L[j], zero_nyquist=False)
    sh = [1] * grid.ndim
    sh[grid.np_axis(j)] = grid.n[j]
    return k.reshape(sh)


def ksq_full(grid: Grid) -> np.ndarray:
    out = np.zeros(grid.shape)
    for j in range(grid.ndim):
        out = out + kfull(grid, j) ** 2
    return out


def lap_full(phi: np.ndarray, grid: Grid) -> np.ndarray:
    """Laplacian with symbol -|k|^2 (Nyquist kept)."""
    return np.real(inv(-ksq_full(grid) * fwd(phi)))


def precond_krho(g: np.ndarray, grid: Grid) -> np.ndarray:
    """Pseudo-inverse of lap_full: multiply by -1/|k|^2, 0 for the mean (k = 0) only."""
    k2 = ksq_full(grid)
    mask = k2 == 0.0
    sym = np.where(mask, 0.0, -1.0 / np.where(mask, 1.0, k2))
    return np.real(inv(sym * fwd(g)))


def null_vector(rho: np.ndarray) -> np.ndarray:
    """w = rho^-1/2: K_rho w = 0 (the image of the constant pressure)."""
    return 1.0 / np.sqrt(rho)


def coeff(rho: np.ndarray, grid: Grid) -> np.ndarray:
    """c = -Lap(w) / w, w = rho^-1/2 (the coefficient of Eq. VDINSE.Krho)."""
    w = null_vector(rho)
    return -lap_full(w, grid) / w


def coeff_paper(rho: np.ndarray, grid: Grid) -> np.ndarray:
    """The coefficient as printed in Eq. VDINSE.Krho: Lap rho / (2 rho) - 3 |grad rho|^2 / (4 rho^2)."""
    g2 = np.zeros(grid.shape)
    for j in range(grid.ndim):
        g2 = g2 + deriv(rho, grid, j) ** 2
    return lap_full(rho, grid) / (2.0 * rho) - 0.75 * g2 / rho ** 2


def apply_krho(rho: np.ndarray, Phi: np.ndarray, grid: Grid, c: np.ndarray | None = None) -> np.ndarray:
    """K~ Phi = Lap Phi + c Phi."""
    if c is None:
        c = coeff(rho, grid)
    return lap_full(Phi, grid) + c * Phi


def project_rhs(g: np.ndarray, rho: np.ndarray) -> np.ndarray:
    """Remove the component of g along w = rho^-1/2 (the range of K~ is w-orthogonal)."""
    w = null_vector(rho)
    return g - (np.vdot(w, g).real / np.vdot(w, w).real) * w


def krho_system(rho: np.ndarray, grid: Grid):
    """(A, M) callables of the K_rho equation in physical space."""
    c = coeff(rho, grid)
    return (lambda v: apply_krho(rho, v, grid, c)), (lambda v: precond_krho(v, grid))


def solve_krho(rho: np.ndarray, f: np.ndarray, grid: Grid, kind: str = "gmres", tol: float = 1e-10,
               maxit: int = 500, restart: int = 30):
    """Solve K~ Phi = P(sqrt(rho) f) for zero-mean Phi; returns (result, phi = sqrt(rho) Phi)."""
    A, M = krho_system(rho, grid)
    b = project_rhs(np.sqrt(rho) * f, rho)
    res = solvers.solve(kind, A, M, b, tol=tol, maxit=maxit, restart=restart)
    return res, np.sqrt(rho) * res.x
