"""Brute-force dense assembly on tiny grids (oracle; test infrastructure only).

The paper characterises its preconditioners by the condition number of the assembled
operators (computed by a singular value decomposition, Sec. 3.1; pressure operators in
Sec. 3.2), with and without left/right preconditioning.  This module assembles any of the
oracle's linear maps column by column (apply to unit vectors) and measures:

* the 2-norm condition number restricted to the range (singular values above a relative
  cut, so that the 2^d null-space directions of the pressure operator are excluded);
* symmetry and definiteness (needed by CG);
* the spectrum of the preconditioned operator M+ L~, which is bounded by
  [1/rho_max, 1/rho_min] on the range: the Rayleigh quotient
  v^T(-L~)v / v^T(-Lap)v = sum_j sum_x (D_j v)^2/rho / sum_j sum_x (D_j v)^2.
"""

from __future__ import annotations

import numpy as np


def assemble(apply, shape) -> np.ndarray:
    """Matrix of the linear map ``apply`` acting on arrays of ``shape`` (column = A e_i)."""
    n = int(np.prod(shape))
    A = np.empty((n, n))
    e = np.zeros(n)
    for i in range(n):
        e[:] = 0.0
        e[i] = 1.0
        A[:, i] = np.asarray(apply(e.reshape(shape))).ravel()
    return A


def cond_on_range(A: np.ndarray, rel_cut: float = 1e-9) -> float:
    """sigma_max / sigma_min over singular values above rel_cut * sigma_max."""
    s = np.linalg.svd(A, compute_uv=False)
    s = s[s > rel_cut * s[0]]
    return float(s[0] / s[-1])


def nullity(A: np.ndarray, rel_cut: float = 1e-9) -> int:
    s = np.linalg.svd(A, compute_uv=False)
    return int(np.sum(s <= rel_cut * s[0]))


def symmetry_defect(A: np.ndarray) -> float:
    return float(np.linalg.norm(A - A.T) / np.linalg.norm(A))


def eig_range(A: np.ndarray, rel_cut: float = 1e-9):
    """Real parts of the eigenvalues of A whose modulus exceeds rel_cut * max modulus."""
    w = np.linalg.eigvals(A)
    w = w[np.abs(w) > rel_cut * np.max(np.abs(w))]
    return w
