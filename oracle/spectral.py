"""Periodic Fourier spectral calculus (oracle; test infrastructure only).

Discretisation (Sec. 3, "Fourier--Fourier--Fourier decomposition": constant-coefficient
elliptic problems are diagonal in Fourier space).  A field on a periodic grid of
``n = (n0, n1, n2)`` points (x fastest; numpy shape ``(n2, n1, n0)``) over a box
``L = (L0, L1, L2)`` is differentiated along axis j by

    D_j = F^-1 diag(i k~_j) F,

with k_j = 2 pi m / L_j for the integer frequency m in [-n/2, n/2) and k~_j equal to
k_j except at the Nyquist index m = -n/2, where it is 0.  Zeroing the Nyquist
wavenumber keeps D_j real and skew-symmetric for even n, so that the discrete pressure
operator sum_j D_j rho^-1 D_j is exactly symmetric (reading of the paper, which does
not discuss the Nyquist mode).  The discrete Laplacian used everywhere (viscous term,
mass diffusion, preconditioners) is sum_j D_j D_j, whose symbol is -|k~|^2.

Null space: D_j phi = 0 for all j exactly when phi only has Fourier modes with every
index in {0, n/2}; these 2^d "corner" modes are the null space of the pressure
operator, and the pseudo-inverse preconditioner maps them to 0 (the paper removes the
k=0 coefficient of the Laplacian through an SVD pseudo-inverse, Sec. 4.2, text before
Table 2; with the Nyquist wavenumber zeroed the corner modes join it).
"""

from __future__ import annotations

from dataclasses import dataclass
import numpy as np
import scipy.fft

# Threads of the library FFT (scipy.fft's ``workers``).  1 everywhere except where the oracle
# is timed as the CPU baseline on a many-core host; the transform computed is the same.
FFT_WORKERS = 1


@dataclass(frozen=True)
class Grid:
    """Periodic grid: ``n[j]`` points over length ``L[j]`` along axis j (j=0 is x)."""

    n: tuple
    L: tuple

    def __post_init__(self):
        if not (1 <= len(self.n) <= 3) or len(self.L) != len(self.n):
            raise ValueError("grid must be 1D, 2D or 3D with one length per axis")
        for m in self.n:
            if m < 2 or m % 2:
                raise ValueError("every axis length must be even and >= 2")

    @property
    def ndim(self) -> int:
        return len(self.n)

    @property
    def shape(self) -> tuple:
        """numpy shape, slowest axis first (z, y, x)."""
        return tuple(reversed(self.n))

    @property
    def size(self) -> int:
        return int(np.prod(self.n))

    def np_axis(self, j: int) -> int:
        """numpy axis of grid axis j (x = 0 is the last numpy axis)."""
        return self.ndim - 1 - j

    def coords(self):
        """Physical coordinates x_j = L_j * i / n_j as broadcastable arrays, axis order x, y, z."""
        out = []
        for j in range(self.ndim):
            c = self.L[j] * np.arange(self.n[j]) / self.n[j]
            sh = [1] * self.ndim
            sh[self.np_axis(j)] = self.n[j]
            out.append(c.reshape(sh))
        return out


def freq_index(n: int) -> np.ndarray:
    """Integer frequencies m in FFT order: 0, 1, ..., n/2-1, -n/2, ..., -1."""
    return np.concatenate([np.arange(0, n // 2), np.arange(-n // 2, 0)])


def wavenumber_1d(n: int, L: float, zero_nyquist: bool = True) -> np.ndarray:
    """k_m = 2 pi m / L in FFT order; the Nyquist entry (m = -n/2) is set to 0 if asked."""
    m = freq_index(n).astype(np.float64)
    k = 2.0 * np.pi * m / L
    if zero_nyquist:
        k[n // 2] = 0.0
    return k


def ktilde(grid: Grid, j: int) -> np.ndarray:
    """k~_j broadcast to the full-spectrum array shape."""
    k = wavenumber_1d(grid.n[j], grid.L[j])
    sh = [1] * grid.ndim
    sh[grid.np_axis(j)] = grid.n[j]
    return k.reshape(sh)


def ksq(grid: Grid) -> np.ndarray:
    """|k~|^2 on the full spectrum (symbol of -Laplacian)."""
    out = np.zeros(grid.shape)
    for j in range(grid.ndim):
        out = out + ktilde(grid, j) ** 2
    return out


def null_mask(grid: Grid) -> np.ndarray:
    """True on the 2^d corner modes where every k~_j vanishes (null space of D_j for all j)."""
    return ksq(grid) == 0.0


# ----------------------------------------------------------------------------------
# Transforms
# ----------------------------------------------------------------------------------

def fwd(phi: np.ndarray) -> np.ndarray:
    """Forward DFT over all axes, unnormalised: phi_hat(k) = sum_x phi(x) e^{-i k.x}.
    Library primitive (scipy.fft), pinned against dft_naive in the tests."""
    return scipy.fft.fftn(phi, workers=FFT_WORKERS)


def inv(phi_hat: np.ndarray) -> np.ndarray:
    """Inverse DFT over all axes (1/N normalised); returns the complex result."""
    return scipy.fft.ifftn(phi_hat, workers=FFT_WORKERS)


def dft_naive_1d(x: np.ndarray, inverse: bool = False) -> np.ndarray:
    """O(n^2) DFT of a 1D sequence written from the definition.

    Forward: X_m = sum_t x_t exp(-2 pi i m t / n);  inverse: x_t = (1/n) sum_m X_m exp(+2 pi i m t / n).
    The phase m*t is reduced modulo n in integers before the trigonometric evaluation so
    that the matrix entries are correctly rounded for every n.
    """
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[0]
    t = np.arange(n)
    phase = np.outer(t, t) % n
    sign = 1.0 if inverse else -1.0
    W = np.exp(sign * 2j * np.pi * phase / n)
    y = W @ x
    return y / n if inverse else y


def dft_naive(phi: np.ndarray, inverse: bool = False) -> np.ndarray:
    """Multi-dimensional DFT by applying the naive 1D DFT along every axis."""
    out = np.asarray(phi, dtype=np.complex128)
    for ax in range(out.ndim):
        out = np.apply_along_axis(dft_naive_1d, ax, out, inverse)
    return out


# ----------------------------------------------------------------------------------
# Differential operators (real fields in, real fields out)
# ----------------------------------------------------------------------------------

def deriv(phi: np.ndarray, grid: Grid, j: int) -> np.ndarray:
    """D_j phi = F^-1 (i k~_j F phi)."""
    return np.real(inv(1j * ktilde(grid, j) * fwd(phi)))


def grad(phi: np.ndarray, grid: Grid) -> list:
    return [deriv(phi, grid, j) for j in range(grid.ndim)]


def div(q: list, grid: Grid) -> np.ndarray:
    """sum_j D_j q_j."""
    out = np.zeros(grid.shape)
    for j in range(grid.ndim):
        out = out + deriv(q[j], grid, j)
    return out


def lap(phi: np.ndarray, grid: Grid) -> np.ndarray:
    """Discrete Laplacian sum_j D_j D_j phi (symbol -|k~|^2)."""
    return np.real(inv(-ksq(grid) * fwd(phi)))


def project_range(f: np.ndarray, grid: Grid) -> np.ndarray:
    """Pi f: remove the null-space (corner) modes so that L~ phi = Pi f is solvable."""
    fh = fwd(f)
    fh[null_mask(grid)] = 0.0
    return np.real(inv(fh))


def precond_pressure(g: np.ndarray, grid: Grid) -> np.ndarray:
    """M+ g = (sum_j D_j D_j)^+ g: multiply by -1/|k~|^2, 0 on the corner modes.

    The constant-density inverse used as preconditioner of the pressure equation
    (Sec. 4.2: the inverse Laplacian, i.e. the pressure operator with constant density;
    Table 2 text: pseudo-inverse with the first coefficient removed).  Unscaled: the
    three solvers are invariant to scaling the preconditioner by a constant.
    """
    k2 = ksq(grid)
    mask = k2 == 0.0
    sym = np.where(mask, 0.0, -1.0 / np.where(mask, 1.0, k2))
    return np.real(inv(sym * fwd(g)))


def precond_velocity(g: np.ndarray, grid: Grid, a: float) -> np.ndarray:
    """V^-1 g = (I - a sum_j D_j D_j)^-1 g: multiply by 1/(1 + a|k~|^2) (Eq. VDINSE.V)."""
    return np.real(inv(fwd(g) / (1.0 + a * ksq(grid))))
