"""Pins of the oracle's spectral calculus (CPU only).

* the library FFT used by the oracle equals the naive O(n^2) DFT written from the
  definition, and the naive DFT maps single modes to Kronecker spectra (closed form);
* D_j differentiates trigonometric polynomials exactly (closed forms, any box length);
* D_j is real skew-symmetric (dense brute force): this is what makes the pressure
  operator symmetric;
* the preconditioners invert the constant-density operators on their range.
"""

import math

import numpy as np
import pytest

from oracle import spectral as sp
from oracle.dense import assemble


@pytest.mark.parametrize("n", [2, 4, 6, 8, 10, 12, 16, 18, 20, 24, 30, 32])
def test_naive_dft_single_mode(n):
    t = np.arange(n)
    for m in range(n):
        x = np.exp(2j * math.pi * m * t / n)
        X = sp.dft_naive_1d(x)
        expect = np.zeros(n, complex)
        expect[m] = n
        assert np.max(np.abs(X - expect)) < 1e-12 * n
        back = sp.dft_naive_1d(X, inverse=True)
        assert np.max(np.abs(back - x)) < 1e-13 * n


@pytest.mark.parametrize("shape", [(12,), (6, 4), (8, 6, 4), (10, 2, 6)])
def test_library_fft_matches_naive(shape):
    rng = np.random.default_rng(0)
    x = rng.standard_normal(shape)
    a = sp.fwd(x)
    b = sp.dft_naive(x)
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(b))
    assert np.max(np.abs(np.real(sp.inv(a)) - x)) < 1e-13


def test_parseval():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((6, 8, 10))
    X = sp.fwd(x)
    assert abs(np.sum(x ** 2) - np.sum(np.abs(X) ** 2) / x.size) < 1e-12 * np.sum(x ** 2)


@pytest.mark.parametrize("L", [2 * math.pi, 1.0, 3.5])
def test_derivative_closed_form_1d(L):
    n = 16
    g = sp.Grid((n,), (L,))
    x = L * np.arange(n) / n
    for m in range(1, n // 2):
        k = 2 * math.pi * m / L
        assert np.max(np.abs(sp.deriv(np.sin(k * x), g, 0) - k * np.cos(k * x))) < 1e-12 * k
        assert np.max(np.abs(sp.deriv(np.cos(k * x), g, 0) + k * np.sin(k * x))) < 1e-12 * k
        assert np.max(np.abs(sp.lap(np.cos(k * x), g) + k * k * np.cos(k * x))) < 1e-11 * k * k
    # the Nyquist mode is in the null space of D (k~ = 0 there)
    ny = np.cos(math.pi * np.arange(n))
    assert np.max(np.abs(sp.deriv(ny, g, 0))) < 1e-13


def test_derivative_closed_form_3d_axes():
    n = (8, 6, 10)
    L = (2 * math.pi, 1.0, 4.0)
    g = sp.Grid(n, L)
    x, y, z = g.coords()
    kx, ky, kz = 2 * math.pi * 3 / L[0], 2 * math.pi * 2 / L[1], 2 * math.pi * 1 / L[2]
    f = np.sin(kx * x) * np.cos(ky * y) * np.sin(kz * z)
    assert np.allclose(sp.deriv(f, g, 0), kx * np.cos(kx * x) * np.cos(ky * y) * np.sin(kz * z), atol=1e-12)
    assert np.allclose(sp.deriv(f, g, 1), -ky * np.sin(kx * x) * np.sin(ky * y) * np.sin(kz * z), atol=1e-12)
    assert np.allclose(sp.deriv(f, g, 2), kz * np.sin(kx * x) * np.cos(ky * y) * np.cos(kz * z), atol=1e-12)
    assert np.allclose(sp.lap(f, g), -(kx ** 2 + ky ** 2 + kz ** 2) * f, atol=1e-10)


@pytest.mark.parametrize("n,L", [((8,), (2 * math.pi,)), ((4, 6), (1.0, 2.0)), ((4, 4, 6), (2 * math.pi,) * 3)])
def test_derivative_skew_symmetric(n, L):
    g = sp.Grid(n, L)
    for j in range(g.ndim):
        D = assemble(lambda v: sp.deriv(v, g, j), g.shape)
        assert np.linalg.norm(D + D.T) <= 1e-13 * np.linalg.norm(D)


def test_null_mask_counts():
    for n in [(8,), (6, 4), (4, 6, 8)]:
        g = sp.Grid(n, (1.0,) * len(n))
        assert int(sp.null_mask(g).sum()) == 2 ** len(n)


def test_preconditioners_invert_constant_density_operators():
    g = sp.Grid((8, 6, 10), (2 * math.pi, 1.0, 3.0))
    rng = np.random.default_rng(3)
    v = sp.project_range(rng.standard_normal(g.shape), g)
    assert np.max(np.abs(sp.precond_pressure(sp.lap(v, g), g) - v)) < 1e-12 * np.max(np.abs(v))
    a = 0.37
    w = rng.standard_normal(g.shape)
    assert np.max(np.abs(sp.precond_velocity(w - a * sp.lap(w, g), g, a) - w)) < 1e-12 * np.max(np.abs(w))
    # the pseudo-inverse maps the null space to zero
    cz = np.ones(g.shape)
    assert np.max(np.abs(sp.precond_pressure(cz, g))) < 1e-14


def test_planted_mistake_nyquist_breaks_pseudo_inverse(monkeypatch):
    """If |k~|^2 kept the Nyquist wavenumber, the preconditioner would no longer be the
    pseudo-inverse of sum_j D_j D_j, and the constant-density pin would fail."""
    g = sp.Grid((8, 6), (2 * math.pi, 1.0))
    rng = np.random.default_rng(4)
    v = rng.standard_normal(g.shape)
    ddv = sum(sp.deriv(sp.deriv(v, g, j), g, j) for j in range(2))
    ok = sp.precond_pressure(ddv, g)
    assert np.max(np.abs(sp.lap(ok, g) - ddv)) < 1e-12 * np.max(np.abs(ddv))
    orig = sp.wavenumber_1d
    monkeypatch.setattr(sp, "wavenumber_1d", lambda n, L, zero_nyquist=True: orig(n, L, zero_nyquist=False))
    bad = sp.precond_pressure(ddv, g)
    assert np.max(np.abs(bad - ok)) > 1e-3 * np.max(np.abs(ok))
