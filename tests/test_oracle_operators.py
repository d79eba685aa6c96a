"""Pins of the oracle's operators against closed forms (CPU only).

The closed forms below are worked out by hand from the continuous definitions
(Eq. VDINSE.Lrho: div(rho^-1 grad p); Eq. VDINSE.zeta: rho^-1 [Lap u + Sc^-1((u.grad)grad rho
+ (grad rho.grad)u)]), using the manufactured fields of Sec. 4.1 (Eq. VDINSE.solexact):
Taylor--Green velocity, p = sin 2x sin 2y sin 2z, rho = 1 + (s-1)/2 (1 + sin x sin y sin z).

* When every product that is differentiated is a trigonometric polynomial below the
  Nyquist index, the spectral result is exact, so the oracle must match the closed form
  to rounding (pressure with a trigonometric-polynomial 1/rho; velocity always, since
  only derivatives of rho and u are differentiated).
* With the paper's rho (1/rho not a polynomial), the pressure apply converges spectrally.
"""

import math

import numpy as np
import pytest

from oracle import spectral as sp
from oracle import operators as op


def tg_fields(n, s=10.0):
    g = sp.Grid((n, n, n), (2 * math.pi,) * 3)
    x, y, z = g.coords()
    sx, cx, sy, cy, sz, cz = np.sin(x), np.cos(x), np.sin(y), np.cos(y), np.sin(z), np.cos(z)
    return g, (sx, cx, sy, cy, sz, cz)


@pytest.mark.parametrize("n", [8, 12, 16])
def test_pressure_exact_for_polynomial_inverse_density(n):
    g, (sx, cx, sy, cy, sz, cz) = tg_fields(n)
    x, y, z = g.coords()
    s2x, c2x, s2y, c2y, s2z, c2z = (np.sin(2 * x), np.cos(2 * x), np.sin(2 * y), np.cos(2 * y),
                                    np.sin(2 * z), np.cos(2 * z))
    a = 1.0 + 0.5 * sx * sy * sz          # a = 1/rho
    p = s2x * s2y * s2z
    gp = (2 * c2x * s2y * s2z, 2 * s2x * c2y * s2z, 2 * s2x * s2y * c2z)
    ga = (0.5 * cx * sy * sz, 0.5 * sx * cy * sz, 0.5 * sx * sy * cz)
    f = a * (-12.0 * p) + sum(ga[j] * gp[j] for j in range(3))
    out = op.apply_pressure(1.0 / a, p * np.ones(g.shape), g)
    assert np.max(np.abs(out - f)) < 1e-11 * np.max(np.abs(f))


@pytest.mark.parametrize("s,ns,final", [(2.0, (8, 16, 24, 32), 1e-11), (10.0, (16, 32, 48, 64), 1e-9)])
def test_pressure_spectral_convergence_paper_density(s, ns, final):
    errs = []
    for n in ns:
        g, (sx, cx, sy, cy, sz, cz) = tg_fields(n)
        x, y, z = g.coords()
        rho = 1.0 + (s - 1) / 2 * (1.0 + sx * sy * sz)
        p = np.sin(2 * x) * np.sin(2 * y) * np.sin(2 * z)
        gp = (2 * np.cos(2 * x) * np.sin(2 * y) * np.sin(2 * z),
              2 * np.sin(2 * x) * np.cos(2 * y) * np.sin(2 * z),
              2 * np.sin(2 * x) * np.sin(2 * y) * np.cos(2 * z))
        grho = ((s - 1) / 2 * cx * sy * sz, (s - 1) / 2 * sx * cy * sz, (s - 1) / 2 * sx * sy * cz)
        f = -12.0 * p / rho - sum(grho[j] * gp[j] for j in range(3)) / rho ** 2
        out = op.apply_pressure(rho, p * np.ones(g.shape), g)
        errs.append(np.max(np.abs(out - f)) / np.max(np.abs(f)))
    # spectral (faster than any power of 1/n): every refinement cuts the error by a
    # growing factor, reaching near-rounding levels
    assert errs[-1] < final
    for e0, e1 in zip(errs, errs[1:]):
        assert e1 < 0.2 * e0


def test_velocity_exact_taylor_green():
    n = 8
    g, (sx, cx, sy, cy, sz, cz) = tg_fields(n)
    s, a, sc = 10.0, 0.01, 0.7
    c = (s - 1) / 2
    rho = 1.0 + c * (1.0 + sx * sy * sz)
    u = np.stack([sx * cy * cz, cx * sy * cz, -2 * cx * cy * sz])
    grho = [c * cx * sy * sz, c * sx * cy * sz, c * sx * sy * cz]
    H = [[-c * sx * sy * sz, c * cx * cy * sz, c * cx * sy * cz],
         [c * cx * cy * sz, -c * sx * sy * sz, c * sx * cy * cz],
         [c * cx * sy * cz, c * sx * cy * cz, -c * sx * sy * sz]]
    du = [[cx * cy * cz, -sx * sy * cz, -sx * cy * sz],
          [-sx * sy * cz, cx * cy * cz, -cx * sy * sz],
          [2 * sx * cy * sz, 2 * cx * sy * sz, -2 * cx * cy * cz]]
    expect = np.empty_like(u)
    for i in range(3):
        t = sum(u[j] * H[j][i] + grho[j] * du[i][j] for j in range(3))
        expect[i] = u[i] - a / rho * (-3.0 * u[i] + t / sc)
    out = op.apply_velocity(rho, u, g, a, 1.0 / sc)
    assert np.max(np.abs(out - expect)) < 1e-12


def test_velocity_1d_matches_paper_form():
    """1D, Sc = 1: V u = (I - a/rho (D^2 + rho'' + rho' D)) u (Eq. VDINSE.Vrho)."""
    n = 32
    g = sp.Grid((n,), (2 * math.pi,))
    x = 2 * math.pi * np.arange(n) / n
    rho = 1.0 + 0.3 * np.sin(x)
    u = np.sin(2 * x) + 0.2 * np.cos(5 * x)
    du = 2 * np.cos(2 * x) - np.sin(5 * x)
    d2u = -4 * np.sin(2 * x) - 5 * np.cos(5 * x)
    a = 0.05
    expect = u - a / rho * (d2u + (-0.3 * np.sin(x)) * u + 0.3 * np.cos(x) * du)
    out = op.apply_velocity(rho, u[None, :], g, a, 1.0)[0]
    assert np.max(np.abs(out - expect)) < 1e-13


def test_constant_density_operators_reduce_to_constant_coefficient():
    g = sp.Grid((6, 8, 4), (1.0, 2.0, 3.0))
    rng = np.random.default_rng(7)
    phi = rng.standard_normal(g.shape)
    rho0 = 2.5
    rho = np.full(g.shape, rho0)
    assert np.allclose(op.apply_pressure(rho, phi, g), sp.lap(phi, g) / rho0, atol=1e-11)
    u = rng.standard_normal((3,) + g.shape)
    a = 0.1
    out = op.apply_velocity(rho, u, g, a, 1.3)
    expect = np.stack([u[i] - a / rho0 * sp.lap(u[i], g) for i in range(3)])
    assert np.allclose(out, expect, atol=1e-11)


def test_planted_mistake_sign_in_velocity_coupling(monkeypatch):
    """Dropping the (u.grad) grad rho term must break the closed-form pin."""
    n = 8
    g, (sx, cx, sy, cy, sz, cz) = tg_fields(n)
    c = 4.5
    rho = 1.0 + c * (1.0 + sx * sy * sz)
    u = np.stack([sx * cy * cz, cx * sy * cz, -2 * cx * cy * sz])
    good = op.apply_velocity(rho, u, g, 0.01, 1.0)
    rd = op.RhoDerivs(rho, g)
    rd.h = [[np.zeros(g.shape)] * 3 for _ in range(3)]
    bad = op.apply_velocity(rho, u, g, 0.01, 1.0, rd)
    assert np.max(np.abs(good - bad)) > 1e-3
