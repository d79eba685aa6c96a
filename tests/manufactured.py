"""Manufactured Taylor--Green solution of the variable-density equations (Sec. 4.1) and the
mass source and body force that make it exact (test helper; uses the oracle's spectral
derivatives on the sampled exact fields, analytic time derivatives).

Exact fields (density ratio s):
    u = cos t sin x cos y cos z,  v = cos t cos x sin y cos z,  w = -2 cos t cos x cos y sin z,
    p = sin t sin 2x sin 2y sin 2z,  rho = 1 + (s - 1)/2 (1 + sin t sin x sin y sin z).
The equations the step discretises (Sec. 2) are
    rho_t + u.grad rho = (Re Sc)^-1 Lap rho + S,
    u_t + (u.grad) u = -grad p / rho + zeta(rho, u) + F,
    zeta(rho, u) = (rho Re)^-1 [Lap u + Sc^-1 ((u.grad) grad rho + (grad rho.grad) u)],
so S and F are those equations' residuals at the exact fields.
"""

import math

import numpy as np

from oracle import operators as op
from oracle import spectral as sp


def grid(n):
    return sp.Grid((n, n, n), (2 * math.pi,) * 3)


def exact(g, t, s):
    x, y, z = g.coords()
    sx, cx, sy, cy, sz, cz = np.sin(x), np.cos(x), np.sin(y), np.cos(y), np.sin(z), np.cos(z)
    full = np.zeros(g.shape)
    shape_u = np.stack([full + sx * cy * cz, full + cx * sy * cz, full - 2 * cx * cy * sz])
    u = math.cos(t) * shape_u
    du = -math.sin(t) * shape_u
    p = full + math.sin(t) * np.sin(2 * x) * np.sin(2 * y) * np.sin(2 * z)
    rho = full + 1 + 0.5 * (s - 1) * (1 + math.sin(t) * sx * sy * sz)
    drho = full + 0.5 * (s - 1) * math.cos(t) * sx * sy * sz
    return rho, u, p, drho, du


def grad_p(g, t, s):
    _, _, p, _, _ = exact(g, t, s)
    return np.stack([sp.deriv(p, g, j) for j in range(3)])


def sources(g, t, s, Re, Sc):
    rho, u, p, drho, du = exact(g, t, s)
    gr = [sp.deriv(rho, g, j) for j in range(3)]
    S = drho + sum(u[j] * gr[j] for j in range(3)) - sp.lap(rho, g) / (Re * Sc)
    adv = np.stack([sum(u[j] * sp.deriv(u[i], g, j) for j in range(3)) for i in range(3)])
    gp = np.stack([sp.deriv(p, g, j) for j in range(3)])
    # zeta = (u - V u) / (a Re) with the oracle's V for a = 1
    zeta = (u - op.apply_velocity(rho, u, g, 1.0, 1.0 / Sc)) / Re
    F = du + adv + gp / rho - zeta
    return S, F


def rms(a):
    return float(np.sqrt(np.mean(a * a)))
