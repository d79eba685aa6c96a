"""Seeded synthetic inputs shaped like the paper's test cases.

This module only builds input fields (densities, right-hand sides, velocity fields,
instance lists and arrival traces) with numpy; it holds none of the solver's arithmetic.
Both the CUDA path and the CPU oracle consume what it returns, so that the two sides
are compared on identical inputs.  Random numbers come from ``numpy.random.default_rng``
with the seed stated for each workload.

Array convention: physical fields are float64 numpy arrays of shape (n2, n1, n0) in 3D,
(n1, n0) in 2D and (n0,) in 1D, x (axis 0) fastest; vector fields stack components
first: (d, *shape).
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def coords(n, L):
    """Physical coordinates of a periodic grid, one broadcastable array per axis (x first)."""
    d = len(n)
    out = []
    for j in range(d):
        c = L[j] * np.arange(n[j]) / n[j]
        sh = [1] * d
        sh[d - 1 - j] = n[j]
        out.append(c.reshape(sh))
    return out


# ---------------------------------------------------------------------------------------
# 1D top-hat (Sec. 3.1, Eq. VDINSE.rho.hat, with the interface positions and width of
# the 1D periodic workload: rho = 1 + (r-1)/2 (tanh((x-a)/d) - tanh((x-b)/d)))
# ---------------------------------------------------------------------------------------

def tophat_1d(n=256, r=3.0, a=math.pi / 2, b=3 * math.pi / 2, d=0.05, L=2 * math.pi):
    x = L * np.arange(n) / n
    return 1.0 + (r - 1.0) * 0.5 * (np.tanh((x - a) / d) - np.tanh((x - b) / d))


def modes_rhs_1d(n=256, nmodes=16, seed=1, L=2 * math.pi):
    """f = sum_{k=1..nmodes} (a_k cos kx + b_k sin kx)/k^2, a_k, b_k ~ N(0,1): zero mean."""
    rng = np.random.default_rng(seed)
    ab = rng.standard_normal((nmodes, 2))
    x = L * np.arange(n) / n
    f = np.zeros(n)
    for k in range(1, nmodes + 1):
        kk = 2 * math.pi * k / L
        f += (ab[k - 1, 0] * np.cos(kk * x) + ab[k - 1, 1] * np.sin(kk * x)) / k ** 2
    return f


# ---------------------------------------------------------------------------------------
# 2D Rayleigh--Taylor-like layer (Sec. 4.2 RTI profile, made doubly periodic: a heavy slab
# between z = 0.5 and z = 1.5, its lower interface perturbed by eta(x))
# ---------------------------------------------------------------------------------------

@dataclass
class RTCase:
    n: tuple
    L: tuple
    rho: np.ndarray
    u: np.ndarray
    Re: float
    Sc: float
    Fr: float
    dt: float
    gravity_axis: int


def rt_2d(nx=512, nz=1024, Lx=1.0, Lz=2.0, s=3.0, delta=0.02, eta_amp=0.05,
          noise=1e-3, seed=2, Re=1000.0, Sc=1.0, Fr=1.0, dt=1e-3):
    x, z = coords((nx, nz), (Lx, Lz))
    eta = eta_amp * np.cos(2 * math.pi * x / Lx)
    rho = 1.0 + (s - 1.0) / 2.0 * (np.tanh((z - 0.5) / delta + eta) - np.tanh((z - 1.5) / delta))
    rho = np.array(np.broadcast_to(rho, (nz, nx)), copy=True)
    rng = np.random.default_rng(seed)
    u = noise * rng.standard_normal((2, nz, nx))
    return RTCase(n=(nx, nz), L=(Lx, Lz), rho=rho, u=u, Re=Re, Sc=Sc, Fr=Fr, dt=dt, gravity_axis=1)


# ---------------------------------------------------------------------------------------
# 3D swirling-jet-like density (Sec. 4.3 swirling jet, with a tanh shear layer) on a 2 pi
# box, jet axis x; base axial velocity V_x = (1 - tanh((r-R)/d))/2, swirl V_theta = q r V_x
# ---------------------------------------------------------------------------------------

@dataclass
class JetCase:
    n: tuple
    L: tuple
    rho: np.ndarray
    u: np.ndarray          # predictor velocity u* (3, n2, n1, n0)


def jet_3d(n=256, s=0.5, R=0.5, d=0.05, q=1.0, noise=1e-3, seed=3, L=2 * math.pi):
    x, y, z = coords((n, n, n), (L, L, L))
    yc, zc = y - L / 2, z - L / 2
    r = np.sqrt(yc ** 2 + zc ** 2)
    prof = np.broadcast_to(0.5 * (1.0 - np.tanh((r - R) / d)), (n, n, n))
    rho = np.ascontiguousarray(1.0 + (s - 1.0) * prof)
    rng = np.random.default_rng(seed)
    u = np.empty((3, n, n, n))
    # V_theta e_theta = q r V_x (-sin t, cos t) in the (y, z) plane
    u[0] = prof
    u[1] = -q * prof * zc
    u[2] = q * prof * yc
    u += noise * rng.standard_normal(u.shape)
    return JetCase(n=(n, n, n), L=(L, L, L), rho=rho, u=u)


# ---------------------------------------------------------------------------------------
# Random rhs for apply/solve parity tests
# ---------------------------------------------------------------------------------------

def random_field(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def smooth_random_field(n, L, seed, kmax=6):
    """Sum of random Fourier modes with |m_j| <= kmax on each axis (band-limited)."""
    rng = np.random.default_rng(seed)
    X = coords(n, L)
    d = len(n)
    f = np.zeros(tuple(reversed(n)))
    for _ in range(12):
        m = rng.integers(-kmax, kmax + 1, size=d)
        ph = rng.uniform(0, 2 * math.pi)
        amp = rng.standard_normal()
        arg = sum(2 * math.pi * m[j] * X[j] / L[j] for j in range(d))
        f = f + amp * np.cos(arg + ph)
    return f


def slab_density(n, L, s, axis, centre, width, thick):
    """Top-hat slab of density ratio s along ``axis``: 1 + (s-1)/2 (tanh((x-c+w/2)/t) - tanh((x-c-w/2)/t)),
    wrapped periodically (the distance to the centre is taken modulo L)."""
    X = coords(n, L)
    xa = X[axis]
    La = L[axis]
    dist = (xa - centre + La / 2) % La - La / 2
    rho = 1.0 + (s - 1.0) / 2.0 * (np.tanh((dist + width / 2) / thick) - np.tanh((dist - width / 2) / thick))
    return np.ascontiguousarray(np.broadcast_to(rho, tuple(reversed(n))))


# ---------------------------------------------------------------------------------------
# Batched uneven instances (96 instances, seed 4) and serving trace (seed 5)
# ---------------------------------------------------------------------------------------

SIZES_2D = (64, 96, 128, 160, 192, 256, 320, 384, 512)
SIZES_3D = (32, 48, 64, 80, 96, 128, 160)


@dataclass
class Instance:
    n: tuple
    L: tuple
    s: float
    axis: int
    centre: float
    thick: float
    tol: float = 1e-10

    def density(self):
        return slab_density(self.n, self.L, self.s, self.axis, self.centre, self.L[self.axis] / 2, self.thick)


def batch_instances(count=96, seed=4, sizes_2d=SIZES_2D, sizes_3d=SIZES_3D, tol=1e-10):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        is3d = (i % 2) == 1
        if is3d:
            m = int(rng.choice(sizes_3d))
            n = (m, m, m)
        else:
            m = int(rng.choice(sizes_2d))
            n = (m, m)
        L = tuple([2 * math.pi] * len(n))
        s = float(math.exp(rng.uniform(math.log(2.0), math.log(50.0))))
        axis = int(rng.integers(0, len(n)))
        centre = float(rng.uniform(0, L[axis]))
        thick = 3.0 * L[axis] / n[axis]
        out.append(Instance(n=n, L=L, s=s, axis=axis, centre=centre, thick=thick, tol=tol))
    return out


def serving_trace(count=20000, rate=2000.0, seed=5, p_big=0.05, big=256):
    """Poisson arrivals: (t_arrival, Instance); 95% drawn like the batched set, 5% 256^3."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    pool = batch_instances(count=max(count, 2), seed=seed + 100)
    out = []
    for i in range(count):
        if rng.uniform() < p_big:
            L = (2 * math.pi,) * 3
            inst = Instance(n=(big, big, big), L=L, s=float(math.exp(rng.uniform(math.log(2), math.log(50)))),
                            axis=int(rng.integers(0, 3)), centre=float(rng.uniform(0, L[0])), thick=3 * L[0] / big)
        else:
            inst = pool[i]
        inst.tol = float(rng.choice([1e-6, 1e-8, 1e-10]))
        out.append((float(t[i]), inst))
    return out
