"""Velocity solves with the float-pair refinement residual (mixed_dd), against the FP64 oracle.

In mixed_dd the refinement residual b - V~ x of the velocity operator (Eq. VDINSE.zeta with the
Crank-Nicolson factor a) is formed with float-pair transforms; the pointwise bracket
rho^-1 (Lap u + Sc^-1 (...)) stays double.  Checked here: the float-pair residual of a converged
FP64 solution agrees with the oracle's double residual within the normwise float-pair scale
2^-47 |V| |x| / |b|; mixed_dd GMRES and RMR solves return a field whose residual under the
oracle's operator is at most the reported one (within that scale), and agree with the oracle's
solution; 1D, 2D and 3D grids and a density ratio up to 20.  The graph batch's mixed_dd
velocity systems are compared with these solves in tests/test_gpu_batch.py.
"""

import math

import numpy as np
import pytest
import torch

import paper_2403_06654_gb300 as vd
from paper_2403_06654_gb300 import inputs
from oracle import spectral as sp
from oracle import operators as op
from oracle import solvers as sv

pytestmark = pytest.mark.gpu

GRIDS = [((64,), (2 * math.pi,)), ((48, 40), (2 * math.pi, 2.0)), ((24, 20, 16), (2 * math.pi,) * 3),
         ((32, 32, 32), (2 * math.pi,) * 3)]


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def N(t):
    return t.detach().cpu().numpy()


def rel2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _case(n, L, s, seed):
    g = sp.Grid(n, L)
    ax = g.ndim - 1
    rho = inputs.slab_density(g.n, g.L, s, ax, 0.4 * L[ax], 0.5 * L[ax], 3 * L[ax] / n[ax])
    b = np.stack([inputs.smooth_random_field(g.n, g.L, seed + c, kmax=5) for c in range(g.ndim)])
    return g, rho, b


def _scale(g, rho, a, x, b):
    """normwise float-pair scale 2^-47 |V| |x| / |b|, |V| <= 1 + a |k|_max^2 max(1/rho) (the
    bracket's first-order terms are smaller for these smooth densities)"""
    kmax2 = sum((math.pi * g.n[j] / g.L[j]) ** 2 for j in range(g.ndim))
    vnorm = 1.0 + a * kmax2 * float(np.max(1.0 / rho)) * 2.0
    return 2.0 ** -47 * vnorm * np.linalg.norm(x) / np.linalg.norm(b)


@pytest.mark.parametrize("n,L", GRIDS)
def test_float_pair_velocity_residual_accuracy(n, L):
    g, rho, b = _case(n, L, 5.0, 41)
    a, isc = 2e-3, 1.0
    G = vd.Grid(n, L)
    G.set_density(T(rho), "velocity")
    x0, i0 = G.solve("velocity", "gmres", T(b), a=a, inv_sc=isc, tol=1e-13, max_it=300, restart=30)
    assert i0["status"] == "converged"
    # one evaluation of b - V x0 in float pairs (warm start, no iteration)
    _, info = G.solve("velocity", "gmres", T(b), x0=x0, a=a, inv_sc=isc, tol=0.0, max_it=0, precision="mixed_dd")
    assert info["iters"] == 0
    A, M = op.velocity_system(rho, g, a, isc)
    xs = N(x0)
    r64 = np.linalg.norm(b - A(xs)) / np.linalg.norm(b)
    bound = _scale(g, rho, a, xs, b)
    assert abs(info["relres_true"] - r64) <= bound, (info["relres_true"], r64, bound)


@pytest.mark.parametrize("solver", ["gmres", "rmr"])
@pytest.mark.parametrize("s", [3.0, 20.0])
@pytest.mark.parametrize("n,L", GRIDS)
def test_mixed_dd_velocity_solves_match_oracle(n, L, s, solver):
    g, rho, b = _case(n, L, s, 43)
    a, isc = 1e-3, 1.0
    A, M = op.velocity_system(rho, g, a, isc)
    ref = sv.gmres(A, M, b, tol=1e-13, maxit=400, restart=60)
    G = vd.Grid(n, L)
    G.set_density(T(rho), "velocity")
    x, info = G.solve("velocity", solver, T(b), a=a, inv_sc=isc, tol=1e-10, max_it=600, restart=30,
                      precision="mixed_dd")
    assert info["status"] == "converged", info
    assert info["relres_true"] <= 1e-10
    xs = N(x)
    r = np.linalg.norm(b - A(xs)) / np.linalg.norm(b)
    bound = _scale(g, rho, a, xs, b)
    # The reported residual is the spectral iterate's.  The inverse real transform of the
    # returned field keeps only the Hermitian part of the kx = 0 (and kx = n0/2) planes, where
    # rounding in the inner float solves leaves a small anti-Hermitian part: the returned field's
    # residual is at most the reported one (2D here: 3.51e-11 against 4.37e-11, in mixed too).
    assert r <= info["relres_true"] + bound, (r, info["relres_true"], bound)
    # the float-pair residual of the returned field itself, against the double one
    _, i2 = G.solve("velocity", solver, T(b), x0=x, a=a, inv_sc=isc, tol=0.0, max_it=0, precision="mixed_dd")
    assert abs(i2["relres_true"] - r) <= bound, (i2["relres_true"], r, bound)
    assert rel2(xs, ref.x) <= s * 1e-9
