"""Single-launch 1D pressure solves (one thread block runs the whole Krylov solve).

vd_solve routes FP64 pressure solves on 1D grids to one kernel launch.  Against the oracle:
solutions match the exact, non-iterative 1D solve (oracle.direct1d) to 1e-10 in relative
2-norm; iteration counts are within one of the oracle's own CG / GMRES / RMR on the same
problem; fixed-iteration iterates (tol 0, k iterations) agree with the oracle's to 1e-10;
histories follow the oracle's.  Lengths cover radix 2 (256, 1024: 64 and 128 threads), mixed
radix (240 = 2^4 3 5), GMRES with several restarts, warm starts, capped solves and a rhs in
the null space.
"""

import math

import numpy as np
import pytest
import torch

import paper_2403_06654_gb300 as vd
from paper_2403_06654_gb300 import inputs
from oracle import operators as op
from oracle import solvers as sv
from oracle import spectral as sp
from oracle.direct1d import solve_pressure_1d

pytestmark = pytest.mark.gpu


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def N(t):
    return t.detach().cpu().numpy()


def rel2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def case(n, r=3.0, d=0.05, seed=1):
    g = sp.Grid((n,), (2 * math.pi,))
    rho = inputs.tophat_1d(n=n, r=r, d=d)
    f = inputs.modes_rhs_1d(n=n, seed=seed)
    return g, rho, f


@pytest.mark.parametrize("n", [256, 240, 1024])
@pytest.mark.parametrize("solver", ["cg", "gmres", "rmr"])
def test_small_solve_matches_exact_and_oracle(n, solver):
    g, rho, f = case(n, d=max(0.05, 8 * math.pi / n))
    exact = solve_pressure_1d(rho, sp.project_range(f, g), g)
    A, M = op.pressure_system(rho, g)
    ref = sv.solve(solver, A, M, sp.project_range(f, g), tol=1e-12, maxit=600, restart=30)
    G = vd.Grid((n,), (2 * math.pi,))
    G.set_density(T(rho))
    l0 = vd.vd_launch_count()
    x, info = G.solve("pressure", solver, T(f), tol=1e-12, max_it=600, restart=30, hist_cap=700)
    launches = vd.vd_launch_count() - l0
    assert info["status"] == "converged", info
    assert rel2(N(x), exact) < 1e-10
    assert abs(info["iters"] - ref.iters) <= 1
    h = np.array(info["hist"])
    k = min(len(h), len(ref.history))
    assert np.allclose(h[:k], ref.history[:k], rtol=1e-6, atol=1e-14)
    # the whole solve is one kernel, except GMRES(30) at n = 1024, whose 32 basis vectors do not
    # fit in shared memory: it runs pass by pass
    if solver == "gmres" and n > 512:
        assert launches > 1
    else:
        assert launches == 1


@pytest.mark.parametrize("solver", ["cg", "gmres", "rmr"])
def test_small_solve_fixed_iterations(solver):
    g, rho, f = case(256, r=8.0, d=0.1, seed=3)
    fb = sp.project_range(f, g)
    A, M = op.pressure_system(rho, g)
    k = 7
    ref = sv.solve(solver, A, M, fb, tol=0.0, maxit=k, restart=3)
    G = vd.Grid((256,), (2 * math.pi,))
    G.set_density(T(rho))
    x, info = G.solve("pressure", solver, T(f), tol=0.0, max_it=k, restart=3)
    assert info["iters"] == k and info["status"] == "max_iter"
    assert rel2(N(x), ref.x) < 1e-10


def test_small_solve_warm_start_and_edge_cases():
    g, rho, f = case(256)
    G = vd.Grid((256,), (2 * math.pi,))
    G.set_density(T(rho))
    x, info = G.solve("pressure", "cg", T(f), tol=1e-12, max_it=400)
    # warm start from the solution: converged at once
    x2, i2 = G.solve("pressure", "cg", T(f), x0=x, tol=1e-10, max_it=400)
    assert i2["status"] == "converged" and i2["iters"] == 0
    # warm start from a perturbed solution: fewer iterations than from zero, same answer
    x0 = x + 1e-3 * T(inputs.random_field(g.shape, 4))
    x3, i3 = G.solve("pressure", "cg", T(f), x0=x0, tol=1e-12, max_it=400)
    assert i3["status"] == "converged" and rel2(N(x3), N(x)) < 1e-10
    # constant + Nyquist rhs (null space): x = 0 at once, the removed part reported
    s = (-1.0) ** np.arange(256)
    xz, iz = G.solve("pressure", "gmres", T(2.0 + 0.5 * s), tol=1e-10, max_it=50)
    assert iz["iters"] == 0 and iz["status"] == "converged" and float(N(xz).max()) == 0.0
    # the removed part of a rhs with a mean
    fb = f + 0.25
    _, ir = G.solve("pressure", "cg", T(fb), tol=1e-12, max_it=400)
    expect = np.linalg.norm(fb - sp.project_range(fb, g)) / np.linalg.norm(fb)
    assert abs(ir["rhs_removed"] - expect) < 1e-12
    # constant density: one iteration for every solver
    G.set_density(T(np.full(g.shape, 2.5)))
    for solver in ("cg", "gmres", "rmr"):
        _, ic = G.solve("pressure", solver, T(f), tol=1e-12, max_it=10)
        assert ic["status"] == "converged" and ic["iters"] == 1
