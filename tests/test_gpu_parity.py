"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (FP64): transforms, derivatives and operator applies are compared element by
element with a relative max-norm bound of 1e-12 (the rounding of a few FFT passes on
O(1e3..1e5)-sized operator norms stays far below); solutions solved to 1e-12/1e-13 on both
sides must agree to 1e-10 in relative 2-norm (the parity bound), and iterates after a
fixed number k of iterations from the same start must agree to 1e-10.
Sizes span several tiles with ragged tails (h0 = n0/2 + 1 columns never a multiple of the
tile width) and radix 2, 3 and 5 lengths.
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
from oracle.direct1d import solve_pressure_1d

pytestmark = pytest.mark.gpu

DEV = "cuda"


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def N(t):
    return t.detach().cpu().numpy()


def relmax(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def rel2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


GRIDS = [
    ((256,), (2 * math.pi,)),
    ((40,), (3.0,)),
    ((48, 30), (2 * math.pi, 1.5)),
    ((64, 40), (1.0, 2.0)),
    ((20, 12, 30), (2 * math.pi, 1.0, 3.0)),
    ((32, 24, 16), (2 * math.pi,) * 3),
    ((128, 16, 12), (2 * math.pi, 1.0, 2.0)),
    ((256, 8, 10), (2 * math.pi,) * 3),
    ((512, 24), (1.0, 2.0)),
]


def smooth_density(g, s=4.0, seed=0):
    f = inputs.smooth_random_field(g.n, g.L, seed, kmax=3)
    f = (f - f.min()) / (f.max() - f.min())
    return 1.0 + (s - 1.0) * f


@pytest.mark.parametrize("n,L", GRIDS)
def test_gradient_and_divergence(n, L):
    g = sp.Grid(n, L)
    G = vd.Grid(n, L)
    phi = inputs.random_field(g.shape, 1)
    got = N(G.gradient(T(phi)))
    for j in range(g.ndim):
        assert relmax(got[j], sp.deriv(phi, g, j)) < 1e-12
    u = inputs.random_field((g.ndim,) + g.shape, 2)
    assert relmax(N(G.divergence(T(u))), sp.div(list(u), g)) < 1e-12


@pytest.mark.parametrize("n,L", GRIDS)
def test_pressure_apply(n, L):
    g = sp.Grid(n, L)
    G = vd.Grid(n, L)
    rho = smooth_density(g)
    G.set_density(T(rho), "pressure")
    phi = inputs.random_field(g.shape, 3)
    got = N(G.apply("pressure", T(phi)))
    assert relmax(got, op.apply_pressure(rho, phi, g)) < 1e-12


@pytest.mark.parametrize("n,L", GRIDS)
def test_velocity_apply(n, L):
    g = sp.Grid(n, L)
    G = vd.Grid(n, L)
    rho = smooth_density(g, 3.0, 4)
    G.set_density(T(rho), "velocity")
    u = inputs.random_field((g.ndim,) + g.shape, 5)
    a, isc = 2e-3, 0.8
    got = N(G.apply("velocity", T(u), a=a, inv_sc=isc))
    assert relmax(got, op.apply_velocity(rho, u, g, a, isc)) < 1e-12


@pytest.mark.parametrize("n,L", GRIDS[:4])
def test_preconditioners(n, L):
    g = sp.Grid(n, L)
    G = vd.Grid(n, L)
    v = inputs.random_field(g.shape, 6)
    assert relmax(N(G.precond("pressure", T(v))), sp.precond_pressure(v, g)) < 1e-13
    u = inputs.random_field((g.ndim,) + g.shape, 7)
    a = 0.01
    got = N(G.precond("velocity", T(u), a=a))
    for i in range(g.ndim):
        assert relmax(got[i], sp.precond_velocity(u[i], g, a)) < 1e-13


@pytest.mark.parametrize("solver", ["cg", "gmres", "rmr"])
def test_config1_1d_solves_match_exact(solver):
    n = 256
    g = sp.Grid((n,), (2 * math.pi,))
    rho = inputs.tophat_1d(n=n)
    f = inputs.modes_rhs_1d(n=n)
    exact = solve_pressure_1d(rho, f, g)
    A, M = op.pressure_system(rho, g)
    ref = sv.solve(solver, A, M, f, tol=1e-12, maxit=400, restart=30)
    G = vd.Grid((n,), (2 * math.pi,))
    G.set_density(T(rho))
    x, info = G.solve("pressure", solver, T(f), tol=1e-12, max_it=400, restart=30, hist_cap=500)
    assert info["status"] == "converged"
    assert rel2(N(x), exact) < 1e-10
    assert abs(info["iters"] - ref.iters) <= 1
    assert info["relres_true"] < 5e-12
    h = np.array(info["hist"])
    k = min(len(h), len(ref.history))
    assert np.allclose(h[:k], ref.history[:k], rtol=1e-6, atol=1e-14)


@pytest.mark.parametrize("solver", ["cg", "gmres", "rmr"])
@pytest.mark.parametrize("n,L", [((40, 24), (2 * math.pi, 1.0)), ((20, 12, 30), (2 * math.pi, 1.0, 3.0))])
def test_pressure_solves_nd(solver, n, L):
    g = sp.Grid(n, L)
    rho = inputs.slab_density(g.n, g.L, 5.0, g.ndim - 1, 0.5 * g.L[-1], 0.5 * g.L[-1], 4 * g.L[-1] / g.n[-1])
    f = inputs.smooth_random_field(g.n, g.L, 9, kmax=4)
    A, M = op.pressure_system(rho, g)
    fb = sp.project_range(f, g)
    ref = sv.solve(solver, A, M, fb, tol=1e-13, maxit=500, restart=30)
    G = vd.Grid(n, L)
    G.set_density(T(rho))
    x, info = G.solve("pressure", solver, T(f), tol=1e-13, max_it=500, restart=30)
    assert info["status"] == "converged"
    assert rel2(N(x), ref.x) < 1e-10
    assert abs(info["iters"] - ref.iters) <= 1


@pytest.mark.parametrize("solver", ["cg", "gmres", "rmr"])
def test_fixed_iterations_iterates_agree(solver):
    n, L = (24, 18, 10), (2 * math.pi, 1.0, 2.0)
    g = sp.Grid(n, L)
    rho = smooth_density(g, 6.0, 11)
    f = sp.project_range(inputs.random_field(g.shape, 12), g)
    A, M = op.pressure_system(rho, g)
    k = 5
    ref = sv.solve(solver, A, M, f, tol=0.0, maxit=k, restart=30)
    G = vd.Grid(n, L)
    G.set_density(T(rho))
    x, info = G.solve("pressure", solver, T(f), tol=0.0, max_it=k, restart=30)
    assert info["iters"] == k and info["status"] == "max_iter"
    assert rel2(N(x), ref.x) < 1e-10


@pytest.mark.parametrize("solver", ["gmres", "rmr"])
@pytest.mark.parametrize("n,L", [((64,), (2 * math.pi,)), ((32, 24), (2 * math.pi, 2 * math.pi)),
                                 ((12, 16, 10), (2 * math.pi,) * 3)])
def test_velocity_solves(solver, n, L):
    g = sp.Grid(n, L)
    rho = smooth_density(g, 3.0, 13)
    b = inputs.random_field((g.ndim,) + g.shape, 14)
    a, isc = 1e-2, 1.0
    A, M = op.velocity_system(rho, g, a, isc)
    ref = sv.gmres(A, M, b, tol=1e-13, maxit=300, restart=60)
    G = vd.Grid(n, L)
    G.set_density(T(rho), "velocity")
    x, info = G.solve("velocity", solver, T(b), a=a, inv_sc=isc, tol=1e-12, max_it=300, restart=30)
    assert info["status"] == "converged"
    assert rel2(N(x), ref.x) < 1e-10


@pytest.mark.parametrize("solver", ["cg", "gmres", "rmr"])
def test_constant_density_one_iteration(solver):
    n, L = (32, 24, 20), (2 * math.pi, 1.0, 3.0)
    g = sp.Grid(n, L)
    G = vd.Grid(n, L)
    G.set_density(T(np.full(g.shape, 2.5)))
    f = inputs.random_field(g.shape, 15)
    x, info = G.solve("pressure", solver, T(f), tol=1e-12, max_it=10)
    assert info["status"] == "converged" and info["iters"] == 1
    ref = sp.precond_pressure(sp.project_range(f, g), g) * 2.5
    assert rel2(N(x), ref) < 1e-12


@pytest.mark.parametrize("solver", ["cg", "gmres", "rmr"])
def test_mixed_precision_reaches_fp64_residual(solver):
    n, L = (48, 40, 32), (2 * math.pi,) * 3
    g = sp.Grid(n, L)
    rho = inputs.slab_density(g.n, g.L, 2.0, 1, math.pi, 2.0, 0.3)
    f = inputs.smooth_random_field(g.n, g.L, 16, kmax=5)
    A, M = op.pressure_system(rho, g)
    ref = sv.solve(solver, A, M, sp.project_range(f, g), tol=1e-13, maxit=500)
    G = vd.Grid(n, L)
    G.set_density(T(rho))
    x, info = G.solve("pressure", solver, T(f), tol=1e-10, max_it=500, precision="mixed")
    assert info["status"] == "converged"
    assert info["relres_true"] <= 1e-10
    assert info["outer_iters"] >= 2
    # error vs the FP64 oracle solution, bounded by kappa * tol with kappa <= rho_max/rho_min = 2
    assert rel2(N(x), ref.x) < 2.5e-10


def test_edge_cases_and_errors():
    n, L = (16, 12), (1.0, 1.0)
    g = sp.Grid(n, L)
    G = vd.Grid(n, L)
    rho = np.full(g.shape, 1.0)
    G.set_density(T(rho))
    # zero rhs and a pure null-space rhs (constant) give x = 0 in zero iterations
    for b in (np.zeros(g.shape), np.full(g.shape, 3.0)):
        x, info = G.solve("pressure", "gmres", T(b), tol=1e-10, max_it=10)
        assert info["iters"] == 0 and info["status"] == "converged"
        assert float(np.max(np.abs(N(x)))) == 0.0
    # invalid density
    with pytest.raises(vd.VDError) as e:
        G.set_density(T(np.full(g.shape, -1.0)))
    assert e.value.status == vd.VD_ERR_INVALID_ARG
    G.set_density(T(rho), "velocity")
    with pytest.raises(vd.VDError) as e:
        G.solve("velocity", "cg", T(np.zeros((2,) + g.shape)), a=0.1)
    assert e.value.status == vd.VD_ERR_INVALID_ARG
    # max_it reached is reported, not raised
    rho2 = smooth_density(g, 8.0, 17)
    G.set_density(T(rho2))
    x, info = G.solve("pressure", "cg", T(inputs.random_field(g.shape, 18)), tol=1e-14, max_it=2)
    assert info["status"] == "max_iter" and info["iters"] == 2


def test_large_axis_2d_config2_shape():
    """512 x 1024 (the 2D workload's grid: longest axis 1024) pressure apply parity."""
    n, L = (512, 1024), (1.0, 2.0)
    g = sp.Grid(n, L)
    case = inputs.rt_2d()
    G = vd.Grid(n, L)
    G.set_density(T(case.rho))
    phi = inputs.smooth_random_field(n, L, 19, kmax=20)
    got = N(G.apply("pressure", T(phi)))
    assert relmax(got, op.apply_pressure(case.rho, phi, g)) < 1e-11


@pytest.mark.parametrize("solver", ["cg", "gmres", "rmr"])
@pytest.mark.parametrize("n,L", [((48, 40, 32), (2 * math.pi,) * 3), ((256,), (2 * math.pi,)),
                                 ((64, 48), (2 * math.pi, 1.0)), ((128, 20, 24), (2 * math.pi,) * 3),
                                 ((256, 16, 16), (2 * math.pi,) * 3)])
def test_mixed_dd_residual_matches_fp64(solver, n, L):
    """Refinement residual in float-pair arithmetic (~2^-48): the returned solution's double
    residual, recomputed here with the double operator, must also meet the tolerance, and the
    solution must match the FP64 oracle within kappa * tol."""
    g = sp.Grid(n, L)
    rho = inputs.slab_density(g.n, g.L, 2.0, g.ndim - 1, 0.5 * g.L[-1], 0.5 * g.L[-1], 4 * g.L[-1] / g.n[-1])
    f = inputs.smooth_random_field(g.n, g.L, 21, kmax=5)
    G = vd.Grid(n, L)
    G.set_density(T(rho))
    tol = 1e-10
    x, info = G.solve("pressure", solver, T(f), tol=tol, max_it=500, precision="mixed_dd")
    assert info["status"] == "converged" and info["relres_true"] <= tol
    fb = sp.project_range(f, g)
    r64 = fb - N(G.apply("pressure", x))
    assert np.linalg.norm(r64) / np.linalg.norm(fb) <= 1.05 * tol
    A, M = op.pressure_system(rho, g)
    ref = sv.solve(solver, A, M, fb, tol=1e-12, maxit=500)
    assert rel2(N(x), ref.x) < 2.5 * tol


@pytest.mark.parametrize("n,L", [((48, 40, 32), (2 * math.pi,) * 3), ((256,), (2 * math.pi,)), ((512,), (2 * math.pi,)),
                                 ((64, 48), (2 * math.pi, 1.0)), ((256, 16, 16), (2 * math.pi,) * 3),
                                 ((30, 20, 50), (2 * math.pi, 1.0, 3.0)), ((256, 256), (2 * math.pi,) * 2)])
def test_float_pair_residual_accuracy(n, L):
    """The float-pair residual b - A x alone: a warm-started mixed_dd solve with max_it = 0
    evaluates it once at x0 (a converged FP64 solution: the residual is 1e-13..1e-11 |b|, so
    the cancellation is maximal) and reports its norm; the same residual through the double
    operator must agree to the normwise float-pair bound 2^-47 |A| |x0| / |b| with
    |A| = |k|_max^2 max(1/rho).  Measured discrepancies are 0.02-0.3 of that bound; it is
    largest on long 1D lines across a sharp interface (5e-11 of |b| at n = 256, 2.6e-10 at
    512), which is the accuracy floor of the float-pair refinement residual there."""
    g = sp.Grid(n, L)
    rho = inputs.slab_density(g.n, g.L, 5.0, g.ndim - 1, 0.5 * g.L[-1], 0.5 * g.L[-1], 4 * g.L[-1] / g.n[-1])
    f = inputs.smooth_random_field(g.n, g.L, 23, kmax=6)
    G = vd.Grid(n, L)
    G.set_density(T(rho))
    x0, info0 = G.solve("pressure", "cg", T(f), tol=1e-13, max_it=1500)
    assert info0["status"] == "converged"
    _, info = G.solve("pressure", "cg", T(f), x0=x0, tol=0.0, max_it=0, precision="mixed_dd")
    assert info["iters"] == 0
    fb = sp.project_range(f, g)
    r64 = fb - N(G.apply("pressure", x0))
    rel64 = np.linalg.norm(r64) / np.linalg.norm(fb)
    assert rel64 < 1e-10
    kmax2 = sum((math.pi * g.n[j] / g.L[j]) ** 2 for j in range(g.ndim))
    bound = 2.0 ** -47 * kmax2 * float(np.max(1.0 / rho)) * np.linalg.norm(N(x0)) / np.linalg.norm(fb)
    assert abs(info["relres_true"] - rel64) <= bound, (info["relres_true"], rel64, bound)


@pytest.mark.parametrize("max_it", [2, 5, 9, 12, 15, 20])
@pytest.mark.parametrize("precision", ["mixed_dd", "mixed"])
def test_capped_mixed_solve_returns_the_reported_iterate(max_it, precision):
    """With an iteration cap (hit in the first or in a later refinement sweep, or not at all),
    the returned field is the iterate whose true residual is reported -- mixed_dd takes it
    from the last refinement residual's fused inverse transform when that sweep was expected
    to be the last, else from a separate inverse transform: the reported relres_true equals
    the residual recomputed from the returned field with the double operator."""
    n, L = (40, 32, 24), (2 * math.pi, 1.0, 2.0)
    g = sp.Grid(n, L)
    rho = inputs.slab_density(g.n, g.L, 10.0, 1, 0.5 * g.L[1], 0.5 * g.L[1], 3 * g.L[1] / g.n[1])
    f = inputs.smooth_random_field(g.n, g.L, 31, kmax=5)
    G = vd.Grid(n, L)
    G.set_density(T(rho))
    x, info = G.solve("pressure", "cg", T(f), tol=1e-10, max_it=max_it, precision=precision)
    assert info["iters"] <= max_it
    assert info["status"] == ("converged" if info["relres_true"] <= 1e-10 else "max_iter")
    fb = sp.project_range(f, g)
    rel = np.linalg.norm(fb - N(G.apply("pressure", x))) / np.linalg.norm(fb)
    assert abs(info["relres_true"] - rel) <= 1e-9 * rel + 1e-13, (info["relres_true"], rel)
