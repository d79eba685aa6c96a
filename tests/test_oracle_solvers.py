"""Pins of the oracle's Krylov solvers (CPU only).

* exact 1D solution (non-iterative direct solve) vs CG / GMRES(30) / RMR on the 1D
  top-hat workload (r = 3, d = 0.05, N = 256, 16 random modes);
* the direct solve itself against a closed form (trigonometric-polynomial 1/rho);
* one-iteration convergence when rho is constant: the preconditioner is then the exact
  inverse on the range (Sec. 4.2: the inverse Laplacian "is the inverse of the operator
  with constant density");
* GMRES finite termination on a tiny grid, CG's kappa-based iteration bound, and the
  invariance of all three solvers to scaling the preconditioner.
"""

import math

import numpy as np
import pytest

from oracle import spectral as sp
from oracle import operators as op
from oracle import solvers as sv
from oracle.direct1d import solve_pressure_1d
from paper_2403_06654_gb300 import inputs


def config1(n=256):
    g = sp.Grid((n,), (2 * math.pi,))
    rho = inputs.tophat_1d(n=n)
    f = inputs.modes_rhs_1d(n=n)
    return g, rho, f


def test_direct1d_closed_form():
    n = 64
    g = sp.Grid((n,), (2 * math.pi,))
    x = 2 * math.pi * np.arange(n) / n
    a = 1.0 + 0.5 * np.sin(x)                 # 1/rho
    p = np.sin(2 * x) + 0.3 * np.cos(3 * x)
    dp = 2 * np.cos(2 * x) - 0.9 * np.sin(3 * x)
    d2p = -4 * np.sin(2 * x) - 2.7 * np.cos(3 * x)
    f = 0.5 * np.cos(x) * dp + a * d2p       # (a p')'
    out = solve_pressure_1d(1.0 / a, f, g)
    assert np.max(np.abs(out - p)) < 1e-13


def test_direct1d_residual_config1():
    g, rho, f = config1()
    p = solve_pressure_1d(rho, f, g)
    r = f - op.apply_pressure(rho, p, g)
    # rounding floor: eps * ||L~|| ||p|| / ||f|| with ||L~|| ~ (n/2)^2 / rho_min ~ 1.6e4
    assert np.linalg.norm(r) < 5e-12 * np.linalg.norm(f)
    assert abs(p.mean()) < 1e-14 and abs(np.sum(p * (-1.0) ** np.arange(g.n[0]))) < 1e-12


@pytest.mark.parametrize("kind", ["cg", "gmres", "rmr"])
def test_config1_solvers_match_direct(kind):
    g, rho, f = config1()
    A, M = op.pressure_system(rho, g)
    p = solve_pressure_1d(rho, f, g)
    res = sv.solve(kind, A, M, f, tol=1e-12, maxit=400, restart=30)
    assert res.status == "converged"
    assert res.relres_true < 5e-12
    assert np.linalg.norm(res.x - p) < 1e-11 * np.linalg.norm(p)


def test_config1_iteration_counts_and_cg_bound():
    """kappa <= rho_max/rho_min = 3; PCG error in the energy norm contracts at least by
    (sqrt(k)-1)/(sqrt(k)+1) per iteration, so 1e-12 needs at most ~ 30 iterations (plus a
    sqrt(kappa) factor between the energy norm and the residual norm)."""
    g, rho, f = config1()
    A, M = op.pressure_system(rho, g)
    kappa = rho.max() / rho.min()
    q = (math.sqrt(kappa) - 1) / (math.sqrt(kappa) + 1)
    bound = math.ceil(math.log(1e-12 / (2 * kappa)) / math.log(q))
    its = {k: sv.solve(k, A, M, f, tol=1e-12, maxit=400).iters for k in ("cg", "gmres", "rmr")}
    assert its["cg"] <= bound
    assert its["gmres"] <= its["cg"] + 1          # GMRES minimises the residual norm
    assert its["rmr"] >= its["gmres"]


@pytest.mark.parametrize("kind", ["cg", "gmres", "rmr"])
@pytest.mark.parametrize("n,L", [((32,), (2 * math.pi,)), ((16, 12), (1.0, 2.0)), ((8, 6, 10), (2 * math.pi,) * 3)])
def test_constant_density_one_iteration_pressure(kind, n, L):
    g = sp.Grid(n, L)
    rho = np.full(g.shape, 2.5)
    f = sp.project_range(inputs.random_field(g.shape, 5), g)
    A, M = op.pressure_system(rho, g)
    res = sv.solve(kind, A, M, f, tol=1e-12, maxit=10)
    assert res.status == "converged" and res.iters == 1
    assert res.relres_true < 1e-12


@pytest.mark.parametrize("kind", ["gmres", "rmr"])
def test_constant_density_one_iteration_velocity(kind):
    g = sp.Grid((8, 6, 10), (2 * math.pi, 1.0, 3.0))
    rho = np.full(g.shape, 1.3)
    a = 0.05 * 1.3
    b = inputs.random_field((3,) + g.shape, 6)
    # with constant rho and a' = a/rho, V~ = I - a' Lap, preconditioned by (I - a' Lap)^-1
    A, _ = op.velocity_system(rho, g, a, 0.5)
    M = lambda v: op.precond_velocity_vec(v, g, a / 1.3)  # noqa: E731
    res = sv.solve(kind, A, M, b, tol=1e-12, maxit=10)
    assert res.status == "converged" and res.iters == 1


def test_gmres_finite_termination():
    n = 16
    g = sp.Grid((n,), (2 * math.pi,))
    x = 2 * math.pi * np.arange(n) / n
    rho = 1.0 + 4.0 * np.exp(-((x - 3.0) ** 2))
    f = sp.project_range(inputs.random_field(g.shape, 8), g)
    A, M = op.pressure_system(rho, g)
    res = sv.gmres(A, M, f, tol=1e-12, maxit=n, restart=n)
    assert res.status == "converged" and res.iters <= n - 2


@pytest.mark.parametrize("kind", ["cg", "gmres", "rmr"])
def test_preconditioner_scaling_invariance(kind):
    g = sp.Grid((24, 16), (2 * math.pi, 2 * math.pi))
    rho = inputs.slab_density(g.n, g.L, 5.0, 1, 2.0, 2.0, 0.3)
    f = sp.project_range(inputs.random_field(g.shape, 9), g)
    A, M = op.pressure_system(rho, g)
    r1 = sv.solve(kind, A, M, f, tol=0.0, maxit=6)
    r2 = sv.solve(kind, A, lambda v: 7.0 * M(v), f, tol=0.0, maxit=6)
    assert np.linalg.norm(r1.x - r2.x) < 1e-12 * np.linalg.norm(r1.x)


def test_rmr_step_is_minimal_residual():
    g = sp.Grid((32,), (2 * math.pi,))
    rho = inputs.tophat_1d(n=32, d=0.3)
    f = sp.project_range(inputs.random_field(g.shape, 10), g)
    A, M = op.pressure_system(rho, g)
    z = M(f)
    w = A(z)
    alpha = np.dot(f, w) / np.dot(w, w)
    base = np.linalg.norm(f - alpha * w)
    for da in (1e-3, -1e-3):
        assert np.linalg.norm(f - (alpha + da) * w) > base
    res = sv.rmr(A, M, f, tol=0.0, maxit=1)
    assert np.linalg.norm(f - A(res.x)) == pytest.approx(base, rel=1e-12)


@pytest.mark.parametrize("kind", ["gmres", "rmr"])
def test_velocity_solvers_agree_2d(kind):
    g = sp.Grid((32, 24), (2 * math.pi, 2 * math.pi))
    rho = inputs.slab_density(g.n, g.L, 3.0, 0, 3.0, 3.0, 0.4)
    b = inputs.random_field((2,) + g.shape, 12)
    A, M = op.velocity_system(rho, g, 1e-2, 1.0)
    ref = sv.gmres(A, M, b, tol=1e-13, maxit=300, restart=60)
    res = sv.solve(kind, A, M, b, tol=1e-12, maxit=300)
    assert res.status == "converged"
    assert np.linalg.norm(res.x - ref.x) < 1e-10 * np.linalg.norm(ref.x)


def test_warm_start_exact_solution_zero_iterations():
    g, rho, f = config1(64)
    A, M = op.pressure_system(rho, g)
    p = solve_pressure_1d(rho, f, g)
    res = sv.cg(A, M, f, x0=p, tol=1e-10)
    assert res.iters == 0 and res.status == "converged"


def test_cg_sign_of_preconditioner_is_irrelevant():
    """Solving with (A, M) or (A, -M): the PCG iterates agree (scaling by c = -1), which is
    why CG may run on the negative semi-definite pair (L~, Lap^+) directly."""
    g, rho, f = config1(64)
    A, M = op.pressure_system(rho, g)
    r1 = sv.cg(A, M, f, tol=0.0, maxit=8)
    r2 = sv.cg(A, lambda v: -M(v), f, tol=0.0, maxit=8)
    assert np.linalg.norm(r1.x - r2.x) < 1e-12 * np.linalg.norm(r1.x)


def test_planted_mistake_unpreconditioned_is_slow():
    """Without the constant-density preconditioner the same solve needs far more iterations."""
    g, rho, f = config1(64)
    A, M = op.pressure_system(rho, g)
    fast = sv.cg(A, M, f, tol=1e-8, maxit=400)
    slow = sv.cg(A, lambda v: -v, f, tol=1e-8, maxit=400)
    assert fast.status == "converged"
    assert slow.iters > 3 * fast.iters
