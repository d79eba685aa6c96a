"""Parity of the CUDA K_rho form (Sec. 4.2, Eq. VDINSE.Krho) with the FP64 oracle.

Applies and preconditioner applies are compared element by element (relative max norm
1e-11: the coefficient c = -Lap(w)/w goes through one more transform pair than the pressure
operator's 1/rho); solutions solved to 1e-12 on both sides agree to 1e-10 in relative
2-norm; the mixed-precision modes reach the same 1e-10 true residual and stay within
1e-8 of the FP64 oracle solution.  Grids span several tiles with ragged tails and radix
2, 3 and 5 lengths.
"""

import math

import numpy as np
import pytest
import torch

import paper_2403_06654_gb300 as vd
from paper_2403_06654_gb300 import inputs
from oracle import krho
from oracle import solvers as sv
from oracle import spectral as sp

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
    ((32, 128, 16), (2 * math.pi, 2 * math.pi, 1.0)),    # y pass on the register kernel (float)
    ((16, 24, 256), (1.0, 2 * math.pi, 2 * math.pi)),    # z pass on the register kernel (float)
]


def smooth_density(g, s=4.0, seed=0):
    f = inputs.smooth_random_field(g.n, g.L, seed, kmax=3)
    f = (f - f.min()) / (f.max() - f.min())
    return 1.0 + (s - 1.0) * f


def setup(n, L, s=4.0):
    g = sp.Grid(n, L)
    G = vd.Grid(n, L)
    rho = smooth_density(g, s)
    G.set_density(T(rho), op="krho")
    return g, G, rho


@pytest.mark.parametrize("n,L", GRIDS)
def test_apply(n, L):
    g, G, rho = setup(n, L)
    Phi = inputs.random_field(g.shape, 5)
    assert relmax(N(G.apply("krho", T(Phi))), krho.apply_krho(rho, Phi, g)) < 1e-11
    # smooth input: the coefficient term is not drowned by the Laplacian
    Phi = inputs.smooth_random_field(n, L, 6, kmax=4)
    assert relmax(N(G.apply("krho", T(Phi))), krho.apply_krho(rho, Phi, g)) < 1e-11


@pytest.mark.parametrize("n,L", GRIDS)
def test_precond(n, L):
    g, G, _ = setup(n, L)
    r = inputs.random_field(g.shape, 7)
    assert relmax(N(G.precond("krho", T(r))), krho.precond_krho(r, g)) < 1e-12


@pytest.mark.parametrize("n,L", GRIDS[::2])
def test_null_vector(n, L):
    g, G, rho = setup(n, L, s=8.0)
    w = krho.null_vector(rho)
    Kw = N(G.apply("krho", T(w)))
    assert np.max(np.abs(Kw)) <= 1e-11 * np.max(krho.ksq_full(g)) * np.max(np.abs(w))


@pytest.mark.parametrize("solver", ["gmres", "rmr", "cg"])
@pytest.mark.parametrize("n,L", [GRIDS[2], GRIDS[5], GRIDS[6]])
def test_solve_fp64(n, L, solver):
    g, G, rho = setup(n, L)
    f = inputs.smooth_random_field(n, L, 8, kmax=5)
    rhs = np.sqrt(rho) * f
    if solver == "rmr":
        # RMR converges slowly on the anisotropic boxes: compare the iterates after 40 steps
        ref = sv.solve(solver, *krho.krho_system(rho, g), krho.project_rhs(rhs, rho), tol=0.0, maxit=40)
        x, info = G.solve("krho", solver, T(rhs), tol=0.0, max_it=40)
        assert info["iters"] == ref.iters == 40
        assert rel2(N(x), ref.x) < 1e-10
        return
    ref = sv.solve(solver, *krho.krho_system(rho, g), krho.project_rhs(rhs, rho), tol=1e-12, maxit=400)
    assert ref.status == "converged"
    x, info = G.solve("krho", solver, T(rhs), tol=1e-12, max_it=400)
    assert info["status"] == "converged" and info["relres_true"] < 1e-11
    assert abs(float(N(x).mean())) < 1e-12 * float(np.max(np.abs(N(x))))
    assert rel2(N(x), ref.x) < 1e-10


@pytest.mark.parametrize("precision", ["mixed", "mixed_dd"])
@pytest.mark.parametrize("n,L", [GRIDS[3], GRIDS[5], GRIDS[7], GRIDS[8], GRIDS[9]])
def test_solve_mixed(n, L, precision):
    g, G, rho = setup(n, L)
    f = inputs.smooth_random_field(n, L, 9, kmax=5)
    rhs = np.sqrt(rho) * f
    ref = sv.solve("gmres", *krho.krho_system(rho, g), krho.project_rhs(rhs, rho), tol=1e-13, maxit=400)
    x, info = G.solve("krho", "gmres", T(rhs), tol=1e-10, max_it=400, precision=precision)
    assert info["status"] == "converged" and info["relres_true"] <= 1e-10
    assert rel2(N(x), ref.x) < 1e-8


@pytest.mark.parametrize("solver", ["cg", "gmres", "rmr"])
def test_constant_density_one_iteration(solver):
    n, L = (24, 20, 16), (2 * math.pi,) * 3
    G = vd.Grid(n, L)
    G.set_density(torch.full(tuple(reversed(n)), 3.0, dtype=torch.float64, device=DEV), op="krho")
    b = T(inputs.random_field(tuple(reversed(n)), 10))
    _, info = G.solve("krho", solver, b, tol=1e-12, max_it=10)
    assert info["status"] == "converged" and info["iters"] == 1


def test_pressure_operator_still_available():
    """A density set for K_rho also serves the pressure operator."""
    n, L = (32, 24, 16), (2 * math.pi,) * 3
    g, G, rho = setup(n, L)
    from oracle import operators as op
    phi = inputs.random_field(g.shape, 11)
    assert relmax(N(G.apply("pressure", T(phi))), op.apply_pressure(rho, phi, g)) < 1e-12
