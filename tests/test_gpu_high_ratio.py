"""Mixed-precision solves at high density ratios, against the FP64 oracle.

The batched and serving workloads draw density ratios up to 50.  Above a ratio of 10 the
inner float operator multiplies by 1/rho in float-pair arithmetic (vd_solve_params.coef_pair
= 0, automatic); the refinement keeps the true residual in double (mixed) or float pairs
(mixed_dd).  Each solve must reach the 1e-10 relative residual, checked here with the
oracle's own FP64 operator (for mixed_dd within the normwise error of its float-pair
residual), and its solution must agree with the oracle's FP64 solution to kappa * tol with
kappa <= rho_max / rho_min (the eigenvalue bound of the preconditioned operator).  Grids reach the register four-step
float kernels (y length 128/256, x half-length 64/128) and the Stockham engine (z 16).

Also here: the part of a pressure right-hand side outside the range (its null-space modes)
is removed before the solve and reported (reading c4), and range_tol > 0 refuses a
right-hand side whose removed part is too large.
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

GRIDS = [((128, 128, 16), (2 * math.pi,) * 3), ((256, 256), (2 * math.pi, 2 * math.pi))]


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def N(t):
    return t.detach().cpu().numpy()


def rel2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _case(n, L, s, seed):
    g = sp.Grid(n, L)
    axis = len(n) - 1 if len(n) == 2 else 1
    rho = inputs.slab_density(g.n, g.L, s, axis, 1.3, math.pi, 3 * L[axis] / n[axis])
    f = inputs.smooth_random_field(g.n, g.L, seed, kmax=5)
    return g, rho, f


@pytest.mark.parametrize("n,L", GRIDS)
@pytest.mark.parametrize("s", [20.0, 50.0])
@pytest.mark.parametrize("precision", ["mixed", "mixed_dd"])
def test_mixed_high_ratio_matches_oracle(n, L, s, precision):
    g, rho, f = _case(n, L, s, 31)
    A, M = op.pressure_system(rho, g)
    fp = sp.project_range(f, g)
    ref = sv.cg(A, M, fp, tol=1e-13, maxit=2000)
    assert ref.status == "converged"
    G = vd.Grid(n, L)
    G.set_density(T(rho))
    x, info = G.solve("pressure", "cg", T(f), tol=1e-10, max_it=2000, precision=precision)
    assert info["status"] == "converged" and info["coef_pair"], info
    xs = N(x)
    # true residual with the oracle's FP64 operator
    r = np.linalg.norm(fp - A(xs)) / np.linalg.norm(fp)
    assert info["relres_true"] <= 1e-10
    if precision == "mixed":
        # the refinement residual is formed in double
        assert r <= 1.05e-10, r
    else:
        # mixed_dd certifies its residual in float-pair arithmetic: it may differ from the
        # double one by up to the normwise float-pair scale 2^-47 |A| |x| / |b| with
        # |A| = |k|_max^2 max(1/rho) (a few 1e-12 measured here at s = 50)
        kmax2 = sum((math.pi * g.n[j] / g.L[j]) ** 2 for j in range(g.ndim))
        bound = 2.0 ** -47 * kmax2 * float(np.max(1.0 / rho)) * np.linalg.norm(xs) / np.linalg.norm(fp)
        assert abs(r - info["relres_true"]) <= bound, (r, info["relres_true"], bound)
        assert r <= 1e-10 + bound, (r, bound)
    assert rel2(xs, ref.x) <= s * 1e-10, rel2(xs, ref.x)


@pytest.mark.parametrize("precision", ["mixed", "mixed_dd"])
def test_coef_pair_switch(precision):
    """The switch follows the density ratio (automatic), or the caller (forced on / off); the
    plain-float multiply still converges to the same solution within the parity bound."""
    n, L = GRIDS[0]
    G = vd.Grid(n, L)
    _, rho, f = _case(n, L, 5.0, 32)
    G.set_density(T(rho))
    _, info = G.solve("pressure", "cg", T(f), tol=1e-10, max_it=2000, precision=precision)
    assert info["status"] == "converged" and not info["coef_pair"]
    _, rho, f = _case(n, L, 50.0, 33)
    G.set_density(T(rho))
    x_auto, ia = G.solve("pressure", "cg", T(f), tol=1e-10, max_it=2000, precision=precision)
    x_off, io = G.solve("pressure", "cg", T(f), tol=1e-10, max_it=2000, precision=precision, coef_pair=-1)
    x_on, i1 = G.solve("pressure", "cg", T(f), tol=1e-10, max_it=2000, precision=precision, coef_pair=1)
    assert ia["coef_pair"] and i1["coef_pair"] and not io["coef_pair"]
    assert torch.equal(x_auto, x_on)
    assert io["status"] == "converged" and io["relres_true"] <= 1e-10
    assert rel2(N(x_off), N(x_on)) <= 2 * 50 * 1e-10


def test_rhs_range_report_and_refusal():
    n, L = (48, 40, 32), (2 * math.pi,) * 3
    g = sp.Grid(n, L)
    rho = inputs.slab_density(g.n, g.L, 4.0, 1, math.pi, 2.0, 0.3)
    f = inputs.smooth_random_field(g.n, g.L, 16, kmax=5)
    f = f - f.mean()
    # add a constant and a Nyquist-corner mode (both in the null space of L~)
    z = np.arange(n[2])[:, None, None]
    y = np.arange(n[1])[None, :, None]
    x = np.arange(n[0])[None, None, :]
    nyq = 0.3 * np.cos(np.pi * x) * np.cos(np.pi * y) * np.cos(np.pi * z)
    b = f + 0.5 + nyq
    expect = np.linalg.norm(b - sp.project_range(b, g)) / np.linalg.norm(b)
    assert expect > 0.01
    G = vd.Grid(n, L)
    G.set_density(T(rho))
    xa, info = G.solve("pressure", "cg", T(b), tol=1e-10, max_it=500)
    assert info["status"] == "converged"
    assert abs(info["rhs_removed"] - expect) <= 1e-12 * max(1.0, expect)
    # the solution is that of the projected right-hand side
    xb, _ = G.solve("pressure", "cg", T(f), tol=1e-10, max_it=500)
    assert rel2(N(xa), N(xb)) < 1e-12
    # a right-hand side in the range reports (almost) nothing removed
    assert info["rhs_removed"] > 0 and _["rhs_removed"] < 1e-14
    with pytest.raises(vd.VDError) as e:
        G.solve("pressure", "cg", T(b), tol=1e-10, max_it=500, range_tol=0.5 * expect)
    assert e.value.status == vd.VD_ERR_RHS_NOT_IN_RANGE
    x2, i2 = G.solve("pressure", "cg", T(b), tol=1e-10, max_it=500, range_tol=2.0 * expect)
    assert i2["status"] == "converged" and torch.equal(x2, xa)
