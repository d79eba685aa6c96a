"""Invariants of the oracle's semi-implicit step (CPU only).

Sec. 2 states that P_rho is an exact projector (P_rho(v) = v for divergence-free v and
P_rho o P_rho = P_rho) and Sec. 4.1 that the divergence of the projected velocity and the
drift of the total mass stay at rounding level.  Discretely: div u^{n+1} = dt (f - L~ phi),
so its norm relative to ||div u*|| is the pressure solve's relative residual; and
sum_x u.D rho = -sum_x rho D.u because D is skew-symmetric, so the mass drift vanishes with
div u^n.
"""

import math

import numpy as np
import pytest

from oracle import spectral as sp
from oracle import step as st
from paper_2403_06654_gb300 import inputs


def small_rt(nx=32, nz=64):
    case = inputs.rt_2d(nx=nx, nz=nz, delta=0.08, s=3.0)
    g = sp.Grid(case.n, case.L)
    return case, g


def test_projection_is_exact_projector():
    case, g = small_rt()
    rho = case.rho
    w = inputs.random_field((2,) + g.shape, 21)
    pw = st.projection(rho, w, g)
    ppw = st.projection(rho, pw, g)
    assert np.linalg.norm(ppw - pw) < 1e-10 * np.linalg.norm(pw)
    assert np.linalg.norm(sp.div(list(pw), g)) < 1e-9 * np.linalg.norm(sp.div(list(w), g))
    # a discretely divergence-free field (D_1 psi, -D_0 psi) is left unchanged
    psi = inputs.random_field(g.shape, 22)
    v = np.stack([sp.deriv(psi, g, 1), -sp.deriv(psi, g, 0)])
    assert np.linalg.norm(st.projection(rho, v, g) - v) < 1e-12 * np.linalg.norm(v)


@pytest.mark.parametrize("vel,pres", [("rmr", "gmres"), ("gmres", "cg")])
def test_steps_divergence_and_mass(vel, pres):
    case, g = small_rt()
    p = st.FlowParams(Re=case.Re, Sc=case.Sc, Fr=case.Fr, gravity_axis=case.gravity_axis,
                      vel_solver=vel, pres_solver=pres, tol=1e-10, maxit=200)
    s = st.FlowState(rho=case.rho.copy(), u=case.u.copy(), gradp=np.zeros_like(case.u),
                     phi=np.zeros(g.shape))
    masses = [s.rho.mean()]
    for _ in range(4):
        s = st.step(s, g, case.dt, p)
        masses.append(s.rho.mean())
        lg = s.log[-1]
        assert lg["vel_status"] == "converged" and lg["pres_status"] == "converged"
        assert lg["pres_relres"] < 1e-9
        divu = np.linalg.norm(sp.div(list(s.u), g))
        assert divu < 1e-6 * np.linalg.norm(s.u)
    # u^0 is not divergence-free and enters steps 1 and 2 (Adams--Bashforth history);
    # from step 3 on the drift is at rounding level
    for m0, m1 in zip(masses[2:], masses[3:]):
        assert abs(m1 - m0) < 1e-12
    # warm-started velocity solves need few iterations (Sec. 3.1: 3 to 5)
    assert s.log[-1]["vel_iters"] <= 8


def test_first_step_reproducible():
    case, g = small_rt(16, 32)
    p = st.FlowParams(Re=case.Re, gravity_axis=1)
    s0 = st.FlowState(rho=case.rho.copy(), u=case.u.copy(), gradp=np.zeros_like(case.u),
                      phi=np.zeros(g.shape))
    a = st.step(s0, g, case.dt, p)
    b = st.step(s0, g, case.dt, p)
    assert np.array_equal(a.u, b.u) and np.array_equal(a.rho, b.rho)
