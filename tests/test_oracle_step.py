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


# --------------------------------------------------------------------------------------
# Second order in time on the manufactured solution of Sec. 4.1 (Re = 1, Sc = 1, s = 10,
# T = pi/4), with its mass source and body force added to the equations.
# --------------------------------------------------------------------------------------

def _tg_errors(n_steps, p_update, n=16, s=10.0, Re=1.0, Sc=1.0, T=math.pi / 4):
    import manufactured as mf
    from oracle import step as ost
    g = mf.grid(n)
    dt = T / n_steps
    rho0, u0, _, _, _ = mf.exact(g, 0.0, s)
    p = ost.FlowParams(Re=Re, Sc=Sc, Fr=1.0, gravity_axis=-1, vel_solver="gmres", pres_solver="cg", tol=1e-12,
                       maxit=400, restart=30, p_update=p_update)
    st = ost.FlowState(rho=rho0.copy(), u=u0.copy(), gradp=np.zeros_like(u0), phi=np.zeros(g.shape))
    for k in range(n_steps):
        S, F = mf.sources(g, (k + 0.5) * dt, s, Re, Sc)
        st = ost.step(st, g, dt, p, mass_source=S, force=F)
    rhoe, ue, _, _, _ = mf.exact(g, T, s)
    return np.array([mf.rms(st.u - ue), mf.rms(st.rho - rhoe), mf.rms(st.gradp - mf.grad_p(g, T - 0.5 * dt, s))])


def test_second_order_in_time_manufactured():
    """Errors of u, rho and grad p (at T - dt/2, where the stored gradient lives) fall by 4x per
    halving of dt (observed orders >= 1.9 at dt = T/8 -> T/16 -> T/32); the grid (16^3) is fine
    enough that the spatial error is far below these (24^3 gives the same errors to 4 digits)."""
    e = [_tg_errors(k, "scalar") for k in (8, 16, 32)]
    for a, b in zip(e, e[1:]):
        order = np.log2(a / b)
        assert np.all(order >= 1.9), order


def test_gradient_form_update_loses_second_order():
    """The gradient form of the pressure update keeps the solenoidal part of its correction;
    at Re = 1 and s = 10 that part accumulates and the pressure-gradient error falls far
    slower than 4x per halving of dt (the scalar form above does not)."""
    e16, e32 = _tg_errors(16, "gradient"), _tg_errors(32, "gradient")
    assert np.log2(e16[2] / e32[2]) < 1.5
    s32 = _tg_errors(32, "scalar")
    assert e32[2] > 3 * s32[2]


# --------------------------------------------------------------------------------------
# Body force (gravity).  The RTI case of Sec. 4.2 adds -Fr^-1 e_z; on a periodic box the
# oracle removes its mean weight (the force becomes -Fr^-1 (1 - <rho>/rho) e_z) so that a
# periodic hydrostatic pressure exists.  Two consequences that do not depend on how the force
# is written pin it:
#  (i)  a density that varies only along gravity is in hydrostatic balance: from rest, the
#       velocity stays zero (to the solve tolerance) step after step.  With the full weight
#       -Fr^-1 e_z no periodic pressure balances the force and the whole box accelerates by
#       dt/Fr per step;
#  (ii) the heavy fluid sinks along gravity (Sec. 4.2: the RTI mushroom grows downward, the
#       heavier fluid penetrating the lighter one): after one step from rest the density-
#       weighted vertical velocity sum_x (rho - <rho>) u_z is negative.  A force of the wrong
#       sign makes the heavy fluid rise.
# --------------------------------------------------------------------------------------

def _stratified(nx=16, nz=32):
    """Horizontally uniform density rho(z) = 1.5 + 0.5 cos(pi z) (ratio 2) on a 1 x 2 box,
    gravity along z.  Smooth on purpose: the Nyquist row of the force (k~ = 0 there, reading
    c1) is not a gradient and is not balanced; here it is below 1e-12 of the force."""
    g = sp.Grid((nx, nz), (1.0, 2.0))
    z = (np.arange(nz) * 2.0 / nz)[:, None]
    rho = 1.5 + 0.5 * np.cos(np.pi * z)
    return g, np.array(np.broadcast_to(rho, (nz, nx)), copy=True)


def _hydrostatic_speed(steps=3, dt=1e-3, Fr=1.0):
    g, rho = _stratified()
    p = st.FlowParams(Re=1000.0, Sc=1.0, Fr=Fr, gravity_axis=1, vel_solver="gmres", pres_solver="cg", tol=1e-12,
                      maxit=300)
    s = st.FlowState(rho=rho, u=np.zeros((2,) + g.shape), gradp=np.zeros((2,) + g.shape), phi=np.zeros(g.shape))
    top = 0.0
    for _ in range(steps):
        s = st.step(s, g, dt, p)
        top = max(top, float(np.max(np.abs(s.u))))
    return top / (dt / Fr)


def _buoyancy_flux_one_step(dt=1e-3):
    # the RT-like layer with a large interface perturbation (eta amplitude 0.5), so that a good
    # part of the force is not balanced by pressure and drives motion at once
    case = inputs.rt_2d(nx=32, nz=64, delta=0.08, s=3.0, eta_amp=0.5)
    g = sp.Grid(case.n, case.L)
    p = st.FlowParams(Re=case.Re, Sc=case.Sc, Fr=case.Fr, gravity_axis=case.gravity_axis, vel_solver="gmres",
                      pres_solver="cg", tol=1e-12, maxit=300)
    s = st.FlowState(rho=case.rho.copy(), u=np.zeros_like(case.u), gradp=np.zeros_like(case.u),
                     phi=np.zeros(g.shape))
    s1 = st.step(s, g, dt, p)
    w = s1.u[case.gravity_axis]
    flux = float(np.sum((case.rho - case.rho.mean()) * w))
    return flux / float(np.sum(np.abs(case.rho - case.rho.mean()) * np.abs(w)))


def test_body_force_hydrostatic_rest():
    assert _hydrostatic_speed() < 1e-8


def test_body_force_heavy_fluid_sinks():
    # normalised flux: -1 if every heavy parcel moves along gravity and every light one against
    assert _buoyancy_flux_one_step() < -0.1


def test_body_force_pins_catch_planted_mistakes(monkeypatch):
    """Planted in the oracle: the full weight (mean not removed) fails pin (i); the wrong
    sign fails pin (ii)."""
    real = st.body_force

    def full_weight(rho_h, grid, p):
        f = np.zeros((grid.ndim,) + grid.shape)
        if p.gravity_axis >= 0:
            f[p.gravity_axis] = -(1.0 / p.Fr)
        return f

    monkeypatch.setattr(st, "body_force", full_weight)
    assert _hydrostatic_speed() > 0.5
    monkeypatch.setattr(st, "body_force", lambda rho_h, grid, p: -real(rho_h, grid, p))
    assert _hydrostatic_speed() < 1e-8
    assert _buoyancy_flux_one_step() > 0.1
