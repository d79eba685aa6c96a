"""One semi-implicit, second-order fractional time step (oracle; test infrastructure only).

Follows Sec. 2 (Eqs. VDINSE.num.momentum.proj, VDINSE.num.mass.proj, VDINSE.num.proj,
VDINSE.Lrho.num, VDINSE.num.gradp.update) on a fully periodic grid:

1. mass (Crank--Nicolson diffusion, Adams--Bashforth advection), diagonal in Fourier:
   (1 - c Lap) rho^{n+1} = (1 + c Lap) rho^n - dt [u.grad rho]^{n+1/2},  c = dt/(2 Re Sc);
2. rho^{n+1/2} = (rho^{n+1} + rho^n)/2;
3. velocity predictor: V~_{rho^{n+1/2}} u* = u^n + dt(-[u.grad u]^{n+1/2}
   - grad p^{n-1/2}/rho^{n+1/2} + f) + (dt/2) zeta(rho^{n+1/2}, u^n), with a = dt/(2 Re);
   (dt/2) zeta(rho, w) = w - V~_rho w;
4. pressure: L~_{rho^{n+1/2}} phi = div u* / dt;
5. projection: u^{n+1} = u* - dt grad(phi) / rho^{n+1/2};
6. pressure update in the paper's scalar form (Eq. VDINSE.num.p.update), stored as its gradient:
   p^{n+1/2} = p^{n-1/2} + phi - Lap^+ div(rho^{n+1/2} (dt/2) zeta(rho^{n+1/2}, grad phi / rho^{n+1/2})),
   i.e. grad p += grad phi - grad Lap^+ div(c) with c the correction field.  The gradient form
   (Eq. VDINSE.num.gradp.update: grad p += grad phi - c) equals it only up to the solenoidal
   part of c, which the gradient form keeps: with variable density that part is not zero, it
   accumulates O(dt^2) per step into grad p and enters the next predictor, which costs the
   scheme its second order in time when viscosity and density variation are both strong
   (Sec. 4.1 workload: Re = 1, s = 10).  The paper's time study marches the scalar form;
   FlowParams.p_update = "gradient" selects the other one.

Optional source terms (Sec. 4.1 adds a mass source and a body force so that a manufactured
field solves the modified equations): mass_source S and force F, both given at t^{n+1/2},
enter as -dt [u.grad rho - S]^{n+1/2} in step 1 and +dt F in the predictor of step 3.

Readings (the paper is silent on these):
* [.]^{n+1/2} by Adams--Bashforth 2 = 1.5 N^n - 0.5 N^{n-1}; the first step uses N^n
  (Euler) and grad p^{-1/2} = 0;
* body force on a periodic box: the gravity force -Fr^-1 e_g (Sec. 4.2, RTI) cannot be
  balanced by a periodic pressure, so its mean weight is removed:
  f = -Fr^-1 (1 - <rho>/rho) e_g evaluated with rho^{n+1/2};
* the Laplacian in the mass equation is the same discrete sum_j D_j D_j as elsewhere.
"""

from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

from .spectral import Grid, deriv, div, fwd, inv, ksq, precond_pressure
from .operators import RhoDerivs, apply_velocity, pressure_system, velocity_system
from .solvers import solve


@dataclass
class FlowParams:
    Re: float = 1000.0
    Sc: float = 1.0
    Fr: float = 1.0
    gravity_axis: int = -1          # -1: no body force
    vel_solver: str = "rmr"
    pres_solver: str = "gmres"
    tol: float = 1e-10
    maxit: int = 200
    restart: int = 30
    p_update: str = "scalar"        # "scalar" (Eq. VDINSE.num.p.update) or "gradient"


@dataclass
class FlowState:
    rho: np.ndarray
    u: np.ndarray                       # (d, *shape)
    gradp: np.ndarray                   # (d, *shape), grad p^{n-1/2}
    phi: np.ndarray                     # warm start of the pressure increment
    n_rho_prev: np.ndarray | None = None
    n_u_prev: np.ndarray | None = None
    step: int = 0
    log: list = field(default_factory=list)


def advect_scalar(u, s, grid):
    return sum(u[j] * deriv(s, grid, j) for j in range(grid.ndim))


def advect_vector(u, grid):
    return np.stack([advect_scalar(u, u[i], grid) for i in range(grid.ndim)])


def body_force(rho_h, grid, p: FlowParams):
    f = np.zeros((grid.ndim,) + grid.shape)
    if p.gravity_axis >= 0:
        f[p.gravity_axis] = -(1.0 / p.Fr) * (1.0 - rho_h.mean() / rho_h)
    return f


def step(st: FlowState, grid: Grid, dt: float, p: FlowParams, mass_source=None, force=None) -> FlowState:
    d = grid.ndim
    rho, u = st.rho, st.u
    # 1. mass equation
    n_rho = advect_scalar(u, rho, grid)
    ab_rho = n_rho if st.n_rho_prev is None else 1.5 * n_rho - 0.5 * st.n_rho_prev
    if mass_source is not None:
        ab_rho = ab_rho - mass_source
    c = dt / (2.0 * p.Re * p.Sc)
    k2 = ksq(grid)
    rho_new = np.real(inv(((1.0 - c * k2) * fwd(rho) - dt * fwd(ab_rho)) / (1.0 + c * k2)))
    # 2. mid-step density
    rho_h = 0.5 * (rho_new + rho)
    # 3. velocity predictor
    a = dt / (2.0 * p.Re)
    inv_sc = 1.0 / p.Sc
    n_u = advect_vector(u, grid)
    ab_u = n_u if st.n_u_prev is None else 1.5 * n_u - 0.5 * st.n_u_prev
    rd = RhoDerivs(rho_h, grid)
    half_zeta_u = u - apply_velocity(rho_h, u, grid, a, inv_sc, rd)
    f_body = body_force(rho_h, grid, p)
    if force is not None:
        f_body = f_body + force
    rhs = u + dt * (-ab_u - st.gradp / rho_h + f_body) + half_zeta_u
    Av, Mv = velocity_system(rho_h, grid, a, inv_sc)
    rv = solve(p.vel_solver, Av, Mv, rhs, x0=u, tol=p.tol, maxit=p.maxit, restart=p.restart)
    u_star = rv.x
    # 4. pressure increment
    f = div(list(u_star), grid) / dt
    Ap, Mp = pressure_system(rho_h, grid)
    rp = solve(p.pres_solver, Ap, Mp, f, x0=st.phi, tol=p.tol, maxit=p.maxit, restart=p.restart)
    phi = rp.x
    # 5. projection
    gphi = np.stack([deriv(phi, grid, j) for j in range(d)])
    u_new = u_star - dt * gphi / rho_h
    # 6. pressure update: correction c = rho_h (dt/2) zeta(rho_h, grad phi / rho_h)
    w = gphi / rho_h
    half_zeta_w = w - apply_velocity(rho_h, w, grid, a, inv_sc, rd)
    corr = rho_h * half_zeta_w
    if p.p_update == "scalar":
        q = precond_pressure(div(list(corr), grid), grid)          # Lap^+ div c
        corr = np.stack([deriv(q, grid, j) for j in range(d)])     # its gradient
    elif p.p_update != "gradient":
        raise ValueError(p.p_update)
    gradp_new = st.gradp + gphi - corr
    log = {"vel_iters": rv.iters, "vel_status": rv.status, "vel_relres": rv.relres_true,
           "pres_iters": rp.iters, "pres_status": rp.status, "pres_relres": rp.relres_true}
    return FlowState(rho=rho_new, u=u_new, gradp=gradp_new, phi=phi, n_rho_prev=n_rho,
                     n_u_prev=n_u, step=st.step + 1, log=st.log + [log])


def projection(rho: np.ndarray, w: np.ndarray, grid: Grid, kind: str = "cg", tol: float = 1e-12,
               maxit: int = 500) -> np.ndarray:
    """P_rho(w) = w - rho^-1 grad L~_rho^-1 div w (the exact projector of Sec. 2, after
    Eq. VDINSE.num.p.update)."""
    A, M = pressure_system(rho, grid)
    res = solve(kind, A, M, div(list(w), grid), tol=tol, maxit=maxit)
    return w - np.stack([deriv(res.x, grid, j) for j in range(grid.ndim)]) / rho
