"""Pins of the oracle's K_rho form (Sec. 4.2, Eq. VDINSE.Krho) against closed forms (CPU only).

* Closed form: with w = rho^-1/2 a trigonometric polynomial, Lap w is exact on the grid, so
  c = -Lap w / w and K Phi = Lap Phi + c Phi are known pointwise for a band-limited Phi,
  including a Nyquist mode (which pins the full-wavenumber Laplacian).
* The coefficient equals the paper's printed one, Lap rho/(2 rho) - 3|grad rho|^2/(4 rho^2),
  up to a discretisation error that decays spectrally with n.
* sqrt(rho) L_rho(phi) and K_rho(phi / sqrt(rho)) agree up to a spectrally small error
  (the substitution that defines the form).
* Dense assembly: symmetric, one-dimensional null space spanned by rho^-1/2.
* Constant density: the preconditioned operator is the identity on zero-mean fields, so
  every solver converges in one iteration.
"""

import math

import numpy as np
import pytest

from oracle import dense
from oracle import krho
from oracle import operators as op
from oracle import solvers
from oracle import spectral as sp


def box(n):
    return sp.Grid(tuple(n), (2 * math.pi,) * len(n))


@pytest.mark.parametrize("n", [(16, 12), (12, 10, 8)])
def test_apply_closed_form(n):
    g = box(n)
    X = g.coords()
    eps = 0.3
    prod = np.ones(g.shape)
    for j in range(g.ndim):
        prod = prod * np.sin(X[j])
    w = 1.0 + eps * prod
    rho = w ** -2
    d = g.ndim
    # Lap w = -d eps prod  =>  c = -Lap w / w = d eps prod / w
    c_exact = d * eps * prod / w
    nyq = n[0] // 2
    full = np.zeros(g.shape)
    Phi = full + np.cos(2 * X[0]) + 0.5 * np.sin(3 * X[1]) + 0.25 * np.cos(nyq * X[0])
    lap_Phi = full - 4 * np.cos(2 * X[0]) - 4.5 * np.sin(3 * X[1]) - 0.25 * nyq ** 2 * np.cos(nyq * X[0])
    np.testing.assert_allclose(krho.coeff(rho, g), c_exact, rtol=0, atol=1e-13)
    got = krho.apply_krho(rho, Phi, g)
    want = lap_Phi + c_exact * Phi
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def test_full_wavenumber_laplacian_keeps_nyquist():
    g = box((8,))
    x = g.coords()[0]
    f = np.cos(4 * x)                     # the Nyquist mode of an 8-point grid
    np.testing.assert_allclose(krho.lap_full(f, g), -16 * f, atol=1e-12)
    # its pseudo-inverse removes the mean only
    h = 1.0 + np.cos(4 * x) + np.sin(x)
    np.testing.assert_allclose(krho.lap_full(krho.precond_krho(h, g), g), h - h.mean(), atol=1e-12)


def test_coefficient_matches_paper_formula_spectrally():
    errs = []
    for m in (16, 32, 64):
        g = box((m, m))
        x, y = g.coords()
        rho = 1.0 + 0.4 * np.sin(x) * np.cos(y)
        errs.append(np.max(np.abs(krho.coeff(rho, g) - krho.coeff_paper(rho, g))))
    assert errs[0] > errs[1] > errs[2] or errs[2] < 1e-12
    assert errs[2] < 1e-10


def test_substitution_matches_lrho_spectrally():
    errs = []
    for m in (16, 32, 64):
        g = box((m, m))
        x, y = g.coords()
        rho = 1.0 + 0.4 * np.sin(x) * np.cos(y)
        phi = np.sin(x) * np.cos(2 * y) + 0.3 * np.cos(3 * x)
        lhs = np.sqrt(rho) * op.apply_pressure(rho, phi, g)
        rhs = krho.apply_krho(rho, phi / np.sqrt(rho), g)
        errs.append(np.max(np.abs(lhs - rhs)) / np.max(np.abs(lhs)))
    assert errs[0] > errs[1] and errs[2] < 1e-9


def slab(g, s=5.0, axis=1):
    X = g.coords()
    L = g.L[axis]
    d = (X[axis] - L / 2 + L / 2) % L - L / 2
    t = 3 * L / g.n[axis]
    return np.ascontiguousarray(np.broadcast_to(
        1.0 + (s - 1.0) / 2 * (np.tanh((d + L / 4) / t) - np.tanh((d - L / 4) / t)), g.shape))


def test_null_vector_exact():
    g = box((32, 24))
    rho = slab(g)
    w = krho.null_vector(rho)
    Kw = krho.apply_krho(rho, w, g)
    scale = np.max(krho.ksq_full(g)) * np.max(np.abs(w))
    assert np.max(np.abs(Kw)) <= 1e-12 * scale


def test_dense_symmetric_nullity_one():
    g = box((8, 8))
    rho = slab(g, s=4.0)
    A = dense.assemble(lambda v: krho.apply_krho(rho, v, g), g.shape)
    assert dense.symmetry_defect(A) < 1e-13
    assert dense.nullity(A) == 1
    w = krho.null_vector(rho).ravel()
    assert np.linalg.norm(A @ w) <= 1e-12 * np.linalg.norm(A, 2) * np.linalg.norm(w)


@pytest.mark.parametrize("kind", ["cg", "gmres", "rmr"])
def test_constant_density_one_iteration(kind):
    g = box((16, 12))
    rho = np.full(g.shape, 2.5)
    f = np.random.default_rng(3).standard_normal(g.shape)
    A, M = krho.krho_system(rho, g)
    b = krho.project_rhs(np.sqrt(rho) * f, rho)
    res = solvers.solve(kind, A, M, b, tol=1e-12, maxit=20)
    assert res.status == "converged" and res.iters == 1


@pytest.mark.parametrize("kind", ["gmres", "rmr"])
def test_solve_recovers_pressure_solution(kind):
    """phi = sqrt(rho) Phi agrees with the L_rho solution up to a spectrally small error."""
    errs = []
    for m in (16, 32):
        g = box((m, m))
        x, y = g.coords()
        rho = 1.0 + 0.4 * np.sin(x) * np.cos(y)
        f = np.cos(x) * np.sin(2 * y) + 0.5 * np.sin(3 * x)
        res, phi = krho.solve_krho(rho, f, g, kind=kind, tol=1e-12)
        assert res.status == "converged" and res.relres_true < 1e-11
        assert abs(res.x.mean()) < 1e-12 * np.max(np.abs(res.x))
        A, M = op.pressure_system(rho, g)
        ref = solvers.solve("gmres", A, M, sp.project_range(f, g), tol=1e-12)
        a, b = phi - phi.mean(), ref.x - ref.x.mean()
        errs.append(np.max(np.abs(a - b)) / np.max(np.abs(b)))
    assert errs[1] < errs[0] and errs[1] < 1e-8


def test_planted_wrong_coefficient_fails_closed_form():
    """Using the printed coefficient with the sign of its second term flipped breaks the pin."""
    g = box((16, 12))
    X = g.coords()
    w = 1.0 + 0.3 * np.sin(X[0]) * np.sin(X[1])
    rho = w ** -2
    g2 = sum(sp.deriv(rho, g, j) ** 2 for j in range(2))
    wrong = krho.lap_full(rho, g) / (2 * rho) + 0.75 * g2 / rho ** 2
    assert np.max(np.abs(wrong - 2 * 0.3 * np.sin(X[0]) * np.sin(X[1]) / w)) > 1e-2
