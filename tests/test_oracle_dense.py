"""Dense brute-force checks of the oracle operators on tiny grids (CPU only).

What the paper and the mathematics fix:
* the discrete pressure operator sum_j D_j rho^-1 D_j is symmetric and negative
  semi-definite, with a null space of dimension 2^d (constant and Nyquist-corner modes);
* the eigenvalues of the preconditioned pressure operator (Lap)^+ L~ on the range lie in
  [1/rho_max, 1/rho_min] (Rayleigh-quotient bound), so its condition number is at most
  rho_max/rho_min whatever n;
* the paper (Sec. 3.1 and 3.2, condition-number figures) reports that the unpreconditioned
  operators are badly conditioned (O(10^4)-O(10^8)) and grow with n, while the
  preconditioned ones stay O(1)-O(10^2) and quasi-independent of n; it states that the
  Fourier expansion behaves like the Chebyshev one it plots.
"""

import math

import numpy as np
import pytest

from oracle import spectral as sp
from oracle import operators as op
from oracle import dense
from paper_2403_06654_gb300 import inputs


def tophat(n, r=3.0, d=0.05):
    return inputs.tophat_1d(n=n, r=r, d=d)


@pytest.mark.parametrize("n", [32, 64, 128])
def test_pressure_1d_symmetric_psd_nullity(n):
    g = sp.Grid((n,), (2 * math.pi,))
    rho = tophat(n, d=0.2)
    A = dense.assemble(lambda v: op.apply_pressure(rho, v, g), g.shape)
    assert dense.symmetry_defect(A) < 1e-13
    w = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert w.max() < 1e-10 * abs(w.min())            # -A is positive semi-definite
    assert dense.nullity(A) == 2


@pytest.mark.parametrize("n,L", [((8, 6), (1.0, 2.0)), ((4, 6, 4), (2 * math.pi,) * 3)])
def test_pressure_nd_symmetric_nullity(n, L):
    g = sp.Grid(n, L)
    rng = np.random.default_rng(11)
    rho = 1.0 + 2.0 * rng.uniform(size=g.shape)
    A = dense.assemble(lambda v: op.apply_pressure(rho, v, g), g.shape)
    assert dense.symmetry_defect(A) < 1e-13
    assert dense.nullity(A) == 2 ** g.ndim


@pytest.mark.parametrize("n", [32, 64, 128, 256])
def test_preconditioned_pressure_eigenvalue_bound(n):
    """Config-1 density (r = 3): eig((Lap)^+ L~) in [1/3, 1] on the range."""
    g = sp.Grid((n,), (2 * math.pi,))
    rho = tophat(n)
    B = dense.assemble(lambda v: sp.precond_pressure(op.apply_pressure(rho, v, g), g), g.shape)
    w = dense.eig_range(B)
    assert np.max(np.abs(w.imag)) < 1e-10
    lo, hi = 1.0 / rho.max(), 1.0 / rho.min()
    assert w.real.min() >= lo * (1 - 1e-10)
    assert w.real.max() <= hi * (1 + 1e-10)
    assert len(w) == n - 2


def test_condition_numbers_vs_n_pressure():
    kap_A, kap_left, kap_right = [], [], []
    for n in (32, 64, 128):
        g = sp.Grid((n,), (2 * math.pi,))
        rho = tophat(n, d=0.1)
        A = dense.assemble(lambda v: op.apply_pressure(rho, v, g), g.shape)
        M = dense.assemble(lambda v: sp.precond_pressure(v, g), g.shape)
        kap_A.append(dense.cond_on_range(A))
        kap_left.append(dense.cond_on_range(M @ A))
        kap_right.append(dense.cond_on_range(A @ M))
    # unpreconditioned: grows like n^2
    assert kap_A[1] / kap_A[0] > 3.0 and kap_A[2] / kap_A[1] > 3.0
    # preconditioned: O(1)-O(10^2) and quasi-independent of n
    for k in (kap_left, kap_right):
        assert max(k) < 100.0
        assert max(k) / min(k) < 1.2


@pytest.mark.parametrize("s", [2.0, 10.0])
def test_condition_numbers_viscous(s):
    """kappa(V_rho) grows with n while the right-preconditioned V_rho V^-1 stays O(1) and
    n-independent (Sec. 3.1, a = 1e-2, top-hat with d = 0.1, x0 = L/5).

    Fourier reading: the left-preconditioned V^-1 V_rho = V^-1 (V_rho V^-1) V is similar to
    V_rho V^-1 (same eigenvalues), but it is strongly non-normal and its 2-norm condition
    number grows like n^2 on this discretisation; the solvers are therefore
    right-preconditioned.
    """
    a = 1e-2
    res = []
    for n in (128, 256):
        g = sp.Grid((n,), (2 * math.pi,))
        x = 2 * math.pi * np.arange(n) / n
        x0 = 2 * math.pi / 5
        rho = 1.0 + (s - 1) / 2 * (np.tanh((x - math.pi + x0) / 0.1) - np.tanh((x - math.pi - x0) / 0.1))
        V = dense.assemble(lambda v: op.apply_velocity(rho, v[None], g, a, 1.0)[0], g.shape)
        P = dense.assemble(lambda v: sp.precond_velocity(v, g, a), g.shape)
        res.append((np.linalg.cond(V), np.linalg.cond(V @ P), np.linalg.cond(P @ V)))
    (kv0, kr0, kl0), (kv1, kr1, kl1) = res
    assert kv1 > 2.0 * kv0                          # grows with n
    assert max(kr0, kr1) < 20.0                     # right-preconditioned stays small
    assert kr1 / kr0 < 1.3                          # and quasi-independent of n
    assert kl1 / kl0 > 3.0                          # left: non-normal, grows (Fourier reading)


def test_constant_density_preconditioned_is_scaled_identity():
    g = sp.Grid((6, 4), (1.0, 1.0))
    rho0 = 1.7
    rho = np.full(g.shape, rho0)
    B = dense.assemble(lambda v: sp.precond_pressure(op.apply_pressure(rho, v, g), g), g.shape)
    P = dense.assemble(lambda v: sp.project_range(v, g), g.shape)
    assert np.max(np.abs(B - P / rho0)) < 1e-13


def test_golden_tophat1d_is_current():
    """tests/golden/tophat1d.json (read by the benchmark beside the GPU's 1D top-hat solves) is
    what its script computes from the oracle now; its eigenvalue ratio meets the rho_max/rho_min
    bound and its preconditioned SVD condition number is O(1)-O(10) (Sec. 3.2) while the
    unpreconditioned one is O(10^4)."""
    import importlib.util
    import json
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    spec = importlib.util.spec_from_file_location("make_tophat1d", os.path.join(here, "make_tophat1d.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    fresh = mod.compute()
    with open(os.path.join(here, "tophat1d.json")) as fh:
        stored = json.load(fh)
    for k in ("kappa_L", "kappa_left_MA", "kappa_right_AM", "eig_ratio_MA"):
        assert abs(stored[k] - fresh[k]) <= 1e-6 * abs(fresh[k]), k
    for s in ("cg", "gmres", "rmr"):
        assert stored["solvers"][s]["iters"] == fresh["solvers"][s]["iters"]
    assert stored["eig_ratio_MA"] <= stored["eig_bound_rho_ratio"] * (1 + 1e-10)
    assert stored["kappa_left_MA"] < 100 and stored["kappa_L"] > 1e4
