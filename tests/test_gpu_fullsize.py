"""Parity at the benchmark's full size (256^3 jet workload), in the launch configuration the
benchmark times (launch shapes autotuned first).

* The double pressure apply L_rho phi (Sec. 2, the operator whose solves are timed) against
  the oracle over the whole 256^3 field.
* The right-hand side f = div u* against the oracle's divergence.
* The headline solve (float inner CG, float-pair refinement residual, tol 1e-10): its output
  phi is checked with the oracle's operator: |P f - L_rho phi| / |P f| <= 1.05e-10, where P
  removes the mean (the range of L_rho).

The oracle needs a few seconds per 256^3 operator application on the host cores.
"""

import math

import numpy as np
import pytest
import torch

import paper_2403_06654_gb300 as vd
from paper_2403_06654_gb300 import inputs
from oracle import operators as op
from oracle import spectral as sp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def jet():
    case = inputs.jet_3d(n=256)
    g = sp.Grid(case.n, case.L)
    G = vd.Grid(case.n, case.L)
    G.set_density(torch.from_numpy(case.rho).cuda())
    vd.vd_autotune(G, ("fp64", "mixed", "mixed_dd"))
    return case, g, G


def test_fullsize_divergence_and_apply(jet):
    case, g, G = jet
    f_gpu = G.divergence(torch.from_numpy(case.u).cuda()).cpu().numpy()
    f_ref = sp.div([case.u[0], case.u[1], case.u[2]], g)
    assert np.max(np.abs(f_gpu - f_ref)) <= 1e-12 * np.max(np.abs(f_ref))
    phi = inputs.smooth_random_field(case.n, case.L, 41, kmax=8)
    got = G.apply("pressure", torch.from_numpy(phi).cuda()).cpu().numpy()
    ref = op.apply_pressure(case.rho, phi, g)
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_fullsize_headline_solve_meets_tolerance_under_the_oracle(jet):
    case, g, G = jet
    f = G.divergence(torch.from_numpy(case.u).cuda())
    x, info = G.solve("pressure", "cg", f, tol=1e-10, max_it=500, precision="mixed_dd")
    assert info["status"] == "converged" and info["relres_true"] <= 1e-10
    fb = sp.project_range(f.cpu().numpy(), g)
    r = fb - op.apply_pressure(case.rho, x.cpu().numpy(), g)
    assert np.linalg.norm(r) / np.linalg.norm(fb) <= 1.05e-10
