"""The launch-shape autotuner on the GPU: it fills the table for every pass of a grid, and
results stay within the parity bounds afterwards (FP64 applies bit-identical: the Stockham
engine's shapes only redistribute whole lines; float and float-pair solves still converge
and match the oracle)."""

import math

import numpy as np
import pytest
import torch

import paper_2403_06654_gb300 as vd
from paper_2403_06654_gb300 import inputs
from oracle import operators as op
from oracle import spectral as sp

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [(48, 40, 30), (128, 64, 80)])
def test_autotune_fills_table_and_keeps_parity(n):
    L = (2 * math.pi,) * 3
    g = sp.Grid(n, L)
    G = vd.Grid(n, L)
    rho = inputs.slab_density(n, L, 6.0, 1, 1.0, math.pi, 3 * L[1] / n[1])
    G.set_density(torch.from_numpy(rho).cuda())
    phi = inputs.random_field(g.shape, 3)
    before = G.apply("pressure", torch.from_numpy(phi).cuda()).clone()
    vd.vd_autotune(G, ("fp64", "mixed", "mixed_dd"))
    tab = vd.vd_autotune_table()
    for ty in (0, 1, 2):
        for axis, m in ((1, n[1]), (2, n[2])):
            for d in (-1, 1):
                assert any(e[:5] == (0, ty, m, axis, d) for e in tab), (ty, axis, d)
        for mode in (0, 1, 2):
            assert any(e[:5] == (1, ty, n[0] // 2, 0, mode) for e in tab)
    after = G.apply("pressure", torch.from_numpy(phi).cuda())
    assert torch.equal(before, after)
    ref = op.apply_pressure(rho, phi, g)
    assert np.max(np.abs(after.cpu().numpy() - ref)) / np.max(np.abs(ref)) < 1e-12
    b = torch.from_numpy(inputs.smooth_random_field(n, L, 4, kmax=4)).cuda()
    for prec in ("mixed", "mixed_dd"):
        x, info = G.solve("pressure", "cg", b, tol=1e-10, max_it=500, precision=prec)
        assert info["status"] == "converged" and info["relres_true"] <= 1e-10
