"""The packed float-pair transform engine against the unpacked one, bit for bit.

The float-pair y/z and x passes (the refinement residual of mixed_dd, Eq. 7 with the
operators of Sec. 2) run their shared-memory transforms on complex float pairs held in packed
two-float registers whenever the transform length has radices 2, 4 and 8 only.  Every packed
operation repeats the unpacked float-pair operation lane by lane in the same order, so a whole
mixed_dd solve must give the same bits with either engine.  The unpacked engine is selected
through the launch-shape table (choice 256 for the float-pair entries); the table is restored
afterwards.  Radix-3 lengths keep the unpacked engine in both runs.
"""

import math

import numpy as np
import pytest
import torch

import paper_2403_06654_gb300 as vd
from paper_2403_06654_gb300 import inputs

pytestmark = pytest.mark.gpu

UNPACKED = 256
# packed lengths: x pass n0/2 = 128, 64, 512; y 64, 512; z 256 (the 64 x 32 x 16 and 48 x 40 x 32
# grids keep the unpacked engine on their short or radix-3/5 axes)
GRIDS = [((256,), (2 * math.pi,)), ((1024,), (2 * math.pi,)), ((128, 64), (2 * math.pi, 2.0)),
         ((64, 512), (2 * math.pi, 4.0)), ((64, 32, 16), (2 * math.pi,) * 3), ((32, 16, 256), (2 * math.pi,) * 3),
         ((48, 40, 32), (2 * math.pi,) * 3)]


def _keys(n):
    """float-pair table keys of the passes a grid of shape n uses"""
    keys = [(1, 2, n[0] // 2, 0, mode) for mode in (0, 1, 2)]
    for axis in range(1, len(n)):
        keys += [(0, 2, n[axis], axis, d) for d in (-1, 1)]
    return keys


def _solve_all(n, L):
    ax = len(n) - 1
    rho = inputs.slab_density(n, L, 20.0, ax, 0.4 * L[ax], 0.5 * L[ax], 3 * L[ax] / n[ax])
    b = torch.from_numpy(np.stack([inputs.smooth_random_field(n, L, 5 + c, kmax=5) for c in range(len(n))])).cuda()
    f = inputs.smooth_random_field(n, L, 9, kmax=5)
    f = torch.from_numpy(f - f.mean()).cuda()
    out = []
    G = vd.Grid(n, L)
    G.set_density(torch.from_numpy(rho).cuda(), "velocity")
    out.append(G.solve("velocity", "gmres", b, a=1e-3, inv_sc=1.0, tol=1e-10, max_it=600, restart=30,
                       precision="mixed_dd"))
    G.set_density(torch.from_numpy(rho).cuda(), "pressure")
    out.append(G.solve("pressure", "cg", f, tol=1e-10, max_it=600, precision="mixed_dd"))
    G.set_density(torch.from_numpy(rho).cuda(), "krho")
    out.append(G.solve("krho", "gmres", f, tol=1e-10, max_it=600, precision="mixed_dd"))
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("n,L", GRIDS)
def test_packed_engine_bit_identical(n, L):
    saved = {tuple(e[:5]): e[5] for e in vd.vd_autotune_table()}
    keys = _keys(n)
    packed = _solve_all(n, L)
    try:
        for k in keys:
            vd.vd_autotune_set(*k, UNPACKED)
        unpacked = _solve_all(n, L)
    finally:
        for k in keys:
            vd.vd_autotune_set(*k, saved.get(k, -1))
    for (xp, ip), (xu, iu) in zip(packed, unpacked):
        assert ip["status"] == "converged", ip
        assert ip["iters"] == iu["iters"] and ip["outer_iters"] == iu["outer_iters"]
        assert ip["relres_true"] == iu["relres_true"]
        assert torch.equal(xp, xu)
