"""The library's event profiler counts the work of the iterations that ran.

Inner CG and RMR iterations are enqueued one batch ahead of the convergence check, so a
batch can be launched after convergence (its kernels return at once).  Such a batch must not
add launches, time or algorithmic bytes to the profile: a 3D pressure apply is four float
y/z passes, so a mixed solve records exactly four per inner iteration.
"""

import math

import pytest
import torch

import paper_2403_06654_gb300 as vd
from paper_2403_06654_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("solver", ["cg", "rmr"])
def test_profile_excludes_speculative_batches(solver):
    n, L = (32, 24, 16), (2 * math.pi,) * 3
    G = vd.Grid(n, L)
    rho = inputs.slab_density(n, L, 4.0, 2, 1.0, math.pi, 3 * L[2] / n[2])
    G.set_density(torch.from_numpy(rho).cuda())
    b = torch.from_numpy(inputs.smooth_random_field(n, L, 5, kmax=4)).cuda()
    G.solve("pressure", solver, b, tol=1e-10, max_it=400, precision="mixed")   # warm-up
    vd.vd_profile_reset()
    vd.vd_profile_enable(True)
    try:
        l0 = vd.vd_launch_count()
        _, info = G.solve("pressure", solver, b, tol=1e-10, max_it=400, precision="mixed")
        launched = vd.vd_launch_count() - l0
    finally:
        vd.vd_profile_enable(False)
    assert info["status"] == "converged"
    axis = vd.vd_profile_read(1)
    assert axis["launches"] == 4 * info["iters"], (axis, info)
    assert launched >= 4 * info["iters"]
