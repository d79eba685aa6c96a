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


def test_span_mode_brackets_whole_inner_solves():
    """Span mode (vd_profile_enable(2)) times each inner float solve between two events and
    carries the algorithmic bytes of every launch inside it: one span per refinement sweep,
    and the same bytes as the per-launch mode's float classes for the same solve."""
    n, L = (48, 32, 24), (2 * math.pi,) * 3
    G = vd.Grid(n, L)
    rho = inputs.slab_density(n, L, 6.0, 1, 1.0, math.pi, 3 * L[1] / n[1])
    G.set_density(torch.from_numpy(rho).cuda())
    b = torch.from_numpy(inputs.smooth_random_field(n, L, 7, kmax=4)).cuda()
    G.solve("pressure", "cg", b, tol=1e-10, max_it=400, precision="mixed_dd")   # warm-up
    totals = {}
    for mode in (1, 2):
        vd.vd_profile_reset()
        vd.vd_profile_enable(mode)
        try:
            _, info = G.solve("pressure", "cg", b, tol=1e-10, max_it=400, precision="mixed_dd")
            torch.cuda.synchronize()
        finally:
            vd.vd_profile_enable(0)
        assert info["status"] == "converged"
        if mode == 1:
            totals[1] = sum(vd.vd_profile_read(c)["alg_bytes"] for c in (1, 3, 7))
            assert vd.vd_profile_read(vd.PROFILE_SPAN_INNER_F32)["launches"] == 0
        else:
            span = vd.vd_profile_read(vd.PROFILE_SPAN_INNER_F32)
            assert span["launches"] == info["outer_iters"] and span["ms"] > 0
            assert vd.vd_profile_read(1)["launches"] == 0   # launches are not timed one by one
            totals[2] = span["alg_bytes"]
    assert totals[1] > 0 and totals[1] == totals[2]


def test_profile_mode_out_of_range():
    with pytest.raises(vd.VDError):
        vd.vd_profile_enable(3)
