"""Request server on the serving mix: every result in the mix equals the same solve alone.

300 requests drawn from the serving distribution (Poisson trace, seed 5: 95% of the batched
sizes 2D 64..512^2 / 3D 32..160^3, 5% 256^3; slab densities of ratio 2..50; tolerances 1e-6,
1e-8 and 1e-10) are first solved one at a time through vd_solve, then submitted all at once
to a fresh server with 8 execution slots, twice per precision mode (mixed_dd and mixed).
Every served solution must be bit-for-bit the solution alone: the solves are deterministic
and share no device data, so any difference is a race (between slots, or between a slot and
the set-up of a grid another slot has just created).  Fresh servers start with empty grid
caches, so grids are created while other slots are running solves.
"""

import pytest
import torch

import paper_2403_06654_gb300 as vd
from paper_2403_06654_gb300 import inputs

pytestmark = pytest.mark.gpu

COUNT = 300


def _requests():
    trace = inputs.serving_trace(count=COUNT, rate=2000.0)
    out = []
    for i, (_, inst) in enumerate(trace):
        rho = torch.from_numpy(inst.density()).cuda()
        b = torch.from_numpy(inputs.smooth_random_field(inst.n, inst.L, 5000 + i, kmax=5)).cuda()
        solver = "gmres" if i % 5 == 4 else "cg"
        out.append((inst, rho, b, solver))
    return out


def _alone(reqs, precision):
    grids, xs = {}, []
    for inst, rho, b, solver in reqs:
        key = tuple(inst.n)
        if key not in grids:
            grids[key] = vd.Grid(inst.n, inst.L)
        G = grids[key]
        G.set_density(rho)
        x, info = G.solve("pressure", solver, b, tol=inst.tol, max_it=500, precision=precision)
        assert info["status"] == "converged" and info["relres_true"] <= inst.tol, (inst.n, inst.tol, info)
        xs.append(x.clone())
    torch.cuda.synchronize()
    for G in grids.values():
        G.close()
    return xs


def _served(reqs, precision, outs):
    """All requests at once; even ids into caller buffers, odd ids server-owned (fetched)."""
    for o in outs:
        o.fill_(float("nan"))
    torch.cuda.synchronize()
    S = vd.vd_server_create(max_inflight=8, hbm_budget=0)
    comps = []
    try:
        for i, (inst, rho, b, solver) in enumerate(reqs):
            q = vd.make_request(i, inst.n, inst.L, rho, b, outs[i] if i % 2 == 0 else None, solver=solver,
                                tol=inst.tol, max_it=500, precision=precision)
            vd.vd_server_submit(S, q, vd.vd_server_request_bytes(q))
        vd.vd_server_drain(S)
        while True:
            got = vd.vd_server_poll(S, 512)
            if not got:
                break
            comps += got
        for c in comps:
            if int(c.id) % 2 == 1 and c.status == 0:
                vd.vd_server_fetch(S, int(c.id), outs[int(c.id)])
        torch.cuda.synchronize()
        assert vd.vd_server_stats(S)["reserved"] == 0
    finally:
        vd.vd_server_destroy(S)
    return comps


@pytest.mark.parametrize("precision", ["mixed_dd", "mixed"])
def test_serving_mix_bitwise_equal_to_alone(precision):
    reqs = _requests()
    ratios = [inst.s for inst, _, _, _ in reqs]
    assert max(ratios) > 20 and {inst.tol for inst, _, _, _ in reqs} == {1e-6, 1e-8, 1e-10}
    alone = _alone(reqs, precision)
    outs = [torch.empty_like(x) for x in alone]
    for run in range(2):
        comps = _served(reqs, precision, outs)
        assert len(comps) == COUNT
        bad_status = [(int(c.id), int(c.status)) for c in comps if c.status != 0]
        assert not bad_status, (run, bad_status[:10])
        differ = [i for i in range(COUNT) if not torch.equal(outs[i], alone[i])]
        assert not differ, (run, differ[:10], [tuple(reqs[i][0].n) for i in differ[:10]])
