"""Failures made on the host, reported as statuses, with the context staying usable.

NaN-poisoned right-hand sides (every precision mode, through the server and through a graph
batch), an iteration cap of 1, and a server whose HBM budget admits nothing.  None of them
faults, traps or hangs the GPU: the solvers detect the non-finite reduction or the cap on the
device and return; the next solve on the same grid converges.
"""

import math

import numpy as np
import pytest
import torch

import paper_2403_06654_gb300 as vd
from paper_2403_06654_gb300 import inputs

pytestmark = pytest.mark.gpu


def setup(n=(32, 24, 16)):
    L = (2 * math.pi,) * len(n)
    G = vd.Grid(n, L)
    rho = torch.from_numpy(inputs.slab_density(n, L, 5.0, 1, 1.0, math.pi, 3 * L[1] / n[1])).cuda()
    G.set_density(rho)
    b = torch.from_numpy(inputs.smooth_random_field(n, L, 3, kmax=4)).cuda()
    return n, L, G, rho, b


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_dd"])
@pytest.mark.parametrize("solver", ["cg", "gmres", "rmr"])
def test_nan_rhs_reports_nonfinite_and_context_survives(precision, solver):
    n, L, G, rho, b = setup()
    bad = b.clone()
    bad[1, 2, 3] = float("nan")
    _, info = G.solve("pressure", solver, bad, tol=1e-10, max_it=100, precision=precision)
    assert info["status"] == "nonfinite"
    x, info = G.solve("pressure", solver, b, tol=1e-10, max_it=300, precision=precision)
    assert info["status"] == "converged" and info["relres_true"] <= 1e-10


def test_iteration_cap_of_one():
    n, L, G, rho, b = setup()
    for precision in ("fp64", "mixed_dd"):
        _, info = G.solve("pressure", "cg", b, tol=1e-12, max_it=1, precision=precision)
        assert info["status"] == "max_iter" and info["iters"] == 1


def test_server_nan_request_isolated():
    n, L, G, rho, b = setup()
    x_ref, info = G.solve("pressure", "gmres", b, tol=1e-10, max_it=300, precision="mixed_dd")
    bad = b.clone()
    bad[0, 0, 0] = float("inf")
    S = vd.vd_server_create(max_inflight=2, hbm_budget=0)
    try:
        xs = {}
        for i in range(5):
            xs[i] = torch.zeros_like(b)
            q = vd.make_request(i, n, L, rho, bad if i == 2 else b, xs[i], solver="gmres", tol=1e-10)
            vd.vd_server_submit(S, q, vd.vd_server_request_bytes(q))
        vd.vd_server_drain(S)
        comps = {int(c.id): c for c in vd.vd_server_poll(S, 16)}
    finally:
        vd.vd_server_destroy(S)
    assert comps[2].status == vd.STATUS_CODES["nonfinite"]
    for i in (0, 1, 3, 4):
        assert comps[i].status == 0 and torch.equal(xs[i], x_ref)


def test_server_budget_admits_nothing():
    n, L, G, rho, b = setup()
    S = vd.vd_server_create(max_inflight=2, hbm_budget=4096)
    try:
        q = vd.make_request(0, n, L, rho, b, None)
        with pytest.raises(vd.VDError) as e:
            vd.vd_server_submit(S, q, vd.vd_server_request_bytes(q))
        assert e.value.status == vd.VD_ERR_OOM
        assert vd.vd_server_stats(S)["submitted"] == 0
    finally:
        vd.vd_server_destroy(S)


def test_batch_with_poisoned_item_and_cap():
    """A NaN right-hand side in one batch item and an iteration cap: statuses per item, the
    other items unaffected, and the graph replays fine afterwards."""
    items = []
    for i, n in enumerate([(32, 32), (24, 20, 16), (48, 40)]):
        L = (2 * math.pi,) * len(n)
        rho = torch.from_numpy(inputs.slab_density(n, L, 4.0, 0, 1.0, math.pi, 3 * L[0] / n[0])).cuda()
        bp = torch.from_numpy(inputs.smooth_random_field(n, L, 30 + i, kmax=4)).cuda()
        items.append({"n": n, "L": L, "rho": rho, "b_pres": bp, "x_pres": torch.zeros_like(bp)})
    items[1]["b_pres"][0, 0, 0] = float("nan")
    B = vd.Batch(items, pres_solver="cg", tol=1e-10, max_it=300, precision="mixed_dd")
    try:
        B.run()
        torch.cuda.synchronize()
        st = [B.info(i)[1]["status"] for i in range(3)]
        assert st == ["converged", "nonfinite", "converged"]
        B.run()
        torch.cuda.synchronize()
        assert [B.info(i)[1]["status"] for i in range(3)] == st
    finally:
        B.close()
    capped = vd.Batch(items[:1], pres_solver="cg", tol=1e-14, max_it=1, precision="fp64")
    try:
        capped.run()
        torch.cuda.synchronize()
        info = capped.info(0)[1]
        assert info["status"] == "max_iter" and info["iters"] == 1
    finally:
        capped.close()
