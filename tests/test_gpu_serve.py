"""Request server (continuous batching): results in the mix equal results alone.

Requests of different grids, density ratios, tolerances and solvers are submitted together
to a server with 4 execution slots and a small HBM budget (so admission has to wait for
memory), and each result is compared with the same solve run alone through vd_solve.  The
solves are deterministic (fixed launch shapes, fixed-order reductions) and share no device
data, so the results must agree bit for bit.
"""

import math

import numpy as np
import pytest
import torch

import paper_2403_06654_gb300 as vd
from paper_2403_06654_gb300 import inputs

pytestmark = pytest.mark.gpu


def make_cases():
    rng = np.random.default_rng(41)
    shapes = [(32, 32), (48, 40), (64, 64), (24, 24, 24), (32, 24, 16), (40, 40, 20), (128, 16, 12), (96, 80)]
    cases = []
    for i in range(16):
        n = shapes[i % len(shapes)]
        L = tuple([2 * math.pi] * len(n))
        s = float(np.exp(rng.uniform(np.log(2), np.log(50))))
        axis = int(rng.integers(0, len(n)))
        rho = inputs.slab_density(n, L, s, axis, float(rng.uniform(0, 2 * math.pi)), math.pi, 3 * L[axis] / n[axis])
        f = inputs.smooth_random_field(n, L, 100 + i, kmax=5)
        tol = [1e-6, 1e-8, 1e-10][i % 3]
        solver = ["cg", "gmres"][i % 2]
        cases.append((n, L, rho, f, tol, solver))
    return cases


def test_server_results_match_alone():
    cases = make_cases()
    alone = []
    dev = []
    for (n, L, rho, f, tol, solver) in cases:
        G = vd.Grid(n, L)
        r = torch.from_numpy(rho).cuda()
        b = torch.from_numpy(f).cuda()
        G.set_density(r)
        x, info = G.solve("pressure", solver, b, tol=tol, max_it=500, precision="mixed_dd")
        alone.append((x.clone(), info))
        dev.append((r, b, torch.zeros_like(b)))
    torch.cuda.synchronize()
    reqs = [vd.make_request(i, c[0], c[1], dev[i][0], dev[i][1], dev[i][2], solver=c[5], tol=c[4])
            for i, c in enumerate(cases)]
    sizes = [vd.vd_server_request_bytes(q) for q in reqs]
    assert all(s > 0 for s in sizes)
    # budget for about two of the largest requests at a time: admission must wait for memory
    S = vd.vd_server_create(max_inflight=4, hbm_budget=2 * max(sizes) + 1)
    try:
        for q, s in zip(reqs, sizes):
            vd.vd_server_submit(S, q, s)
        vd.vd_server_drain(S)
        comps = vd.vd_server_poll(S, 64)
        st = vd.vd_server_stats(S)
    finally:
        vd.vd_server_destroy(S)
    assert len(comps) == len(cases) and st["completed"] == len(cases) and st["reserved"] == 0
    torch.cuda.synchronize()
    for c in comps:
        i = int(c.id)
        xa, info = alone[i]
        assert c.status == 0 and info["status"] == "converged"
        assert c.iters == info["iters"]
        assert c.relres_true <= cases[i][4]
        xs = dev[i][2]
        err = float((xs - xa).abs().max() / xa.abs().max())
        assert err == 0.0, (i, err)
        assert c.t_submit <= c.t_start <= c.t_done


def test_server_rejects_oversized_request():
    n, L = (64, 64, 64), (2 * math.pi,) * 3
    r = torch.ones((64, 64, 64), dtype=torch.float64, device="cuda")
    q = vd.make_request(0, n, L, r, r, torch.zeros_like(r))
    S = vd.vd_server_create(max_inflight=1, hbm_budget=1 << 20)
    try:
        with pytest.raises(vd.VDError) as e:
            vd.vd_server_submit(S, q, vd.vd_server_request_bytes(q))
        assert e.value.status == vd.VD_ERR_OOM
    finally:
        vd.vd_server_destroy(S)


@pytest.mark.parametrize("precision", ["mixed", "mixed_dd"])
def test_server_concurrent_identical_requests_bitwise(precision):
    """48 copies of one 128^3 request (float inner transforms on the register four-step
    kernels) served on 8 slots: every result equals the solve run alone, bit for bit.
    Kernels of other streams share the SMs here, so a missing barrier inside a kernel
    shows up as a differing result."""
    n, L = (128, 128, 128), (2 * math.pi,) * 3
    rho = torch.from_numpy(inputs.slab_density(n, L, 36.0, 2, 1.0, math.pi, 3 * L[2] / n[2])).cuda()
    b = torch.from_numpy(inputs.smooth_random_field(n, L, 7, kmax=5)).cuda()
    G = vd.Grid(n, L)
    G.set_density(rho)
    ref, info = G.solve("pressure", "cg", b, tol=1e-10, max_it=500, precision=precision)
    assert info["status"] == "converged"
    xs = [torch.zeros_like(b) for _ in range(48)]
    S = vd.vd_server_create(max_inflight=8, hbm_budget=0)
    try:
        for i, x in enumerate(xs):
            q = vd.make_request(i, n, L, rho, b, x, solver="cg", tol=1e-10, precision=precision)
            vd.vd_server_submit(S, q, vd.vd_server_request_bytes(q))
        vd.vd_server_drain(S)
        comps = []
        while True:
            got = vd.vd_server_poll(S, 64)
            if not got:
                break
            comps += got
    finally:
        vd.vd_server_destroy(S)
    torch.cuda.synchronize()
    assert len(comps) == 48
    assert all(c.status == 0 and c.iters == info["iters"] for c in comps)
    bad = [i for i, x in enumerate(xs) if not torch.equal(x, ref)]
    assert not bad, bad


def test_server_owned_solutions_fetch_and_release():
    """Requests without an output buffer: the solution stays in server memory (counted in
    the budget) until fetched or released; fetched results equal the solves alone."""
    cases = make_cases()[:6]
    alone, dev = [], []
    for (n, L, rho, f, tol, solver) in cases:
        G = vd.Grid(n, L)
        r = torch.from_numpy(rho).cuda()
        b = torch.from_numpy(f).cuda()
        G.set_density(r)
        x, info = G.solve("pressure", solver, b, tol=tol, max_it=500, precision="mixed_dd")
        alone.append(x.clone())
        dev.append((r, b))
    torch.cuda.synchronize()
    S = vd.vd_server_create(max_inflight=3, hbm_budget=0)
    try:
        reqs = [vd.make_request(i, c[0], c[1], dev[i][0], dev[i][1], None, solver=c[5], tol=c[4])
                for i, c in enumerate(cases)]
        for q in reqs:
            vd.vd_server_submit(S, q, vd.vd_server_request_bytes(q))
        vd.vd_server_drain(S)
        comps = vd.vd_server_poll(S, 64)
        assert len(comps) == len(cases) and all(c.status == 0 and c.x for c in comps)
        held = vd.vd_server_stats(S)["reserved"]
        assert held >= sum(8 * int(np.prod(c[0])) for c in cases)
        for i in range(len(cases) - 1):
            out = torch.empty_like(alone[i])
            vd.vd_server_fetch(S, i, out)
            torch.cuda.synchronize()
            assert torch.equal(out, alone[i]), i
        last = len(cases) - 1
        vd.vd_server_release(S, last)
        assert vd.vd_server_stats(S)["reserved"] == 0
        with pytest.raises(vd.VDError) as e:
            vd.vd_server_release(S, last)
        assert e.value.status == vd.VD_ERR_INVALID_ARG
    finally:
        vd.vd_server_destroy(S)


def test_server_cancel_queued_requests():
    """With one slot the later requests queue; cancelled ones produce no completion, the rest
    complete, and a request that already completed cannot be cancelled."""
    n, L = (64, 64, 64), (2 * math.pi,) * 3
    rho = torch.from_numpy(inputs.slab_density(n, L, 20.0, 1, 1.0, math.pi, 3 * L[1] / n[1])).cuda()
    b = torch.from_numpy(inputs.smooth_random_field(n, L, 12, kmax=5)).cuda()
    S = vd.vd_server_create(max_inflight=1, hbm_budget=0)
    try:
        for i in range(6):
            q = vd.make_request(i, n, L, rho, b, None, solver="cg", tol=1e-10, precision="fp64")
            vd.vd_server_submit(S, q, vd.vd_server_request_bytes(q))
        vd.vd_server_cancel(S, 3)
        vd.vd_server_cancel(S, 5)
        vd.vd_server_drain(S)
        comps = vd.vd_server_poll(S, 64)
        assert sorted(int(c.id) for c in comps) == [0, 1, 2, 4]
        assert all(c.status == 0 for c in comps)
        for c in comps:
            vd.vd_server_release(S, int(c.id))
        with pytest.raises(vd.VDError) as e:
            vd.vd_server_cancel(S, 0)
        assert e.value.status == vd.VD_ERR_INVALID_ARG
        st = vd.vd_server_stats(S)
        assert st["reserved"] == 0 and st["completed"] == 4
    finally:
        vd.vd_server_destroy(S)
