"""Batched solves recorded into one CUDA graph (conditional WHILE loops, one launch).

Each instance's results must equal the same solve run through vd_solve (same kernels in the
same order; the graph only replaces the host's loop), the pressure solutions must match the
FP64 oracle, new right-hand sides must be picked up without rebuilding the graph, and a run
must launch no kernel from the host (everything is replayed from the graph).
"""

import math

import numpy as np
import pytest
import torch

import paper_2403_06654_gb300 as vd
from paper_2403_06654_gb300 import inputs
from oracle import operators as op
from oracle import solvers as sv
from oracle import spectral as sp

pytestmark = pytest.mark.gpu

SHAPES = [(64, 48), (40, 40), (24, 20, 16), (32, 32, 32), (96, 64), (20, 24, 30)]


def make_items(seed=0):
    rng = np.random.default_rng(seed)
    items, meta = [], []
    for i, n in enumerate(SHAPES):
        L = tuple([2 * math.pi] * len(n))
        s = float(np.exp(rng.uniform(np.log(2), np.log(20))))
        axis = int(rng.integers(0, len(n)))
        rho = inputs.slab_density(n, L, s, axis, float(rng.uniform(0, 2 * math.pi)), math.pi, 3 * L[axis] / n[axis])
        bp = inputs.smooth_random_field(n, L, 50 + i, kmax=4)
        bv = np.stack([inputs.smooth_random_field(n, L, 70 + 3 * i + c, kmax=4) for c in range(len(n))])
        d = {"n": n, "L": L, "rho": torch.from_numpy(rho).cuda(), "a": 1e-3, "inv_sc": 1.0,
             "b_vel": torch.from_numpy(bv).cuda(), "x_vel": torch.zeros(bv.shape, dtype=torch.float64, device="cuda"),
             "b_pres": torch.from_numpy(bp).cuda(), "x_pres": torch.zeros(bp.shape, dtype=torch.float64, device="cuda")}
        items.append(d)
        meta.append((n, L, rho, bp, bv))
    return items, meta


@pytest.mark.parametrize("vel_solver,pres_solver,precision", [("gmres", "cg", "fp64"), ("rmr", "gmres", "fp64"),
                                                              ("gmres", "cg", "mixed_dd"), ("gmres", "rmr", "mixed")])
def test_batch_matches_single_solves(vel_solver, pres_solver, precision):
    """The graph replays the host loop's decisions (refinement sweeps included) on the device."""
    items, meta = make_items()
    B = vd.Batch(items, vel_solver=vel_solver, pres_solver=pres_solver, tol=1e-10, max_it=400, restart=20,
                 precision=precision)
    try:
        l0 = vd.vd_launch_count()
        B.run()
        torch.cuda.synchronize()
        assert vd.vd_launch_count() == l0          # nothing launched from the host
        for i, (n, L, rho, bp, bv) in enumerate(meta):
            iv, ip = B.info(i)
            G = vd.Grid(n, L)
            G.set_density(items[i]["rho"], op="velocity")
            xv, sv_ = G.solve("velocity", vel_solver, items[i]["b_vel"], a=1e-3, inv_sc=1.0, tol=1e-10, max_it=400,
                              restart=20, precision=precision)
            xp, sp_ = G.solve("pressure", pres_solver, items[i]["b_pres"], tol=1e-10, max_it=400, restart=20,
                              precision=precision)
            assert iv["status"] == sv_["status"] == "converged", (i, iv, sv_)
            assert ip["status"] == sp_["status"] == "converged", (i, ip, sp_)
            assert iv["iters"] == sv_["iters"] and ip["iters"] == sp_["iters"], (i, iv, sv_, ip, sp_)
            assert iv["outer_iters"] == sv_["outer_iters"] and ip["outer_iters"] == sp_["outer_iters"]
            assert iv["relres_true"] <= 1e-10 * 1.01 and ip["relres_true"] <= 1e-10 * 1.01
            err = float((items[i]["x_vel"] - xv).abs().max() / xv.abs().max())
            assert err <= 1e-13, (i, err)
            # pressure: the same kernels in the same order, bit for bit (vd_solve's float-pair
            # residual also carries the final inverse transform; the graph runs it separately)
            assert torch.equal(items[i]["x_pres"], xp), (i, float((items[i]["x_pres"] - xp).abs().max()))
    finally:
        B.close()


def test_batch_pressure_matches_oracle_and_new_rhs():
    items, meta = make_items(1)
    B = vd.Batch(items, vel_solver="gmres", pres_solver="cg", tol=1e-12, max_it=500)
    try:
        B.run()
        torch.cuda.synchronize()
        for i in (0, 2):
            n, L, rho, bp, _ = meta[i]
            g = sp.Grid(n, L)
            A, M = op.pressure_system(rho, g)
            ref = sv.cg(A, M, sp.project_range(bp, g), tol=1e-12, maxit=500)
            x = items[i]["x_pres"].cpu().numpy()
            assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) < 1e-10
        # new right-hand sides in the same buffers: the replay reads them
        first = [it["x_pres"].clone() for it in items]
        for it in items:
            it["b_pres"].mul_(-2.0)
        B.run()
        torch.cuda.synchronize()
        for it, x0 in zip(items, first):
            err = float((it["x_pres"] + 2.0 * x0).abs().max() / x0.abs().max())
            assert err < 1e-10
    finally:
        B.close()


def test_batch_rejects_cg_velocity():
    items, _ = make_items()
    with pytest.raises(vd.VDError) as e:
        vd.Batch(items[:1], vel_solver="cg")
    assert e.value.status == vd.VD_ERR_INVALID_ARG
