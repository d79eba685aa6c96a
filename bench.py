#!/usr/bin/env python
"""Benchmark: preconditioned variable-density pressure solves at 256^3.

Workload: 3D periodic 256^3 grid on a 2 pi box, swirling-jet-like density
rho(r) = 1 + (s-1)(1 - tanh((r-R)/d))/2 (s = 0.5, R = 0.5, d = 0.05, jet axis x), and the
right-hand side f = div u* of a predictor velocity made of the axial + swirl (ratio 1) base
flow plus seeded 1e-3 noise.  One step = one solve of L_rho phi = f to a 1e-10 relative
residual from a zero initial guess (CG, constant-density preconditioner), verified by the
true double-precision residual that the library returns.

The headline value is the mixed-precision solve rate (float transforms inside double
iterative refinement); the plain double-precision rate is measured beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "solves/s to 1e-10 rel. residual at 256^3, mixed vs FP64; p50/p99 latency"
WORKLOAD = ("3D periodic 256^3 swirling-jet-like density (s=0.5, R=0.5, d=0.05, 2pi box), "
            "rhs = div of axial+swirl(q=1) velocity + 1e-3 noise (seed 3); pressure solve to 1e-10, x0 = 0")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--solver", default="cg", choices=["cg", "gmres", "rmr"])
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--precision", default="mixed_dd", choices=["mixed_dd", "mixed", "fp64"],
                    help="headline precision mode (the other modes are timed beside it)")
    ap.add_argument("--side-steps", type=int, default=10, help="timed solves of the other mixed mode")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


DTYPES = {"mixed_dd": "f32 inner / f64 refinement, residual transforms in float-pair (~2^-48) arithmetic",
          "mixed": "f32 inner / f64 refinement and residual", "fp64": "f64"}

# FP64 arithmetic peak of the GB300 CUDA cores: 1.25 TFLOP/s nominal (recipe table: FP64 is
# far below B200); counted with an FMA as two flops.
FP64_PEAK_TFLOPS = 1.25
# Float-pair arithmetic: 152 SMs x 128 FP32 lanes x 2.07 GHz x 2 = 80.5 TFLOP/s of FP32 FMA; one
# float-pair add costs 11 FP32 instructions and a multiply 7 (9 on average, an FFT being
# mostly adds and twiddle products), so one float-pair flop ~ 9 FP32 issue slots.
DD_PEAK_TFLOPS = 152 * 128 * 2.07e9 / 9 / 1e12


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    mx.append(float(p[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, p[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_setup(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
# ------------------------------------------------------------------------------------------

def oracle_iteration_seconds(n, reps=1):
    """Time one oracle CG iteration of the full-size workload: operator apply, preconditioner
    apply and the vector updates of PCG (the oracle's own code, unmodified)."""
    import numpy as np
    from oracle import operators as op
    from oracle import spectral as sp
    from paper_2403_06654_gb300 import inputs

    case = inputs.jet_3d(n=n)
    g = sp.Grid(case.n, case.L)
    A, M = op.pressure_system(case.rho, g)
    p = inputs.random_field(g.shape, 99)
    r = inputs.random_field(g.shape, 98)
    x = np.zeros(g.shape)
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        q = A(p)
        alpha = float(np.dot(r.ravel(), M(r).ravel())) / float(np.dot(p.ravel(), q.ravel()))
        x = x + alpha * p
        r = r - alpha * q
        z = M(r)
        p = z + 0.5 * p
        ts.append(time.perf_counter() - t0)
    return min(ts)


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import numpy as np  # noqa: F401

    iters = 14   # CG iterations of the double-precision solve of this workload (measured on the GPU path)
    for _ in range(args.warmup):
        oracle_iteration_seconds(args.n)
    t = []
    for _ in range(args.steps):
        t.append(oracle_iteration_seconds(args.n))
    per_iter = statistics.median(t)
    value = 1.0 / (per_iter * iters)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_iter * iters * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": WORKLOAD, "solver": "cg", "precision": "fp64"},
           "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                            "sample": f"each step: one oracle CG iteration at {args.n}^3 (operator, preconditioner, "
                                      f"updates), scaled to {iters} iterations per solve"},
           "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


# ------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------

def main():
    args = parse()
    rank, world, local = dist_setup(args)
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch

    import paper_2403_06654_gb300 as vd
    from paper_2403_06654_gb300 import inputs

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    vd.lib()   # fails loudly when the library is missing
    n = args.n
    L = (2 * math.pi,) * 3
    case = inputs.jet_3d(n=n)
    G = vd.Grid(case.n, L, device=dev)
    rho_d = torch.from_numpy(case.rho).to(dev)
    G.set_density(rho_d)
    f = G.divergence(torch.from_numpy(case.u).to(dev))
    del case
    stream = torch.cuda.current_stream()
    x = torch.zeros_like(f)
    kw = dict(tol=args.tol, max_it=500, restart=30)

    def solve(prec):
        _, info = G.solve("pressure", args.solver, f, out=x, precision=prec, **kw)
        if info["status"] != "converged" or not (info["relres_true"] <= args.tol):
            raise SystemExit(f"solve failed: {info}")
        return info

    head = args.precision
    side = "mixed" if head == "mixed_dd" else "mixed_dd"
    # warm-up
    for _ in range(args.warmup):
        solve(head)
    solve(side)
    solve("fp64")

    # ---------------- timed: headline precision ----------------
    sampler = ClockSampler(local)
    vd.vd_profile_reset()
    vd.vd_profile_enable(True)
    l0 = vd.vd_launch_count()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    barrier()
    sampler.start()
    infos = []
    ev[0].record(stream)
    for k in range(args.steps):
        infos.append(solve(head))
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    vd.vd_profile_enable(False)
    launches = vd.vd_launch_count() - l0
    lat = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    t_mixed = ev[0].elapsed_time(ev[args.steps]) / 1e3
    prof = {c: vd.vd_profile_read(c) for c in vd.PROFILE_CLASSES}
    if pg is not None:
        tt = torch.tensor([t_mixed], device=dev)
        pg.all_reduce(tt, op=pg.ReduceOp.MAX)
        t_mixed = float(tt.item())

    # double-precision check of the last headline solution (outside the timed region)
    fb = f.clone()
    r64 = fb - G.apply("pressure", x)
    # the pressure right-hand side is projected onto the range: remove its null-space part
    r64 = r64 - r64.mean()
    fmean = fb - fb.mean()
    verified = float(torch.linalg.vector_norm(r64) / torch.linalg.vector_norm(fmean))

    # ---------------- timed: the other mixed mode ----------------
    ev3 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    barrier()
    ev3[0].record(stream)
    infos_side = [solve(side) for _ in range(args.side_steps)]
    ev3[1].record(stream)
    torch.cuda.synchronize()
    barrier()
    t_side = ev3[0].elapsed_time(ev3[1]) / 1e3

    # ---------------- timed: plain FP64 ----------------
    ev2 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    barrier()
    ev2[0].record(stream)
    infos64 = [solve("fp64") for _ in range(args.fp64_steps)]
    ev2[1].record(stream)
    torch.cuda.synchronize()
    barrier()
    t64 = ev2[0].elapsed_time(ev2[1]) / 1e3
    if pg is not None:
        tt = torch.tensor([t64], device=dev)
        pg.all_reduce(tt, op=pg.ReduceOp.MAX)
        t64 = float(tt.item())

    # ---------------- end to end through host buffers ----------------
    rho_h = rho_d.cpu().pin_memory()
    f_h = f.cpu().pin_memory()
    x_h = torch.empty_like(f_h).pin_memory()
    rho_e = torch.empty_like(rho_d)
    f_e = torch.empty_like(f)
    barrier()
    t0 = time.perf_counter()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.e2e_steps):
        rho_e.copy_(rho_h, non_blocking=True)
        f_e.copy_(f_h, non_blocking=True)
        G.set_density(rho_e)
        _, info = G.solve("pressure", args.solver, f_e, out=x, precision=head, **kw)
        if info["status"] != "converged":
            raise SystemExit(f"e2e solve failed: {info}")
        x_h.copy_(x, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    t_e2e = e0.elapsed_time(e1) / 1e3
    wall_e2e = time.perf_counter() - t0
    if pg is not None:
        tt = torch.tensor([t_e2e], device=dev)
        pg.all_reduce(tt, op=pg.ReduceOp.MAX)
        t_e2e = float(tt.item())

    # ---------------- roofline of the dominant kernel class ----------------
    pk, pk_src = peaks()
    # per inner (float) Krylov iteration: float passes + float vector kernels
    n_inner = sum(i["iters"] for i in infos)
    f32c = [c for c in prof if vd.PROFILE_CLASSES[c] in ("axis_f32", "xpass_f32", "vec_f32")]
    it_ms = sum(prof[c]["ms"] for c in f32c) / max(n_inner, 1)
    it_bytes = sum(prof[c]["alg_bytes"] for c in f32c) / max(n_inner, 1)
    per_iter = {"ms": it_ms, "alg_bytes": it_bytes, "achieved_gbs": it_bytes / (it_ms / 1e3) / 1e9,
                "frac_of_hbm": it_bytes / (it_ms / 1e3) / 1e9 / pk["hbm_gbs"],
                "iterations": n_inner,
                "includes": "float transform passes + float Krylov vector kernels of the inner CG, per iteration"}
    dom = max((c for c in prof if c != 4), key=lambda c: prof[c]["ms"])
    d = prof[dom]
    name = vd.PROFILE_CLASSES[dom]
    per_launch_ms = d["ms"] / max(d["launches"], 1)
    if name.endswith("f32"):
        achieved = d["alg_bytes"] / (d["ms"] / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / pk["hbm_gbs"], "traffic": None,
                "peak_source": f"{pk_src} hbm_gbs (MEASURED_PEAKS.json)" if pk_src == "measured" else "fallback",
                "alg_bytes_per_launch": d["alg_bytes"] / max(d["launches"], 1), "ms_per_launch": per_launch_ms}
    else:
        achieved = d["alg_flops"] / (d["ms"] / 1e3) / 1e12
        pk_alu = FP64_PEAK_TFLOPS if name.endswith("f64") else DD_PEAK_TFLOPS
        roof = {"bound": "alu", "kernel": name, "achieved": achieved, "peak": pk_alu, "unit": "TFLOP/s",
                "frac": achieved / pk_alu, "traffic": None,
                "peak_source": ("nominal GB300 FP64 (recipe table), FMA = 2 flops" if name.endswith("f64") else
                                "float-pair peak derived from the FP32 unit count and clock (see DESIGN.md)"),
                "alg_flops_per_launch": d["alg_flops"] / max(d["launches"], 1), "ms_per_launch": per_launch_ms,
                "hbm_gbs_achieved": d["alg_bytes"] / (d["ms"] / 1e3) / 1e9}
    classes = {vd.PROFILE_CLASSES[c]: {"launches": prof[c]["launches"], "ms": prof[c]["ms"],
                                       "GB/s": prof[c]["alg_bytes"] / max(prof[c]["ms"], 1e-9) / 1e6}
               for c in prof}

    # ---------------- CPU oracle baseline (rank 0, N = 1) ----------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        iters64 = infos64[0]["iters"]
        t_it = oracle_iteration_seconds(n)
        cpu = {"value": 1.0 / (t_it * iters64), "unit": "solves/s", "cores": 1, "kind": "oracle",
               "sample": f"one oracle CG iteration of the {n}^3 solve ({t_it:.1f} s: operator, preconditioner, "
                         f"updates; numpy single-threaded), scaled to the {iters64} CG iterations of the FP64 solve"}

    total_solves = args.steps * world
    value = total_solves / t_mixed
    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_mixed / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[head], "data": "synthetic",
        "config": {"workload": WORKLOAD, "solver": args.solver, "precision": head, "tol": args.tol,
                   "grid": [n, n, n], "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (each 256^3 field 134 MB; working set ~1.6 GB)"},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "mean": float(np.mean(lat))},
        "iters": infos[-1]["iters"], "outer_iters": infos[-1]["outer_iters"],
        "relres_true_max": max(i["relres_true"] for i in infos),
        "relres_fp64_check": verified,
        side: {"value": args.side_steps * world / t_side, "unit": "solves/s",
               "ms_per_step": t_side / args.side_steps * 1e3, "iters": infos_side[-1]["iters"],
               "relres_true_max": max(i["relres_true"] for i in infos_side), "dtype": DTYPES[side]},
        "fp64": {"value": args.fp64_steps * world / t64, "unit": "solves/s",
                 "ms_per_step": t64 / args.fp64_steps * 1e3, "iters": infos64[-1]["iters"],
                 "relres_true_max": max(i["relres_true"] for i in infos64), "dtype": "f64"},
        "headline_over_fp64": (value) / (args.fp64_steps * world / t64),
        "e2e": {"value": args.e2e_steps * world / t_e2e, "unit": "solves/s",
                "h2d_bytes_per_step": int(rho_h.numel() * 8 + f_h.numel() * 8),
                "d2h_bytes_per_step": int(x_h.numel() * 8), "wall_s": wall_e2e,
                "includes": "H2D of rho and f from pinned host memory, density setup, solve, D2H of phi"},
        "gpu_launches": int(launches),
        "roofline": roof,
        "per_iteration": per_iter,
        "kernel_classes": classes,
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    if pg is not None:
        pg.barrier()
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
