#!/usr/bin/env python
"""Benchmark: preconditioned variable-density pressure solves at 256^3.

Workload: 3D periodic 256^3 grid on a 2 pi box, swirling-jet-like density
rho(r) = 1 + (s-1)(1 - tanh((r-R)/d))/2 (s = 0.5, R = 0.5, d = 0.05, jet axis x), and the
right-hand side f = div u* of a predictor velocity made of the axial + swirl (ratio 1) base
flow plus seeded 1e-3 noise.  One step = one solve of L_rho phi = f to a 1e-10 relative
residual from a zero initial guess (CG, constant-density preconditioner), verified by the
true double-precision residual that the library returns.

The headline value is the mixed-precision solve rate (float transforms inside double
iterative refinement); the plain double-precision rate is measured beside it.  The headline
steps run without instrumentation; the same number of solves then runs again with CUDA
events around every kernel (the roofline and kernel-class figures), and a third time with
events around each inner float solve only (the per-iteration figure).

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


def parse(argv=None):
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
    ap.add_argument("--no-extras", action="store_true", help="skip the 1D and 2D workload measurements")
    ap.add_argument("--rt-steps", type=int, default=100)
    ap.add_argument("--mode", default="solve", choices=["solve", "serve", "batch"],
                    help="solve: the 256^3 solve-rate line (with a short serving run); serve: the serving line")
    ap.add_argument("--no-serve", action="store_true", help="skip the short serving run of the solve line")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched graph run of the solve line")
    ap.add_argument("--no-autotune", action="store_true", help="keep the built-in launch shapes")
    ap.add_argument("--serve-count", type=int, default=None, help="requests of the serving trace")
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="mean arrival rate (req/s)")
    ap.add_argument("--serve-inflight", type=int, default=8, help="server execution slots")
    return ap.parse_args(argv)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


DTYPES = {"mixed_dd": "f32 inner / f64 refinement, residual transforms in float-pair (~2^-48) arithmetic",
          "mixed": "f32 inner / f64 refinement and residual", "fp64": "f64"}

# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of a kernel class,
# averaged over its launches in one ncu capture of this workload, with the capture it came
# from; reported only for that class, and only while the kernel is unchanged since.
MEASURED_TRAFFIC = {"axis_f32": (229.4e6, "profiles/sections_jet256_mixed_dd.md (capture of commit 1459b41; float axis kernels unchanged since dc550e0)")}


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


def max_over_ranks(t, pg, device):
    """The job's duration is its slowest rank's: max of t over the ranks (t itself at N = 1)."""
    if pg is None:
        return float(t)
    import torch
    tt = torch.tensor([float(t)], dtype=torch.float64, device=device)
    pg.all_reduce(tt, op=pg.ReduceOp.MAX)
    return float(tt.item())


def sum_over_ranks(v, pg, device):
    """Whole-job total of a per-rank quantity (v itself at N = 1)."""
    if pg is None:
        return float(v)
    import torch
    tt = torch.tensor([float(v)], dtype=torch.float64, device=device)
    pg.all_reduce(tt, op=pg.ReduceOp.SUM)
    return float(tt.item())


# ------------------------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
# ------------------------------------------------------------------------------------------

def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


class OracleSolve:
    """The oracle's own CG solve of the full-size workload (its code unmodified; its library FFT
    on `workers` threads).  Set-up (inputs, rhs = div u*, operator closures) is not timed; a
    timed solve covers the range projection of the rhs and the CG iterations.  The operator is
    wrapped to stamp the time of each application: one per iteration after the initial one."""

    def __init__(self, n, workers):
        from oracle import operators as op
        from oracle import spectral as sp
        from paper_2403_06654_gb300 import inputs
        sp.FFT_WORKERS = int(workers)
        self.workers = int(workers)
        case = inputs.jet_3d(n=n)
        self.g = sp.Grid(case.n, case.L)
        self.f = sp.div(list(case.u), self.g)
        self.A, self.M = op.pressure_system(case.rho, self.g)
        self.stamps = []

    def solve(self, tol=1e-10, maxit=500):
        from oracle import solvers as sv
        from oracle import spectral as sp
        self.stamps = []

        def A(p):
            self.stamps.append(time.perf_counter())
            return self.A(p)

        t0 = time.perf_counter()
        r = sv.cg(A, self.M, sp.project_range(self.f, self.g), tol=tol, maxit=maxit)
        t1 = time.perf_counter()
        # the last operator application is _finish's true residual, not an iteration
        return {"seconds": t1 - t0, "iters": r.iters, "status": r.status, "relres_true": r.relres_true}


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
    """The reference arm: the FP64 oracle on the host cores.  A step is one CG iteration of the
    oracle's 256^3 solve; complete solves run back to back until at least `steps` iterations
    are timed, after `warmup` iterations of a discarded solve.  value = complete solves per
    second over the timed solves; ms_per_step = their time per iteration."""
    if rank != 0:
        return 0
    from oracle import spectral as sp
    cores = host_cores()
    orc = OracleSolve(args.n, cores)
    if args.warmup > 0:
        orc.solve(maxit=args.warmup)
    solves, iters = [], 0
    t0 = time.perf_counter()
    while iters < max(args.steps, 1):
        r = orc.solve()
        if r["status"] != "converged":
            raise SystemExit(f"oracle solve failed: {r}")
        solves.append(r)
        iters += r["iters"]
    t = time.perf_counter() - t0
    value = len(solves) / t
    sample = (f"each step: one CG iteration of the oracle's {args.n}^3 solve (complete solves back to back: "
              f"{len(solves)} solves of {solves[0]['iters']} iterations, {t:.1f} s); oracle FFT on {cores} threads "
              f"(scipy.fft workers), numpy elementwise work on 1")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / iters * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": WORKLOAD, "solver": "cg", "precision": "fp64"},
           "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                            "sample": sample, "seconds_per_solve": t / len(solves),
                            "relres_true": solves[0]["relres_true"]},
           "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    sp.FFT_WORKERS = 1
    print(json.dumps(out), flush=True)
    return 0


# ------------------------------------------------------------------------------------------
# secondary workloads (reported beside the headline, outside its timed region)
# ------------------------------------------------------------------------------------------

def extra_tophat1d(dev):
    """1D periodic N = 256 top-hat (r = 3, d = 0.05), 16-mode rhs: CG, GMRES(30), RMR to 1e-12."""
    import numpy as np
    import torch
    import paper_2403_06654_gb300 as vd
    from paper_2403_06654_gb300 import inputs

    n = 256
    G = vd.Grid((n,), (2 * math.pi,), device=dev)
    G.set_density(torch.from_numpy(inputs.tophat_1d(n=n)).to(dev))
    f = torch.from_numpy(inputs.modes_rhs_1d(n=n)).to(dev)
    out = {}
    for solver in ("cg", "gmres", "rmr"):
        kw = dict(tol=1e-12, max_it=400, restart=30, check_every=8)
        x, info = G.solve("pressure", solver, f, **kw)
        ts = []
        for _ in range(30):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            G.solve("pressure", solver, f, out=x, **kw)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e3)
        out[solver] = {"iters": info["iters"], "status": info["status"], "relres": info["relres"],
                       "relres_true": info["relres_true"], "us_per_solve_median": float(np.median(ts))}
    res = {"workload": "1D periodic N=256 top-hat r=3 d=0.05, 16-mode rhs (seed 1), tol 1e-12, x0 = 0",
           "dtype": "f64", "solvers": out}
    # condition numbers of this operator from dense assembly and the oracle's own iteration
    # counts, stored by tests/golden/make_tophat1d.py
    try:
        with open(os.path.join(ROOT, "tests", "golden", "tophat1d.json")) as fh:
            gold = json.load(fh)
        res["dense_assembly"] = {k: gold[k] for k in ("kappa_L", "kappa_left_MA", "kappa_right_AM", "eig_ratio_MA",
                                                      "eig_bound_rho_ratio")}
        res["oracle_iters"] = {k: v["iters"] for k, v in gold["solvers"].items()}
    except (OSError, KeyError, ValueError):
        pass
    return res


def extra_krho(dev, G, rho_d, f, x_l, reps=5):
    """The K_rho form (Sec. 4.2) on the headline 256^3 workload: K~ Phi = sqrt(rho) f to 1e-10,
    phi = sqrt(rho) Phi; solve rate per solver and precision next to the L_rho form."""
    import numpy as np
    import torch
    import paper_2403_06654_gb300 as vd

    n = G.shape
    Gk = vd.Grid(tuple(reversed(n)), G.L, device=dev)
    Gk.set_density(rho_d, op="krho")
    rhs = torch.sqrt(rho_d) * f
    out = {}
    Phi = None
    for solver in ("cg", "gmres"):
        for prec in ("mixed_dd", "fp64"):
            k = reps if prec != "fp64" else 2
            Phi, info = Gk.solve("krho", solver, rhs, tol=1e-10, max_it=500, precision=prec)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(k):
                Phi, info = Gk.solve("krho", solver, rhs, out=Phi, tol=1e-10, max_it=500, precision=prec)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / k
            out[f"{solver}/{prec}"] = {"iters": info["iters"], "status": info["status"],
                                       "relres_true": info["relres_true"], "ms_per_solve": ms,
                                       "solves_per_s": 1e3 / ms}
    phi = torch.sqrt(rho_d) * Phi
    a, b = phi - phi.mean(), x_l - x_l.mean()
    return {"workload": "same 256^3 jet as the headline; K~ Phi = sqrt(rho) f, phi = sqrt(rho) Phi, tol 1e-10",
            "solvers": out,
            "phi_vs_lrho_rel2": float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)),
            "note": ("K~ and L~ are different discretisations of the same equation.  This rhs is the divergence of "
                     "the 1e-3 white noise on a divergence-free base flow, so it lives at the grid scale, where the "
                     "two differ at O(1) (the oracle shows 0.4 relative on a noise-dominated 2D case and 1e-6 for a "
                     "smooth rhs with the same 2-cell interface)")}


def extra_rt2d(dev, steps):
    """2D 512 x 1024 Rayleigh--Taylor-like layer: semi-implicit steps (RMR velocity, GMRES pressure, FP64)."""
    import numpy as np
    import torch
    import paper_2403_06654_gb300 as vd
    from paper_2403_06654_gb300 import inputs

    case = inputs.rt_2d()
    G = vd.Grid(case.n, case.L, device=dev)
    F = vd.Flow(G, Re=case.Re, Sc=case.Sc, Fr=case.Fr, gravity_axis=case.gravity_axis, vel_solver="rmr",
                pres_solver="gmres", tol=1e-10, max_it=200, restart=30)
    F.set_state(torch.from_numpy(case.rho).to(dev), torch.from_numpy(case.u).to(dev))
    for _ in range(2):
        F.step(case.dt)
    F.set_state(torch.from_numpy(case.rho).to(dev), torch.from_numpy(case.u).to(dev))
    infos = []
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        infos.append(F.step(case.dt))
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    rho, u, _, _ = F.state()
    div = G.divergence(u)
    ok = all(i["status"] == "converged" for i in infos)
    return {"workload": "2D 512x1024 RT-like layer (s=3, interface 0.02, eta 0.05 cos, Re=1000, Sc=1, Fr=1, "
                        "dt=1e-3, 1e-3 velocity noise seed 2), RMR velocity + GMRES pressure to 1e-10",
            "dtype": "f64", "steps": steps, "ms_per_step": ms / steps, "all_converged": ok,
            "vel_iters_mean": float(np.mean([i["vel_iters"] for i in infos])),
            "pres_iters_mean": float(np.mean([i["pres_iters"] for i in infos])),
            "pres_iters_first_last": [infos[0]["pres_iters"], infos[-1]["pres_iters"]],
            "div_u_rel": float(torch.linalg.vector_norm(div) / torch.linalg.vector_norm(u)),
            "mass_drift_rel": float(abs(rho.mean().item() - float(np.mean(case.rho))) / float(np.mean(case.rho)))}


# ------------------------------------------------------------------------------------------
# serving: Poisson request stream through the request server
# ------------------------------------------------------------------------------------------

SERVE_VARIANTS = 4   # distinct densities materialised per grid size (cycled over the trace)


class _ServeInputs:
    """Device inputs of a serving trace: per grid size, one band-limited rhs and the densities of
    its first SERVE_VARIANTS trace instances (cycled).  Solutions stay in server memory until
    the client releases them, so nothing is allocated on the submit path."""

    def __init__(self, dev):
        self.dev = dev
        self.rhs, self.dens = {}, {}

    def add(self, trace):
        import torch
        from paper_2403_06654_gb300 import inputs
        dev = self.dev
        for _, inst in trace:
            key = tuple(inst.n)
            if key not in self.rhs:
                self.rhs[key] = torch.from_numpy(inputs.smooth_random_field(inst.n, inst.L, 900 + sum(inst.n),
                                                                            kmax=5)).to(dev)
                self.dens[key] = []
            if len(self.dens[key]) < SERVE_VARIANTS:
                self.dens[key].append(torch.from_numpy(inst.density()).to(dev))

    def take(self, i, inst):
        """Inputs of trace entry i: a function of the entry alone (its size and index), so that the
        served request and the same request solved alone get the same density and rhs."""
        key = tuple(inst.n)
        return self.dens[key][i % len(self.dens[key])], self.rhs[key]


def run_trace(vd, trace, src, max_inflight, precision, solver="cg"):
    """Open-loop: request i is submitted at its arrival time (host monotonic clock) whatever the
    server's state; each completion is polled, recorded and its solution released."""
    import torch
    torch.cuda.synchronize()
    S = vd.vd_server_create(max_inflight=max_inflight, hbm_budget=0)
    pending = {}
    recs = []

    def collect():
        while True:
            got = vd.vd_server_poll(S, 1024)
            if not got:
                return
            for c in got:
                take(c)

    def take(c):
        key, t_sched, tol = pending.pop(int(c.id))
        if c.x:
            vd.vd_server_release(S, int(c.id))
        recs.append({"id": int(c.id), "n": key, "tol": tol, "status": int(c.status), "iters": int(c.iters),
                     "relres_true": float(c.relres_true), "t_sched": t_sched, "t_submit": float(c.t_submit),
                     "t_start": float(c.t_start), "t_done": float(c.t_done)})

    try:
        t0 = time.monotonic() + 0.05
        for i, (ta, inst) in enumerate(trace):
            t_sched = t0 + ta
            while True:
                dt = t_sched - time.monotonic()
                if dt <= 0:
                    break
                collect()
                if dt > 2e-4:
                    time.sleep(min(dt - 1e-4, 1e-3))
            rho, b = src.take(i, inst)
            q = vd.make_request(i, inst.n, inst.L, rho, b, None, solver=solver, tol=inst.tol, max_it=500,
                                precision=precision)
            pending[i] = (tuple(inst.n), t_sched, inst.tol)
            vd.vd_server_submit(S, q, vd.vd_server_request_bytes(q))
        vd.vd_server_drain(S)
        collect()
    finally:
        vd.vd_server_destroy(S)
    return recs, t0


def serve_summary(recs, t0, rate):
    import numpy as np
    lat = np.array([r["t_done"] - r["t_sched"] for r in recs]) * 1e3
    wait = np.array([r["t_start"] - r["t_sched"] for r in recs]) * 1e3
    svc = np.array([r["t_done"] - r["t_start"] for r in recs]) * 1e3
    lag = np.array([r["t_submit"] - r["t_sched"] for r in recs]) * 1e3
    span = max(r["t_sched"] for r in recs) - t0
    makespan = max(r["t_done"] for r in recs) - t0
    big = np.array([r["n"] == (256, 256, 256) for r in recs])
    bad = [r for r in recs if not (r["status"] == 0 and r["relres_true"] <= r["tol"])]
    ok = not bad
    # only requests that reached their tolerance count as served solves
    return {"offered_rate": rate, "requests": len(recs), "solves_per_s": (len(recs) - len(bad)) / makespan,
            "n_failures": len(bad),
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "max": float(lat.max()), "mean": float(lat.mean())},
            "latency_ms_256cubed": ({"p50": float(np.percentile(lat[big], 50)),
                                     "p99": float(np.percentile(lat[big], 99))} if big.any() else None),
            "queue_wait_ms": {"p50": float(np.percentile(wait, 50)), "p99": float(np.percentile(wait, 99))},
            "service_ms": {"p50": float(np.percentile(svc, 50)), "p99": float(np.percentile(svc, 99))},
            "submit_lag_ms_p99": float(np.percentile(lag, 99)),
            "arrival_span_s": span, "makespan_s": makespan,
            "keeps_up": bool(makespan <= 1.1 * span + 1.0), "all_converged": ok,
            "failures": [{k: r[k] for k in ("id", "n", "tol", "status", "iters", "relres_true")} for r in bad[:8]]}


def one_at_a_time(vd, trace, src, precision, dev):
    """The same requests solved one after another on one stream through vd_solve (no server)."""
    import torch
    grids = {}
    torch.cuda.synchronize()
    t = time.perf_counter()
    for i, (_, inst) in enumerate(trace):
        key = tuple(inst.n)
        if key not in grids:
            grids[key] = vd.Grid(inst.n, inst.L, device=dev)
        G = grids[key]
        rho, b = src.take(i, inst)
        G.set_density(rho)
        _, info = G.solve("pressure", "cg", b, tol=inst.tol, max_it=500, precision=precision)
        if info["status"] != "converged":
            raise SystemExit(f"one-at-a-time solve failed: {info}")
    torch.cuda.synchronize()
    return len(trace) / (time.perf_counter() - t)


def run_serving(vd, dev, count, rate, max_inflight, sweep=(), baseline_count=200, precision="mixed_dd"):
    """Poisson trace (mean `rate` req/s) of pressure solves, 95% from the batched-instance size mix
    and 5% 256^3, tolerances 1e-6 / 1e-8 / 1e-10 uniform, served open-loop; plus the first
    `baseline_count` requests solved one at a time in FP64 and in the serving precision, and the
    same requests submitted all at once to the server."""
    from paper_2403_06654_gb300 import inputs
    trace = inputs.serving_trace(count=count, rate=rate)
    # each sweep point: about 4 s of arrivals
    sweep_traces = [(r, inputs.serving_trace(count=int(min(count, max(500, 4 * r))), rate=r)) for r in sweep]
    src = _ServeInputs(dev)
    src.add(trace)
    for _, tr in sweep_traces:
        src.add(tr)
    # warm-up: every worker meets most grid sizes; pools and plans are built outside the timed trace
    warm = sorted({tuple(inst.n): (0.0, inst) for _, inst in trace}.values(), key=lambda p: p[1].n)
    run_trace(vd, [(0.0, inst) for _ in range(max_inflight) for _, inst in warm], src, max_inflight, precision)
    recs, t0 = run_trace(vd, trace, src, max_inflight, precision)
    out = serve_summary(recs, t0, rate)
    out["max_inflight"] = max_inflight
    out["precision"] = precision
    if sweep:
        rows = []
        for r, tr in sweep_traces:
            rr, t0r = run_trace(vd, tr, src, max_inflight, precision)
            s = serve_summary(rr, t0r, r)
            rows.append({k: s[k] for k in ("offered_rate", "requests", "solves_per_s", "latency_ms", "keeps_up",
                                           "makespan_s", "all_converged")})
        out["rate_sweep"] = rows
        kept = [row["offered_rate"] for row in rows if row["keeps_up"]]
        out["sustainable_rate"] = max(kept) if kept else None
    base = trace[:baseline_count]
    out["one_at_a_time"] = {"requests": len(base),
                            "fp64_solves_per_s": one_at_a_time(vd, base, src, "fp64", dev),
                            precision + "_solves_per_s": one_at_a_time(vd, base, src, precision, dev)}
    # the same requests all at once through the server (its capacity on this mix)
    rb, t0b = run_trace(vd, [(0.0, inst) for _, inst in base], src, max_inflight, precision)
    out["one_at_a_time"]["server_all_at_once_solves_per_s"] = len(rb) / (max(r["t_done"] for r in rb) - t0b)
    return out


BATCH_WORKLOAD = ("96 uneven instances (seed 4): 2D 64..512^2 / 3D 32..160^3, slab density ratio 2..50 "
                  "log-uniform, interface 3 cells; per instance the coupled velocity system (a = 1e-3, Sc = 1, "
                  "GMRES(30)) and the pressure system (CG), tol 1e-10, x0 = 0; band-limited rhs")


def run_batch(vd, dev, count=96, tol=1e-10, reps=2, precision="mixed_dd"):
    """All solves of the batch in one graph launch vs the same solves one at a time through vd_solve."""
    import numpy as np
    import torch
    from paper_2403_06654_gb300 import inputs
    insts = inputs.batch_instances(count=count)
    items = []
    for i, inst in enumerate(insts):
        nd = len(inst.n)
        rho = torch.from_numpy(inst.density()).to(dev)
        bp = torch.from_numpy(inputs.smooth_random_field(inst.n, inst.L, 300 + i, kmax=5)).to(dev)
        bv = torch.from_numpy(np.stack([inputs.smooth_random_field(inst.n, inst.L, 400 + 3 * i + c, kmax=5)
                                        for c in range(nd)])).to(dev)
        items.append({"n": inst.n, "L": inst.L, "rho": rho, "a": 1e-3, "inv_sc": 1.0, "b_vel": bv,
                      "x_vel": torch.zeros_like(bv), "b_pres": bp, "x_pres": torch.zeros_like(bp)})
    t0 = time.perf_counter()
    B = vd.Batch(items, vel_solver="gmres", pres_solver="cg", tol=tol, max_it=500, restart=30, precision=precision,
                 device=dev)
    t_build = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    B.run()   # warm-up
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    l0 = vd.vd_launch_count()
    ev[0].record(stream)
    for _ in range(reps):
        B.run(stream)
    ev[1].record(stream)
    torch.cuda.synchronize()
    host_launches = vd.vd_launch_count() - l0
    t_graph = ev[0].elapsed_time(ev[1]) / 1e3 / reps
    infos = [B.info(i) for i in range(count)]
    ok = all(v["status"] == "converged" and p["status"] == "converged" for v, p in infos)
    nodes = B.graph_nodes()
    B.close()
    # the same solves one at a time (host-driven loop), with the profiler for algorithmic bytes
    vd.vd_profile_reset()
    vd.vd_profile_enable(True)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for it in items:
        G = vd.Grid(it["n"], it["L"], device=dev)
        G.set_density(it["rho"], op="velocity")
        G.solve("velocity", "gmres", it["b_vel"], a=1e-3, inv_sc=1.0, out=it["x_vel"], tol=tol, max_it=500,
                precision=precision)
        G.solve("pressure", "cg", it["b_pres"], out=it["x_pres"], tol=tol, max_it=500, precision=precision)
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t1
    vd.vd_profile_enable(False)
    prof = {c: vd.vd_profile_read(c) for c in vd.PROFILE_CLASSES}
    alg_bytes = sum(p["alg_bytes"] for p in prof.values())
    ncomp = sum(len(it["n"]) + 1 for it in items)
    return {"workload": BATCH_WORKLOAD, "precision": precision, "instances": count, "systems": 2 * count,
            "component_solves": ncomp,
            "graph_launches_per_run": 1, "host_kernel_launches_per_run": host_launches // reps,
            "graph_nodes_top_level": nodes, "build_s": t_build,
            "graph_s_per_run": t_graph, "systems_per_s": 2 * count / t_graph,
            "component_solves_per_s": ncomp / t_graph,
            "one_at_a_time_s": t_seq, "one_at_a_time_systems_per_s": 2 * count / t_seq,
            "graph_speedup": t_seq / t_graph,
            "alg_bytes_per_run": alg_bytes, "alg_gbs": alg_bytes / t_graph / 1e9,
            "vel_iters": [v["iters"] for v, _ in infos], "pres_iters": [p["iters"] for _, p in infos],
            "max_relres_true": max(max(v["relres_true"], p["relres_true"]) for v, p in infos),
            "all_converged": ok}


SERVE_WORKLOAD = ("Poisson arrivals (seed 5) of pressure solves: 95% batched-instance mix (2D 64..512^2, "
                  "3D 32..160^3, slab density ratio 2..50 log-uniform, interface 3 cells), 5% 256^3; "
                  "tol 1e-6/1e-8/1e-10 uniform; CG, x0 = 0; open-loop submission")


def serve_line(args, vd, dev, rank, world, pg):
    """The serving line: the full trace at the configured rate, a rate sweep, and one-at-a-time runs."""
    count = args.serve_count or 20000
    sampler = ClockSampler(dev.index)
    sampler.start()
    l0 = vd.vd_launch_count()
    s = run_serving(vd, dev, count, args.serve_rate, args.serve_inflight,
                    sweep=(100.0, 150.0, 200.0, 250.0, 500.0, 1000.0, 2000.0), baseline_count=200)
    launches = vd.vd_launch_count() - l0
    clocks = sampler.stop()
    value = sum_over_ranks(s["solves_per_s"], pg, dev)
    out = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": s["requests"],
           "warmup": args.serve_inflight, "ms_per_step": 1e3 / max(value, 1e-9), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": DTYPES["mixed_dd"], "data": "synthetic",
           "config": {"workload": SERVE_WORKLOAD, "requests": count, "rate": args.serve_rate,
                      "max_inflight": args.serve_inflight, "parallelism": f"replicas x{world}",
                      "l2": "mixed: small requests are L2-resident, 256^3 inputs exceed L2"},
           "latency_ms": s["latency_ms"], "serving": s, "gpu_launches": int(launches), "clocks": clocks,
           "mode": "serve"}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if pg is not None:
        pg.barrier()
        pg.destroy_process_group()
    return 0


def cufft_compare(vd, G, dev, reps=20):
    """Plain 3D real transforms of the headline grid: the library's passes (vd_fft_r2c /
    vd_fft_c2r) next to cuFFT (torch.fft.rfftn / irfftn, a comparison baseline outside the
    product path), double and float, CUDA events over `reps` back-to-back launches each."""
    import torch
    shape = G.shape
    out = {}
    g = torch.Generator(device=dev)
    g.manual_seed(11)
    x64 = torch.randn(shape, dtype=torch.float64, device=dev, generator=g)
    for prec, x in (("fp64", x64), ("mixed", x64.float())):
        xh = G.fft_r2c(x, prec)
        back = G.fft_c2r(xh, prec)
        ref = torch.fft.rfftn(x)
        bref = torch.fft.irfftn(ref, s=shape)
        rel = float(torch.linalg.vector_norm(xh - ref) / torch.linalg.vector_norm(ref))

        def timed(fn):
            fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                fn()
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps

        t = {"ours_r2c_ms": timed(lambda: G.fft_r2c(x, prec, out=xh)),
             "ours_c2r_ms": timed(lambda: G.fft_c2r(xh, prec, out=back)),
             "cufft_r2c_ms": timed(lambda: torch.fft.rfftn(x)),
             "cufft_c2r_ms": timed(lambda: torch.fft.irfftn(ref, s=shape))}
        t["r2c_ours_over_cufft"] = t["ours_r2c_ms"] / t["cufft_r2c_ms"]
        t["c2r_ours_over_cufft"] = t["ours_c2r_ms"] / t["cufft_c2r_ms"]
        t["rel_diff_vs_cufft"] = rel
        t["dtype"] = "f64" if prec == "fp64" else "f32"
        out[t["dtype"]] = t
        del xh, back, ref, bref
    out["grid"] = list(reversed(shape))
    out["note"] = ("cuFFT via torch.fft (comparison only, never on the solve path); ours = the x, y and z "
                   "passes of the library, three HBM round trips per 3D transform")
    return out


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
    if args.mode == "serve":
        return serve_line(args, vd, dev, rank, world, pg)
    if args.mode == "batch":
        res = run_batch(vd, dev, precision="mixed_dd")
        res64 = run_batch(vd, dev, precision="fp64", reps=1)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "mode": "batch", "value": res["systems_per_s"], "unit": "systems/s",
                              "n_gpus": world, "higher_is_better": True, "dtype": DTYPES["mixed_dd"],
                              "data": "synthetic", "config": {"workload": BATCH_WORKLOAD}, "batch": res,
                              "batch_fp64": res64}), flush=True)
        return 0
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

    def solve(prec, dst=None):
        _, info = G.solve("pressure", args.solver, f, out=x if dst is None else dst, precision=prec, **kw)
        if info["status"] != "converged" or not (info["relres_true"] <= args.tol):
            raise SystemExit(f"solve failed: {info}")
        return info

    # every timed headline solve writes a buffer of its own, checked after the timed region
    xs = [torch.empty_like(f) for _ in range(args.steps)]

    head = args.precision
    side = "mixed" if head == "mixed_dd" else "mixed_dd"
    tuned = None
    if not args.no_autotune:
        t_tune = time.perf_counter()
        vd.vd_autotune(G, ("fp64", "mixed", "mixed_dd"))
        tuned = {"seconds": time.perf_counter() - t_tune,
                 "table": [e for e in vd.vd_autotune_table() if e[2] in (n, n // 2)]}
    # warm-up
    for _ in range(args.warmup):
        solve(head)
    solve(side)
    solve("fp64")

    # ---------------- timed: headline precision (no instrumentation) ----------------
    sampler = ClockSampler(local)
    l0 = vd.vd_launch_count()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    barrier()
    sampler.start()
    infos = []
    nvtx = getattr(torch.cuda, "nvtx", None)
    if nvtx is not None:
        nvtx.range_push("timed")   # lets a profiler select exactly the timed solves
    ev[0].record(stream)
    for k in range(args.steps):
        infos.append(solve(head, xs[k]))
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    if nvtx is not None:
        nvtx.range_pop()
    barrier()
    clocks = sampler.stop()
    launches = vd.vd_launch_count() - l0
    lat = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    t_mixed = ev[0].elapsed_time(ev[args.steps]) / 1e3

    # ---------------- the same solves again, every kernel bracketed by CUDA events ----------------
    # (per-kernel durations for the roofline and the kernel classes; the events themselves cost
    # a few percent of the step, so the headline above is taken without them)
    vd.vd_profile_reset()
    vd.vd_profile_enable(True)
    evp = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    evp[0].record(stream)
    infos_prof = [solve(head) for _ in range(args.steps)]
    evp[1].record(stream)
    torch.cuda.synchronize()
    vd.vd_profile_enable(False)
    t_prof = evp[0].elapsed_time(evp[1]) / 1e3
    prof = {c: vd.vd_profile_read(c) for c in vd.PROFILE_CLASSES}

    # ---------------- and once more in span mode: each inner float solve timed as a whole ----------------
    # (two events per inner solve instead of two per kernel: the per-iteration figure below)
    vd.vd_profile_reset()
    vd.vd_profile_enable(2)
    infos_span = [solve(head) for _ in range(args.steps)]
    torch.cuda.synchronize()
    vd.vd_profile_enable(0)
    span = vd.vd_profile_read(vd.PROFILE_SPAN_INNER_F32)
    t_mixed = max_over_ranks(t_mixed, pg, dev)

    # double-precision check of every timed headline solution (outside the timed region): the
    # residual through the library's FP64 operator; the rhs of this workload is the divergence
    # of a velocity, whose only null-space content is the mean
    fmean = f - f.mean()
    fnorm = float(torch.linalg.vector_norm(fmean))
    verified_all = []
    for xk in xs:
        r64 = f - G.apply("pressure", xk)
        r64 = r64 - r64.mean()
        verified_all.append(float(torch.linalg.vector_norm(r64)) / fnorm)
    verified = max(verified_all)
    del xs

    # ---------------- timed: the other mixed mode ----------------
    ev3 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    barrier()
    ev3[0].record(stream)
    infos_side = [solve(side) for _ in range(args.side_steps)]
    ev3[1].record(stream)
    torch.cuda.synchronize()
    barrier()
    t_side = max_over_ranks(ev3[0].elapsed_time(ev3[1]) / 1e3, pg, dev)

    # ---------------- timed: plain FP64 ----------------
    ev2 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    barrier()
    ev2[0].record(stream)
    infos64 = [solve("fp64") for _ in range(args.fp64_steps)]
    ev2[1].record(stream)
    torch.cuda.synchronize()
    barrier()
    t64 = ev2[0].elapsed_time(ev2[1]) / 1e3
    t64 = max_over_ranks(t64, pg, dev)

    # ---------------- end to end through host buffers ----------------
    # Every step copies its rho and f from pinned host memory, sets the density up, solves and
    # copies phi back.  The copies run on a copy stream, double-buffered, so that step k+1's
    # inputs arrive and step k-1's result leaves while step k solves (the H2D/D2H link and the
    # SMs work at the same time, as a serving loop would use them).
    rho_h = rho_d.cpu().pin_memory()
    f_h = f.cpu().pin_memory()
    x_h = [torch.empty_like(f_h).pin_memory() for _ in range(2)]
    rho_e = [torch.empty_like(rho_d) for _ in range(2)]
    f_e = [torch.empty_like(f) for _ in range(2)]
    x_e = [torch.empty_like(f) for _ in range(2)]
    cs = torch.cuda.Stream(device=dev)
    in_ready = [torch.cuda.Event() for _ in range(2)]
    out_done = [torch.cuda.Event() for _ in range(2)]
    solved = [torch.cuda.Event() for _ in range(2)]

    def h2d(k):
        b = k % 2
        with torch.cuda.stream(cs):
            rho_e[b].copy_(rho_h, non_blocking=True)
            f_e[b].copy_(f_h, non_blocking=True)
            in_ready[b].record(cs)

    barrier()
    t0 = time.perf_counter()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    cs.wait_event(e0)
    h2d(0)
    for k in range(args.e2e_steps):
        b = k % 2
        if k + 1 < args.e2e_steps:
            h2d(k + 1)   # buffers (k+1) % 2 were last read by solve k-1, which has returned
        stream.wait_event(in_ready[b])
        if k >= 2:
            stream.wait_event(out_done[b])   # x_e[b] still leaving for step k-2
        G.set_density(rho_e[b])
        _, info = G.solve("pressure", args.solver, f_e[b], out=x_e[b], precision=head, **kw)
        if info["status"] != "converged":
            raise SystemExit(f"e2e solve failed: {info}")
        solved[b].record(stream)
        with torch.cuda.stream(cs):
            cs.wait_event(solved[b])
            x_h[b].copy_(x_e[b], non_blocking=True)
            out_done[b].record(cs)
    stream.wait_stream(cs)
    e1.record(stream)
    torch.cuda.synchronize()
    x_h = x_h[0]
    t_e2e = e0.elapsed_time(e1) / 1e3
    wall_e2e = time.perf_counter() - t0
    t_e2e = max_over_ranks(t_e2e, pg, dev)

    # ---------------- roofline of the dominant kernel class ----------------
    pk, pk_src = peaks()
    alu = {"fp64_tflops": vd.vd_alu_rate(0) / 1e12, "fp32_tflops": vd.vd_alu_rate(1) / 1e12,
           "float_pair_tflops": vd.vd_alu_rate(2) / 1e12,
           "how": "vd_alu_rate: independent FMA (float-pair: multiply + add) chains, 8 blocks x 256 threads per "
                  "SM, best of three launches; an FMA or a float-pair multiply-add counts 2 flops"}
    # per inner (float) Krylov iteration: float passes + float vector kernels.  Primary: the
    # span pass (each inner solve between two events: host gaps included, no per-kernel events);
    # beside it the sum of the per-kernel event durations of the instrumented pass.
    n_inner = sum(i["iters"] for i in infos_prof)
    f32c = [c for c in prof if vd.PROFILE_CLASSES[c] in ("axis_f32", "xpass_f32", "vec_f32")]
    k_ms = sum(prof[c]["ms"] for c in f32c) / max(n_inner, 1)
    k_bytes = sum(prof[c]["alg_bytes"] for c in f32c) / max(n_inner, 1)
    n_span = sum(i["iters"] for i in infos_span)
    it_ms = span["ms"] / max(n_span, 1)
    it_bytes = span["alg_bytes"] / max(n_span, 1)
    per_iter = {"ms": it_ms, "alg_bytes": it_bytes, "achieved_gbs": it_bytes / (it_ms / 1e3) / 1e9,
                "frac_of_hbm": it_bytes / (it_ms / 1e3) / 1e9 / pk["hbm_gbs"],
                "iterations": n_span, "inner_solves": span["launches"],
                "includes": "whole inner float CG solves (transform passes, vector kernels, host gaps) "
                            "between two CUDA events each, divided by their iterations",
                "from_kernel_events": {"ms": k_ms, "alg_bytes": k_bytes,
                                       "frac_of_hbm": k_bytes / (k_ms / 1e3) / 1e9 / pk["hbm_gbs"],
                                       "note": "sum of per-kernel event durations (each inflated by the "
                                               "events around it)"}}
    dom = max((c for c in prof if c != 4), key=lambda c: prof[c]["ms"])
    d = prof[dom]
    name = vd.PROFILE_CLASSES[dom]
    per_launch_ms = d["ms"] / max(d["launches"], 1)
    if name.endswith("f32"):
        achieved = d["alg_bytes"] / (d["ms"] / 1e3) / 1e9
        tr = MEASURED_TRAFFIC.get(name)
        roof = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / pk["hbm_gbs"], "traffic": tr[0] if tr else None,
                "traffic_source": tr[1] if tr else None,
                "peak_source": f"{pk_src} hbm_gbs (MEASURED_PEAKS.json)" if pk_src == "measured" else "fallback",
                "alg_bytes_per_launch": d["alg_bytes"] / max(d["launches"], 1), "ms_per_launch": per_launch_ms}
    else:
        achieved = d["alg_flops"] / (d["ms"] / 1e3) / 1e12
        pk_alu = alu["fp64_tflops"] if name.endswith("f64") else alu["float_pair_tflops"]
        roof = {"bound": "alu", "kernel": name, "achieved": achieved, "peak": pk_alu, "unit": "TFLOP/s",
                "frac": achieved / pk_alu, "traffic": None,
                "peak_source": "measured in this run by vd_alu_rate (" +
                               ("FP64 FMA" if name.endswith("f64") else "float-pair multiply-add") + ")",
                "alg_flops_per_launch": d["alg_flops"] / max(d["launches"], 1), "ms_per_launch": per_launch_ms,
                "hbm_gbs_achieved": d["alg_bytes"] / (d["ms"] / 1e3) / 1e9}
    classes = {vd.PROFILE_CLASSES[c]: {"launches": prof[c]["launches"], "ms": prof[c]["ms"],
                                       "GB/s": prof[c]["alg_bytes"] / max(prof[c]["ms"], 1e-9) / 1e6}
               for c in prof}

    # ---------------- secondary workloads ----------------
    extras = None
    if not args.no_extras:
        extras = {"tophat1d": extra_tophat1d(dev), "rt2d": extra_rt2d(dev, args.rt_steps),
                  "krho256": extra_krho(dev, G, rho_d, f, x), "cufft": cufft_compare(vd, G, dev)}

    batch = None
    if not args.no_batch:
        batch = run_batch(vd, dev, precision="mixed_dd")
        batch = {k: v for k, v in batch.items() if k not in ("vel_iters", "pres_iters")}
    serving = None
    if not args.no_serve:
        serving = run_serving(vd, dev, args.serve_count or 2000, args.serve_rate, args.serve_inflight)

    # ---------------- CPU oracle baseline (rank 0, N = 1) ----------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = host_cores()
        orc = OracleSolve(n, cores)
        r = orc.solve(tol=args.tol)
        t_it1 = None
        try:
            from oracle import spectral as osp
            osp.FFT_WORKERS = 1
            t_it1 = oracle_iteration_seconds(n)
        finally:
            osp.FFT_WORKERS = 1
        cpu = {"value": 1.0 / r["seconds"], "unit": "solves/s", "cores": cores, "kind": "oracle",
               "sample": (f"one complete oracle CG solve of this {n}^3 workload to {args.tol:g} ({r['iters']} "
                          f"iterations, {r['seconds']:.1f} s, true relres {r['relres_true']:.2e}); library FFT on "
                          f"{cores} threads, numpy elementwise work on 1"),
               "seconds_per_solve": r["seconds"], "iters": r["iters"],
               "one_thread_seconds_per_iteration": t_it1}

    total_solves = args.steps * world
    value = total_solves / t_mixed
    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_mixed / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[head], "data": "synthetic",
        "config": {"workload": WORKLOAD, "solver": args.solver, "precision": head, "tol": args.tol,
                   "grid": [n, n, n], "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (each 256^3 field 134 MB; working set ~1.6 GB)",
                   "launch_shapes": "autotuned before the timed region" if tuned else "built-in"},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "mean": float(np.mean(lat))},
        "iters": infos[-1]["iters"], "outer_iters": infos[-1]["outer_iters"],
        "relres_true_max": max(i["relres_true"] for i in infos),
        "relres_fp64_check": verified,
        "relres_fp64_check_note": "max over every timed solve of the residual through the FP64 operator",
        "alu_rates": alu,
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
                "includes": "H2D of rho and f from pinned host memory, density setup, solve, D2H of phi; "
                            "copies on a copy stream, double-buffered, overlapping the neighbouring steps' solves"},
        "gpu_launches": int(launches),
        "roofline": roof,
        "per_iteration": per_iter,
        "kernel_classes": classes,
        "profiled_pass": {"steps": args.steps, "ms_per_step": t_prof / args.steps * 1e3,
                          "note": "roofline and kernel_classes come from this second pass of the same solves "
                                  "with CUDA events around every kernel; per_iteration from a third pass with "
                                  "events around each inner solve only"},
        "clocks": clocks,
        "cpu_baseline": cpu,
        "workloads": extras,
        "serving": serving,
        "batch": batch,
        "autotune": tuned,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    if pg is not None:
        pg.barrier()
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
