#!/usr/bin/env python3
"""Throughput of the per-step hot path on one GB300.

Workload: the 4 x 4 x 1 mm block as one degree-2 B-spline patch with
64 x 64 x 16 elements (78,408 control points, 36,864 lateral and 36,864
bottom quadrature points), a 20-track meander (3.5 mm tracks, 0.1 mm hatch,
P = 250 W, v = 1.2 m/s, dt = 5 us, theta = 0.5), full history kept.  The
timed steps start mid-scan (step 5,840: the 10-track point, where a step
costs the average step of the whole scan, since the active source count
grows by one per step).

A "step" is one theta-step of the whole hot path: source coefficients,
history sums at every boundary quadrature point, boundary integrals, bottom
projection, theta right-hand side, PCG.  ``value`` is theta-steps/s of the
mixed path (FP32 history sum and operator values; FP64 state, boundary
integrals and Krylov vectors; the block's faces are axis-aligned rectangles,
so the history sums are evaluated separably, as matrix products over the
sources; fast-diagonalization preconditioners, solves started from T^n),
replayed as CUDA graphs (16 steps per graph) with the inputs resident in
HBM.  Timed beside it: the same path with extrapolated initial guesses, with
the Jacobi preconditioner, with the pairwise history sums, the plain FP64
path (pairwise sums) and FP64 with the separable sums.  Also in the line:
the plate with a hole, the 256-instance batched sweep, the learned warm
start, and the heat-loss diagnostic of Sections 3.1-3.2 (integrated |q~ +
q^| along the top arc of the quarter-cylinder part, single source and
contour scan, on two meshes).

``--impl reference`` times the FP64 CPU oracle (the reference arm) on a
bounded sample of the same step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "point-source evals/s and θ-steps/s, mixed+learned vs plain FP64, one GB300"
UNIT = "theta-steps/s"
START_STEP = 5840
N_MONITOR = 64


def start_step(args):
    if args.start_step is not None:
        return args.start_step
    return max(0, START_STEP - args.steps // 2 - args.warmup)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--hist", default="auto", choices=["auto", "pairwise", "separable"],
                    help="evaluation of the history sums of the main context")
    ap.add_argument("--start-step", type=int, default=None,
                    help="first timed step; default: the timed steps are centred on step 5,840")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"],
                    help="path timed in the main region")
    ap.add_argument("--guess", default="previous", choices=["extrapolate", "previous"],
                    help="initial guess of the theta-step solves in the main region")
    ap.add_argument("--batch-steps", type=int, default=2000,
                    help="theta-steps of the 256-instance batched leg (0: skip the leg)")
    ap.add_argument("--batch-instances", type=int, default=256,
                    help="instances of the batched leg (256: the sweep; fewer for profiling)")
    ap.add_argument("--learned-pairs", type=int, default=2000,
                    help="training pairs of the learned warm-start leg (0: skip the leg)")
    ap.add_argument("--learned-epochs", type=int, default=20)
    ap.add_argument("--legs", default="all",
                    help="comma list of the legs after the main timed region to run: stages, "
                         "variants, cutoff, e2e, batched, plate, lasers, arc, learned, cpu (default all; the "
                         "form used for profiling one leg)")
    ap.add_argument("--quick", action="store_true",
                    help="main timed region only (no stage, FP64, e2e or CPU legs): "
                         "the form used under ncu")
    return ap.parse_args()


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def shard(n, rank, world):
    """Contiguous share [lo, hi) of n independent units (instances) for one
    rank; the first n % world ranks take one more.  No unit is shared, so the
    ranks need no collective on the data path."""
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def max_over_ranks(value, dist, device="cpu"):
    """The largest of the ranks' values (the job's time: the slowest rank)."""
    return _reduce_ranks(value, dist, device, "MAX")


def sum_over_ranks(value, dist, device="cpu"):
    """The sum of the ranks' values (work done by the whole job)."""
    return _reduce_ranks(value, dist, device, "SUM")


def _reduce_ranks(value, dist, device, op):
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=getattr(dist.ReduceOp, op))
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
CLOCK_Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def clocks_start(dev):
    f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    try:
        p = subprocess.Popen(["nvidia-smi", f"--query-gpu={CLOCK_Q}", "--format=csv,noheader,nounits",
                              "-lms", "50", "-i", str(dev)], stdout=f, stderr=subprocess.DEVNULL)
    except OSError:
        p = None
    return p, f.name


def clocks_stop(h):
    p, path = h
    if p is not None:
        p.terminate()
        try:
            p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            p.kill()
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    try:
        for line in open(path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(path)
    except OSError:
        pass
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
            "samples": len(sm)}


def profile_traffic(name, src):
    """DRAM bytes per launch from the committed ncu summary profiles/<name>.md,
    or None when the kernel source changed since that capture."""
    import hashlib
    try:
        text = open(os.path.join(ROOT, "profiles", name + ".md")).read()
        sha = hashlib.sha256(open(os.path.join(ROOT, "paper_2511_20432_gb300", "csrc", src), "rb").read()).hexdigest()
    except OSError:
        return None
    vals = dict(l.split(":", 1) for l in text.splitlines() if l.startswith(("source_sha256:", "dram_bytes_per_launch:")))
    if vals.get("source_sha256", "").strip() != sha:
        return None
    return float(vals["dram_bytes_per_launch"])


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


# ---------------------------------------------------------------------------
# The oracle as it stands, on the host cores (the reference arm and the
# cpu_baseline leg): the history sums of whole steps, split by boundary point
# over worker processes (spawn: the parent may already hold a CUDA context),
# and whole oracle steps (history, boundary load, projection, LU solve) of
# the 2 x 1 x 0.5 mm cuboid.
# ---------------------------------------------------------------------------
_OW = {}


def _ow_init(lat_x, lat_n, bot_x, E, mat):
    _OW.update(lat_x=lat_x, lat_n=lat_n, bot_x=bot_x, E=E, mat=mat)


def _ow_part(args):
    from oracle import pointsource
    kind, q0, q1, stride, xs, age = args
    sl = slice(q0, q1, stride)
    if kind == "lat":
        return pointsource.dTdn_tilde(_OW["lat_x"][sl], _OW["lat_n"][sl], xs, age, _OW["E"],
                                      _OW["mat"])
    return pointsource.T_tilde(_OW["bot_x"][sl], xs, age, _OW["E"], _OW["mat"])


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def host_cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


class OracleHistory:
    """The oracle's history sums (dT~/dn at the lateral points, T~ at the
    bottom points) of one step of a workload, every ``stride``-th point of
    each list, on ``procs`` worker processes."""

    def __init__(self, wl, procs):
        import multiprocessing as mp
        from oracle import assembly, sources
        from oracle.geometry import PatchGeom
        from oracle.solver import FACE_DIRICHLET, FACE_NEUMANN
        self.wl = wl
        g = PatchGeom(wl.patch)
        self.lat = assembly.boundary_points(g, FACE_NEUMANN)
        self.bot = assembly.boundary_points(g, FACE_DIRICHLET)
        self.xs = sources.discretize(wl.scan, wl.dt)
        self.E = sources.energy(wl.scan, wl.dt)
        self.procs = procs
        self.q = len(self.lat["x"]) + len(self.bot["x"])
        self.pool = mp.get_context("spawn").Pool(
            procs, _ow_init, (self.lat["x"], self.lat["n"], self.bot["x"], self.E, wl.material))

    def close(self):
        self.pool.close()
        self.pool.join()

    def _tasks(self, n, stride, parts):
        from oracle import pointsource
        K = min(n, len(self.xs))
        xs, age = self.xs[:K], pointsource.ages(n, K, self.wl.dt, self.wl.material,
                                                self.wl.scan.spot_radius)
        tasks, pts = [], 0
        for kind, Q in (("lat", len(self.lat["x"])), ("bot", len(self.bot["x"]))):
            cuts = [int(Q * k / parts) // stride * stride for k in range(parts)] + [Q]
            for a, b in zip(cuts[:-1], cuts[1:]):
                if b > a:
                    tasks.append((kind, a, b, stride, xs, age))
                    pts += len(range(a, b, stride))
        return tasks, pts, K

    def step(self, n, stride=1):
        """Evaluate step n on the pool; returns (seconds, points, pairs)."""
        tasks, pts, K = self._tasks(n, stride, 4 * self.procs)
        t0 = time.perf_counter()
        self.pool.map(_ow_part, tasks)
        return time.perf_counter() - t0, pts, pts * K

    def step_single(self, n, stride):
        """The same in this process alone (one core)."""
        tasks, pts, K = self._tasks(n, stride, 1)
        t0 = time.perf_counter()
        _ow_init(self.lat["x"], self.lat["n"], self.bot["x"], self.E, self.wl.material)
        for t in tasks:
            _ow_part(t)
        return time.perf_counter() - t0, pts, pts * K


def oracle_whole_steps_cuboid():
    """Whole oracle theta-steps (history sums, boundary load, bottom
    projection, sparse-LU theta solve) of the 2 x 1 x 0.5 mm cuboid, all 150
    steps of its track, one core; set-up (assembly, factorisation) apart."""
    import workloads as W
    from oracle.solver import Model
    wl = W.cuboid_single_track(theta=0.5, n_steps=150)
    t0 = time.perf_counter()
    m = Model(wl)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    m.run(wl.n_steps)
    t_run = time.perf_counter() - t0
    return {"workload": wl.name, "steps": wl.n_steps, "setup_s": t_setup, "run_s": t_run,
            "steps_per_s": wl.n_steps / t_run, "cores": 1,
            "what": "whole oracle steps: history sums, boundary load, projection, LU solve"}

def block_config(wl, n0, n_first):
    """The workload keys shared by both arms' lines (same dict in each)."""
    n_el = [len(set(k)) - 1 for k in wl.patch.knots]
    q_lat = 2 * 9 * (n_el[0] + n_el[1]) * n_el[2]
    q_bot = 9 * n_el[0] * n_el[1]
    return {"workload": wl.name + f" mid-scan from step {n0}", "n_dof": wl.patch.n_dof,
            "q_lat": q_lat, "q_bot": q_bot, "active_sources_first": n_first,
            "theta": wl.theta, "dt": wl.dt}


def oracle_history_timing(wl, n_first, steps, warmup, budget_s, single_s=4.0):
    """Time the oracle's history sums of ``steps`` consecutive steps from
    step n_first (after ``warmup`` untimed ones) on all host cores; each step
    evaluates every stride-th boundary point, the stride chosen so that the
    timed and warm-up steps take about ``budget_s`` (stride 1 = whole steps).
    Also one core on a sample of about ``single_s`` seconds."""
    import math
    import statistics as stt
    procs = host_cores()
    t0 = time.perf_counter()
    oh = OracleHistory(wl, procs)
    t_setup = time.perf_counter() - t0
    try:
        dt_c, pts_c, _ = oh.step(n_first, 64)              # calibration
        per_step = budget_s / max(1, steps + warmup)
        stride = max(1, math.ceil(oh.q * (dt_c / pts_c) / per_step))
        for i in range(warmup):
            oh.step(n_first - warmup + i, stride)
        ts, pts, pairs = [], 0, 0
        for i in range(steps):
            t, p, pr = oh.step(n_first + i, stride)
            ts.append(t)
            pts += p
            pairs += pr
        n_mid = n_first + steps // 2
        stride1 = max(stride, math.ceil(oh.q * (dt_c / pts_c) * procs / single_s))
        t1, p1, pr1 = oh.step_single(n_mid, stride1)
    finally:
        oh.close()
    frac = pts / (steps * oh.q)
    ms = 1e3 * stt.mean(ts)
    return {"procs": procs, "setup_s": t_setup, "stride": stride, "points_per_step": pts // steps,
            "points_whole_step": oh.q, "ms_per_sampled_step": ms,
            "steps_per_s": frac / (ms / 1e3), "pairs_per_s": pairs / sum(ts),
            "single_thread": {"stride": stride1, "points": p1, "s": t1, "pairs_per_s": pr1 / t1,
                              "steps_per_s": (p1 / oh.q) / t1}}


def _sample_text(h, n_first):
    whole = "whole steps" if h["stride"] == 1 else (
        f"every {h['stride']}-th boundary point ({h['points_per_step']} of "
        f"{h['points_whole_step']}) per step, scaled to whole steps")
    return (f"oracle history sums (dT~/dn at every lateral point, T~ at every bottom point, all "
            f"active sources) of consecutive steps from step {n_first}: {whole}, on "
            f"{h['procs']} worker processes; the boundary load, the projection and the theta "
            "solve are not in it (whole oracle steps of the 2 x 1 x 0.5 mm cuboid, solve "
            "included, are reported beside it)")


def run_reference(args):
    """The reference arm: the FP64 CPU oracle as it stands on the host cores,
    on the GPU arm's workload and steps (bounded: about 90 s of stepping)."""
    rank, world, _ = env_rank()
    if rank != 0:
        return
    import workloads as W
    wl = W.block_meander(20, theta=0.5)
    n0 = start_step(args)
    n_first = n0 + args.warmup + 1
    h = oracle_history_timing(wl, n_first, args.steps, args.warmup, 90.0)
    whole = oracle_whole_steps_cuboid()
    cpu = {"value": h["steps_per_s"], "unit": UNIT, "cores": h["procs"], "kind": "oracle",
           "sample": _sample_text(h, n_first), "cpu_model": host_cpu_model(),
           "pairs_per_s": h["pairs_per_s"], "single_thread": h["single_thread"],
           "cuboid_whole_steps": whole}
    line = {
        "impl": "reference", "metric": METRIC, "value": h["steps_per_s"], "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": h["ms_per_sampled_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": block_config(wl, n0, n_first),
        "value_basis": "value = (evaluated points / points of a whole step) / ms_per_step",
        "point_source_evals_per_s": h["pairs_per_s"],
        "cpu_baseline": cpu,
        "e2e": {"value": h["steps_per_s"], "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def cpu_baseline_block(wl, n_first):
    """cpu_baseline of the GPU arm's line: the same timing on a 20 s budget."""
    h = oracle_history_timing(wl, n_first, 4, 1, 20.0)
    return {"value": h["steps_per_s"], "unit": UNIT, "cores": h["procs"], "kind": "oracle",
            "sample": _sample_text(h, n_first), "cpu_model": host_cpu_model(),
            "pairs_per_s": h["pairs_per_s"], "single_thread": h["single_thread"],
            "cuboid_whole_steps": oracle_whole_steps_cuboid()}


# ---------------------------------------------------------------------------
# learned warm start on the block mesh: training pairs from seeded meanders
# (random hatch angle and spacing, power, speed), evaluated on the benchmark
# scan at the benchmark state
# ---------------------------------------------------------------------------
def learned_leg(sa, W, wl, state, stream, n_pairs, epochs, K_eval):
    import numpy as np
    import torch
    th, dt = wl.theta, wl.dt
    idx = W.warm_start_input_rows(wl.patch)
    probe = sa.context_from_workload(wl, precision=sa.SA_MIXED)
    n_free = probe.sizes().n_free
    probe.close()
    n_scans = max(4, min(50, n_pairs // 1000))
    per = max(1, n_pairs // n_scans)
    X = torch.empty((per * n_scans, len(idx)), dtype=torch.bfloat16, device="cuda")
    Y = torch.empty((per * n_scans, n_free), dtype=torch.bfloat16, device="cuda")
    t0 = time.perf_counter()
    row = 0
    for k in range(n_scans):
        scan = W.learned_scan(k)
        wtr = W.Workload(f"train_{k}", wl.patch, wl.material, scan, dt=dt, theta=th, n_steps=10 ** 6)
        c = sa.context_from_workload(wtr, precision=sa.SA_MIXED, cuda_stream=stream, use_graph=1)
        c.step(th, dt, 200)
        c.set_recorder(X[row:row + per], Y[row:row + per], idx)
        c.step(th, dt, per)
        row += c.recorded()
        c.set_recorder(None, None, None)
        c.close()
    t_rec = time.perf_counter() - t0
    net = sa.MLP(len(idx), 256, n_free, seed=7)
    t0 = time.perf_counter()
    loss = None
    for ep in range(epochs):
        perm = torch.randperm(row, device="cuda")
        for b in range(0, row, 64):
            sel = perm[b:b + 64]
            net.train_step(X[sel].contiguous(), Y[sel].contiguous(), 1e-3, want_loss=False)
    torch.cuda.synchronize()
    loss, _ = net.gradients(X[:64].contiguous(), Y[:64].contiguous())
    t_train = time.perf_counter() - t0
    out = {"training_pairs": row, "epochs": epochs, "record_s": t_rec, "train_s": t_train,
           "final_minibatch_loss": loss, "n_in": int(len(idx)), "hidden": 256, "n_out": n_free,
           "params": net.n_params(), "evaluation": {}}
    for pre_name, pre in (("jacobi", sa.SA_PRECOND_JACOBI), ("fd", sa.SA_PRECOND_AUTO)):
        for learned in (False, True):
            c = sa.context_from_workload(wl, precision=sa.SA_MIXED, cuda_stream=stream, use_graph=1,
                                         precond=pre)
            c.step(th, dt, 0)
            c.set_state(*state)
            if learned:
                c.set_warm_start(net, idx)
            c.step(th, dt, 3)
            c.step(th, dt, 0)
            ms = time_graph(c, th, dt, K_eval, stream)
            st = c.step(th, dt, 0)
            key = pre_name + ("_learned" if learned else "_cold")
            out["evaluation"][key] = {"steps_per_s": K_eval / (ms / 1e3),
                                      "pcg_iters_per_step": st.pcg_iters_total / K_eval}
            if learned:
                used = 0
                for _ in range(10):
                    used += c.step(th, dt, 1).ws_used_last
                out["evaluation"][key]["learned_guess_kept_fraction"] = used / 10
            c.close()
    net.close()
    return out


def plate_leg(sa, W, stream, n_ff, K):
    """The 3 x 3 x 0.5 mm plate with a hole (degree 3, 48 x 48 x 8, closed
    seam): theta-steps/s over K steps after n_ff untimed steps of its
    contour scan, fast diagonalization against Jacobi."""
    wl = W.plate_with_hole()
    out = {"workload": wl.name, "first_step": n_ff + 3, "steps": K}
    state = None
    for name, pre in (("fd", sa.SA_PRECOND_AUTO), ("jacobi", sa.SA_PRECOND_JACOBI)):
        c = sa.context_from_workload(wl, precision=sa.SA_MIXED, cuda_stream=stream, use_graph=1,
                                     precond=pre)
        if state is None:
            c.step(wl.theta, wl.dt, n_ff)
            state = c.get_state()
        else:
            c.step(wl.theta, wl.dt, 0)
            c.set_state(*state)
        c.step(wl.theta, wl.dt, 3)
        c.step(wl.theta, wl.dt, 0)
        ms = time_graph(c, wl.theta, wl.dt, K, stream)
        st = c.step(wl.theta, wl.dt, 0)
        out[name] = {"steps_per_s": K / (ms / 1e3), "pcg_iters_per_step": st.pcg_iters_total / K,
                     "bottom_iters_per_step": st.bot_iters_total / K}
        if name == "fd":
            out["n_dof"] = c.sizes().n_dof
            out["nnz_a"] = c.sizes().nnz_a
        c.close()
    return out


def two_lasers_leg(sa, W, stream, n_ff, K):
    """Two lasers on the benchmark's block (reading R22): the 20-track
    meander and the same meander mirrored across the block's mid-plane
    y = 2 mm, switched on together.  By superposition each laser runs in a
    context of its own (the same part); a two-laser theta-step is one step of
    each, and T at the monitor points is sa_eval_T_superposed of the two.
    Times K steps of both after n_ff untimed ones."""
    import numpy as np
    import torch
    wl = W.block_meander(20, theta=0.5)
    sc = wl.scan
    mirrored = W.Scan(path=np.column_stack([sc.path[:, 0], 4.0e-3 - sc.path[:, 1], sc.path[:, 2]]),
                      seg_on=sc.seg_on, power=sc.power, absorptivity=sc.absorptivity,
                      speed=sc.speed, spot_radius=sc.spot_radius)
    wls = [wl, W.Workload(wl.name + "_mirrored", wl.patch, wl.material, mirrored, dt=wl.dt,
                          theta=wl.theta, n_steps=wl.n_steps)]
    ctxs = [sa.context_from_workload(w, precision=sa.SA_MIXED, cuda_stream=stream, use_graph=1)
            for w in wls]
    th, dt = wl.theta, wl.dt
    for c in ctxs:
        c.step(th, dt, n_ff + 3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for c in ctxs:
        c.step(th, dt, K, stats=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    rng = np.random.default_rng(5)
    mon = np.column_stack([rng.uniform(0.2e-3, 3.8e-3, 64), rng.uniform(0.2e-3, 3.8e-3, 64),
                           rng.uniform(0.5e-3, 1.0e-3, 64)])
    t0 = time.perf_counter()
    T = sa.eval_T_superposed(ctxs, mon)
    t_eval = time.perf_counter() - t0
    st = [c.step(th, dt, 0) for c in ctxs]
    out = {"workload": wl.name + " + mirrored meander", "first_step": n_ff + 4, "steps": K,
           "two_laser_steps_per_s": K / (ms / 1e3),
           "pcg_iters_per_step": sum(x.pcg_iters_total for x in st) / (2 * K),
           "superposed_eval_ms_64_points": 1e3 * t_eval,
           "monitor_T_max_K": float(np.nanmax(T))}
    for c in ctxs:
        c.close()
    return out


def batched_leg(sa, W, stream, n_inst, n_steps, rank=0, world=1, dist=None):
    """The batched sweep: n_inst seeded instances (uneven boxes, powers,
    speeds, track counts) stepped together for n_steps theta-steps (the
    first 3 untimed), one launch per stage for all instances.  With several
    ranks each takes a contiguous share of the instances (no collective on
    the data path); the time is the slowest rank's."""
    import numpy as np
    t0 = time.perf_counter()
    lo, hi = shard(n_inst, rank, world)
    wls = [W.batched_instance(i, n_steps=n_steps) for i in range(lo, hi)]
    ctxs = [sa.context_from_workload(wl, precision=sa.SA_MIXED) for wl in wls]
    b = sa.Batch(ctxs, precision=sa.SA_MIXED, cuda_stream=stream, use_graph=1)
    setup_s = time.perf_counter() - t0
    th, dt = wls[0].theta, wls[0].dt
    b.step(th, dt, 3)
    # launch shapes from the project's tuner (history tiles, solve grid),
    # cached by batch sizes in the build folder
    t1 = time.perf_counter()
    shapes = b.tune(os.path.join(ROOT, "paper_2511_20432_gb300", "_build", "batch_shapes.jsonl"),
                    at_step=max(1, n_steps // 2))
    tune_s = time.perf_counter() - t1
    sz = [c.sizes() for c in ctxs]
    K = n_steps - 3
    pairs = sum((z.q_lat + z.q_bot) * sum(min(n, z.n_src) for n in range(4, n_steps + 1)) for z in sz)
    if dist:
        dist.barrier()
    ms = max_over_ranks(time_graph(b, th, dt, K, stream), dist, "cuda")
    pairs = sum_over_ranks(pairs, dist, "cuda")
    m_it, b_it = b.iters()
    out = {"instances": n_inst, "steps": n_steps, "timed_steps": K, "setup_s": setup_s,
           "tuned_shapes": shapes, "tune_s": tune_s,
           "ms_per_step": ms / K, "instance_steps_per_s": n_inst * K / (ms / 1e3),
           ("point_source_equivalent_pairs_per_s" if shapes["hist_separable"] else
            "point_source_evals_per_s"): pairs / (ms / 1e3),
           "total_control_variables": int(sum_over_ranks(sum(z.n_dof for z in sz), dist, "cuda")),
           "total_boundary_points": int(sum_over_ranks(sum(z.q_lat + z.q_bot for z in sz), dist, "cuda")),
           "last_step_main_iters_max": int(max_over_ranks(int(m_it.max()), dist, "cuda")),
           "last_step_bottom_iters_max": int(max_over_ranks(int(b_it.max()), dist, "cuda")),
           "ranks": world}
    b.close()
    for c in ctxs:
        c.close()
    return out


def quarter_cylinder_leg(sa, W, stream, case="single_source",
                         meshes=((32, 16, 16), (64, 32, 32)), n_arc=721):
    """The quarter-cylinder part (Table 2 net, degree 2, uniform meshes of
    n_el elements) under the Section 3.1 single source (observed after 19
    steps, t = 1.9e-4 s) or the Section 3.2 contour scan (t = 2e-3 and 3e-3
    s): the heat-loss rates q~ and q^ at n_arc points of the top arc, the
    integrated |q~ + q^| and |q~| (trapezoid rule along the arc) and their
    ratio, the adiabatic residual of the discretisation, in FP64 and mixed;
    steps/s of the run (graph replay)."""
    import numpy as np
    import torch
    if case == "single_source":
        make, at = W.quarter_cylinder_single_source, (19,)
    else:
        make, at = W.quarter_cylinder_contour, (200, 300)
    th, pts, nrm, ds = W.quarter_cylinder_arc_points(n_arc)
    out = {"workload": "quarter_cylinder_" + case, "arc_points": n_arc, "meshes": []}
    for n_el in meshes:
        wl = make(n_el, n_steps=at[-1])
        row = {"n_el": list(n_el)}
        for name, prec in (("fp64", sa.SA_FP64), ("mixed", sa.SA_MIXED)):
            c = sa.context_from_workload(wl, precision=prec, cuda_stream=stream, use_graph=1)
            res = {"n_dof": c.sizes().n_dof, "t": []}
            done, t_steps = 0, 0.0
            for n in at:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                c.step(wl.theta, wl.dt, n - done)
                torch.cuda.synchronize()
                t_steps += time.perf_counter() - t0
                done = n
                t0 = time.perf_counter()
                qt, qh = c.eval_flux(pts, nrm)
                t_eval = time.perf_counter() - t0
                net = float(np.sum(np.abs(qt + qh) * ds))
                ana = float(np.sum(np.abs(qt) * ds))
                res["t"].append({"t_s": n * wl.dt, "int_abs_net_W_per_m": net,
                                 "int_abs_qtilde_W_per_m": ana, "net_over_qtilde": net / ana,
                                 "max_abs_net_W_per_m2": float(np.abs(qt + qh).max()),
                                 "max_abs_qtilde_W_per_m2": float(np.abs(qt).max()),
                                 "eval_ms": 1e3 * t_eval})
            res["steps_per_s"] = done / t_steps
            row[name] = res
            c.close()
        out["meshes"].append(row)
    return out


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def time_graph(ctx, th, dt, K, stream):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    ctx.step(th, dt, K, stats=False)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def run_ours(args):
    import numpy as np
    import torch
    import paper_2511_20432_gb300 as sa
    import workloads as W

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    wl = W.block_meander(20, theta=0.5)
    th, dt = wl.theta, wl.dt
    stream = torch.cuda.Stream()
    prec = sa.SA_MIXED if args.precision == "mixed" else sa.SA_FP64
    guess = sa.SA_GUESS_EXTRAPOLATE if args.guess == "extrapolate" else sa.SA_GUESS_PREVIOUS
    hist = {"auto": sa.SA_HIST_AUTO, "pairwise": sa.SA_HIST_PAIRWISE,
            "separable": sa.SA_HIST_SEPARABLE}[args.hist]
    ctx = sa.context_from_workload(wl, precision=prec, cuda_stream=stream, use_graph=1,
                                   initial_guess=guess, hist_mode=hist)
    n0 = start_step(args)
    ctx.step(th, dt, n0)                       # untimed fast-forward to mid-scan
    ctx.step(th, dt, args.warmup)              # warm-up (graph instantiated, caches warm)
    sz = ctx.sizes()
    q_pts = sz.q_lat + sz.q_bot
    state = ctx.get_state()
    K = args.steps
    n_first = n0 + args.warmup + 1
    pairs = q_pts * sum(min(n_first + i, sz.n_src) for i in range(K))

    # ---- timed region: K graph replays ---------------------------------------
    # The clock sampler starts 0.4 s before the timed region and runs until
    # at least 1 s of the same mid-scan stepping has followed it, so that it
    # sees samples however short the K steps are.
    clk = clocks_start(local)
    time.sleep(0.4)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms = time_graph(ctx, th, dt, K, stream)
    stats = ctx.step(th, dt, 0)                # counters accumulated over the timed steps
    t_w0 = time.perf_counter()
    K_w = 0
    while time.perf_counter() - t_w0 < 1.0:
        ctx.step(th, dt, 64, stats=False)
        torch.cuda.synchronize()
        K_w += 64
    clocks = clocks_stop(clk)
    clocks["window"] = (f"sampled every 50 ms from 0.4 s before the timed region to "
                        f"{K_w} steps of the same stepping after it")
    ms = max_over_ranks(ms, dist, "cuda")
    if clocks.get("sm_mhz"):
        clocks["ms_x_sm_mhz_per_step"] = ms / K * clocks["sm_mhz"]
    iters_avg = stats.pcg_iters_total / K
    bot_avg = stats.bot_iters_total / K
    value = world * K / (ms / 1e3)
    evals = world * pairs / (ms / 1e3)
    # separable sums: the pairs are not evaluated one by one (one FMA each);
    # the exponentials are the factors, sep_factors per active source
    exps = world * sz.sep_factors * sum(min(n_first + i, sz.n_src) for i in range(K)) / (ms / 1e3)
    if args.quick:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                              "steps": K, "warmup": args.warmup, "ms_per_step": ms / K,
                              "precision": args.precision, "guess": args.guess, "start_step": n0,
                              ("point_source_equivalent_pairs_per_s" if sz.hist_separable else
                               "point_source_evals_per_s"): evals, "pcg_iters_per_step": iters_avg,
                              "bot_iters_per_step": bot_avg, "clocks": clocks}))
        if dist:
            dist.destroy_process_group()
        return

    def fresh(precision, g, **kw):
        kw.setdefault("hist_mode", hist)
        c = sa.context_from_workload(wl, precision=precision, cuda_stream=stream, initial_guess=g, **kw)
        c.step(th, dt, 0)
        c.set_state(*state)
        return c

    # ---- stage breakdown (CUDA events on the launching stream, direct launches)
    K_t = min(K, 40)
    ctx_t = fresh(prec, guess, stage_timing=1)
    ctx_t.step(th, dt, 3)
    ctx_t.stage_times()
    st_t = ctx_t.step(th, dt, K_t)
    stage_ms, k_timed = ctx_t.stage_times()
    stage_avg = {k: v / k_timed for k, v in stage_ms.items()}
    iters_t = st_t.pcg_iters_total / K_t
    pairs_t = q_pts * (min(state[0] + 3 + K_t // 2, sz.n_src))
    ctx_t.close()

    want = lambda leg: args.legs == "all" or leg in args.legs.split(",")
    K_c = min(K, 60)
    cold_steps = jacobi_steps = pairwise_steps = fp64_steps = fp64_sep_steps = float("nan")
    st_c = st_j = None
    pairs_p, ms_p = 0, float("nan")
    other = sa.SA_GUESS_EXTRAPOLATE if guess == sa.SA_GUESS_PREVIOUS else sa.SA_GUESS_PREVIOUS
    if want("variants"):
        # ---- the other initial guess, Jacobi, and the plain FP64 path
        ctx_c = fresh(prec, other, use_graph=1)
        ctx_c.step(th, dt, 3)
        ctx_c.step(th, dt, 0)
        ms_c = time_graph(ctx_c, th, dt, K_c, stream)
        st_c = ctx_c.step(th, dt, 0)
        cold_steps = K_c / (ms_c / 1e3)
        ctx_c.close()
        # the same path with the Jacobi preconditioner
        ctx_j = fresh(prec, guess, use_graph=1, precond=sa.SA_PRECOND_JACOBI)
        ctx_j.step(th, dt, 3)
        ctx_j.step(th, dt, 0)
        ms_j = time_graph(ctx_j, th, dt, K_c, stream)
        st_j = ctx_j.step(th, dt, 0)
        jacobi_steps = K_c / (ms_j / 1e3)
        ctx_j.close()
        # the same path with the pairwise history sums
        ctx_p = fresh(prec, guess, use_graph=1, hist_mode=sa.SA_HIST_PAIRWISE)
        ctx_p.step(th, dt, 3)
        ms_p = time_graph(ctx_p, th, dt, K_c, stream)
        pairwise_steps = K_c / (ms_p / 1e3)
        n_p = state[0] + 3 + 1
        pairs_p = q_pts * sum(min(n_p + i, sz.n_src) for i in range(K_c))
        ctx_p.close()
        # plain FP64 (pairwise history sums, as the method states them) and FP64
        # with the separable sums
        K64 = min(K, 12)
        ctx64 = fresh(sa.SA_FP64, sa.SA_GUESS_PREVIOUS, use_graph=1, hist_mode=sa.SA_HIST_PAIRWISE)
        ctx64.step(th, dt, 2)
        ms64 = time_graph(ctx64, th, dt, K64, stream)
        fp64_steps = K64 / (ms64 / 1e3)
        ctx64.close()
        ctx64s = fresh(sa.SA_FP64, sa.SA_GUESS_PREVIOUS, use_graph=1, hist_mode=sa.SA_HIST_SEPARABLE)
        ctx64s.step(th, dt, 2)
        ms64s = time_graph(ctx64s, th, dt, K_c, stream)
        fp64_sep_steps = K_c / (ms64s / 1e3)
        ctx64s.close()

    # ---- opt-in history cutoff (not the paper's method): pairs skipped and
    # steps/s at two budgets, on the block and on a 6 x 6 x 1 mm block with
    # the same meander near one corner
    cutoff = None
    if want("cutoff"):
        cutoff = {"block": {}, "block_6x6x1mm": {}}
        for eta in (0.0, 1e-6, 1e-4):
            c = fresh(prec, guess, use_graph=1, hist_cutoff=eta)
            c.step(th, dt, 3)
            c.step(th, dt, 0)
            ms_x = time_graph(c, th, dt, K_c, stream)
            st_x = c.step(th, dt, 0)
            n_x = state[0] + 3 + 1
            pairs_x = q_pts * sum(min(n_x + i, sz.n_src) for i in range(K_c))
            cutoff["block"][f"{eta:g}"] = {"steps_per_s": K_c / (ms_x / 1e3),
                                          "pairs_skipped_fraction": st_x.hist_pairs_skipped / pairs_x}
            c.close()
        wl6 = W.block_meander(20, theta=0.5, n_el=(96, 96, 16), size=(6e-3, 6e-3, 1e-3))
        for eta in (0.0, 1e-6, 1e-4):
            c = sa.context_from_workload(wl6, precision=prec, cuda_stream=stream, use_graph=1,
                                         hist_cutoff=eta)
            c.step(th, dt, n0)
            z6 = c.sizes()
            ms_x = time_graph(c, th, dt, K_c, stream)
            st_x = c.step(th, dt, 0)
            pairs_x = (z6.q_lat + z6.q_bot) * sum(min(n0 + 1 + i, z6.n_src) for i in range(K_c))
            cutoff["block_6x6x1mm"][f"{eta:g}"] = {
                "steps_per_s": K_c / (ms_x / 1e3), "n_dof": z6.n_dof,
                "pairs_skipped_fraction": st_x.hist_pairs_skipped / pairs_x}
            c.close()

    # ---- end to end through the public API with host buffers -------------------
    e2e = None
    if want("e2e"):
        rng = np.random.default_rng(3)
        mon = np.column_stack([rng.uniform(0.2e-3, 3.8e-3, N_MONITOR), rng.uniform(0.2e-3, 3.8e-3, N_MONITOR),
                               rng.uniform(0.5e-3, 1.0e-3, N_MONITOR)])
        # the monitor points and their temperatures in pinned host memory
        mon_pin = torch.empty((N_MONITOR, 3), dtype=torch.float64, pin_memory=True)
        mon_pin.copy_(torch.from_numpy(np.ascontiguousarray(mon)))
        mon = mon_pin.numpy()
        T_pin = torch.empty(N_MONITOR, dtype=torch.float64, pin_memory=True).numpy()
        K_e = min(K, 100)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(K_e):
            ctx.step(th, dt, 1, stats=False)        # enqueued; device flags stay set until read
            T_mon = ctx.eval_T(mon, out=T_pin)      # host points in, host temperatures out (synchronous)
        st_e = ctx.step(th, dt, 0)                  # the status of those steps (raises on a flag)
        t_e2e = time.perf_counter() - t0
        e2e = world * K_e / t_e2e
        assert np.isfinite(T_mon).all() and st_e.pcg_iters_total >= K_e

    # ---- the batched sweep (256 instances, 2000 steps) ------------------------------
    batched = (batched_leg(sa, W, stream, args.batch_instances, args.batch_steps, rank, world, dist)
               if args.batch_steps > 3 and want("batched") else None)

    # ---- the plate with a hole ---------------------------------------------------
    plate = plate_leg(sa, W, stream, 1000, min(K, 300)) if world == 1 and want("plate") else None

    # ---- two lasers by superposition (a leg of its own; an error is reported, not raised)
    lasers = None
    if world == 1 and want("lasers"):
        try:
            lasers = two_lasers_leg(sa, W, stream, n0, min(K, 300))
        except Exception as exc:   # the main line stands without this leg
            lasers = {"error": f"{type(exc).__name__}: {exc}"}

    # ---- the quarter-cylinder part: heat-loss rates along the top arc ------------
    qcyl = quarter_cylinder_leg(sa, W, stream) if world == 1 and want("arc") else None
    qcon = quarter_cylinder_leg(sa, W, stream, "contour") if world == 1 and want("arc") else None

    # ---- learned warm start (bounded: a few thousand training pairs) -------------
    learned = None
    if args.learned_pairs > 0 and world == 1 and want("learned"):
        learned = learned_leg(sa, W, wl, state, stream, args.learned_pairs, args.learned_epochs,
                              min(K, 100))

    # ---- roofline of the dominant kernel ------------------------------------------
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    total = sum(stage_avg.values())
    shares = {k: v / total for k, v in stage_avg.items()}
    n_free, nnz_a = sz.n_free, sz.nnz_a
    warm = 1 if guess == sa.SA_GUESS_EXTRAPOLATE else 0
    # algorithmic bytes of one main-solve launch: every SpMV reads the FP32
    # values and 16-bit column offsets once and the published vector once;
    # set-up reads r0 and D^{-1} (FP64), reads and writes x (FP64), reads u
    # back (FP32); fast diagonalization: each application (one at set-up, one
    # per further iteration) reads and writes the FP32 vector in its three
    # plane-form passes and reads the scaling S
    pcg_bytes = ((iters_t + warm) * (6 * nnz_a + 4 * n_free) + (36 + 4 * warm) * n_free +
                 max(iters_t, 1.0) * (3 * 8 + 4) * n_free)
    # history: pairwise, FP32 lane-operations per pair (flux 8, T 6) on 128
    # FP32 lanes/clk/SM (MUFU ex2, 32/clk/SM, not binding); separable, one
    # FFMA per pair (the factors' exponentials are overhead)
    sep = bool(sz.hist_separable)
    pairs_clk = 128.0 if sep else 128.0 * q_pts / (8 * sz.q_lat + 6 * sz.q_bot)
    kernels = {
        "pcg": {"bound": "hbm", "bytes_per_launch": pcg_bytes, "ms": stage_avg["pcg"],
                "achieved_gbs": pcg_bytes / (stage_avg["pcg"] * 1e-3) / 1e9,
                "iters_per_step": iters_t, "warm_start_spmv": warm},
        "history": {"bound": "alu", "pairs_per_launch": pairs_t, "ms": stage_avg["history"],
                    "achieved_gpairs": pairs_t / (stage_avg["history"] * 1e-3) / 1e9,
                    "peak_gpairs": n_sm * sm_max * 1e6 * pairs_clk / 1e9},
    }
    dom = "history" if stage_avg["history"] >= stage_avg["pcg"] else "pcg"
    if dom == "history":
        k = kernels["history"]
        roof = {"bound": "alu", "achieved": k["achieved_gpairs"], "peak": k["peak_gpairs"],
                "unit": "Gpairs/s", "frac": k["achieved_gpairs"] / k["peak_gpairs"],
                "traffic": (profile_traffic("k_sep_gemm_block_meander", "sa_sep.cu") if sep else
                            profile_traffic("k_history_mixed_block_meander", "sa_history.cu")),
                "kernel": "k_sep_gemm + k_sep_reduce" if sep else "k_history_mixed",
                "peak_basis": f"{n_sm} SMs x {sm_max:.0f} MHz x {pairs_clk:.1f} pairs/clk/SM " +
                              ("(FP32 pipe: 128 lanes/clk, one FFMA a pair)" if sep else
                               "(FP32 pipe: 128 lanes/clk, 8 ops a flux pair, 6 a T pair)")}
    else:
        k = kernels["pcg"]
        roof = {"bound": "hbm", "achieved": k["achieved_gbs"], "peak": hbm, "unit": "GB/s",
                "frac": k["achieved_gbs"] / hbm if hbm else None,
                "traffic": profile_traffic("k_pcg_smem_block_meander", "sa_solve.cu"),
                "kernel": "k_pcg_smem (free block)", "peak_basis": "hbm_gbs of measured",
                "note": "algorithmic bytes count every SpMV's pass over the operator; later "
                        "passes of a launch hit L2 (traffic: one ncu-captured launch)"}
    # prologue, history (bottom, lateral; separable: a product and a reduction
    # each, and no prologue in the mixed path), gather (bottom, lateral),
    # projection (which also writes the Dirichlet increments: the block's
    # projection runs in shared memory), right-hand side (two slice sets),
    # PCG (which also finalizes the step)
    launches_per_step = 9 + warm + ((1 if prec == sa.SA_MIXED else 2) if sep else 0)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": block_config(wl, n0, n_first),
        "path": {"precision": "mixed: FP32 history sum and operator values, FP64 state, "
                              "boundary integrals and Krylov vectors",
                 "history_evaluation": "separable" if sep else "pairwise",
                 "initial_guess": args.guess,
                 "preconditioner": "fast diagonalization (main solve and bottom projection)",
                 "nnz_a": nnz_a,
                 "l2": "no flush: per-step inputs larger than L2 (operators in SELL-32: "
                       "~170 MB of FP32 values and indices; 129 MB L2)",
                 "parallelism": "replicas" if world > 1 else "single"},
        # precision gain like for like (both separable), then against the
        # plain FP64 path as the method states the sums (pairwise)
        "precision_gain_separable": value / (world * fp64_sep_steps),
        "mixed_over_fp64_pairwise": value / (world * fp64_steps),
        ("point_source_equivalent_pairs_per_s" if sep else "point_source_evals_per_s"): evals,
        "history_exponentials_per_s": exps if sep else evals,
        "point_source_evals_per_s_pairwise_leg": world * pairs_p / (ms_p / 1e3),
        "steps_per_s_other_guess": world * cold_steps,
        "pcg_iters_per_step_other_guess": st_c.pcg_iters_total / K_c if st_c else None,
        "other_guess": "extrapolate" if other == sa.SA_GUESS_EXTRAPOLATE else "previous",
        "steps_per_s_jacobi": world * jacobi_steps,
        "pcg_iters_per_step_jacobi": st_j.pcg_iters_total / K_c if st_j else None,
        "steps_per_s_pairwise_history": world * pairwise_steps,
        "fp64_pairwise_steps_per_s": world * fp64_steps,
        "fp64_separable_steps_per_s": world * fp64_sep_steps,
        "pcg_iters_per_step": iters_avg, "bot_iters_per_step": bot_avg,
        "stage_ms": stage_avg, "stage_share": shares, "kernels": kernels,
        "roofline": roof,
        "e2e": ({"value": e2e, "unit": UNIT, "h2d_bytes_per_step": N_MONITOR * 3 * 8,
                 "d2h_bytes_per_step": N_MONITOR * 8,
                 "loop": "per step: sa_step (no statistics) + sa_eval_T of the monitor points "
                         "(host in, host out, one synchronisation); the statistics of all the "
                         "steps read once at the end (their flags stay set until read)"}
                if e2e is not None else None),
        "history_cutoff": cutoff,
        "plate_with_hole": plate,
        "two_lasers": lasers,
        "quarter_cylinder_single_source": qcyl,
        "quarter_cylinder_contour": qcon,
        "batched_256": batched,
        "learned_warm_start": learned,
        "gpu_launches": launches_per_step * K,
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and want("cpu"):
        line["cpu_baseline"] = cpu_baseline_block(wl, n_first + K // 2)
    if rank == 0:
        print(json.dumps(finite(line)))
    if dist:
        dist.destroy_process_group()


def finite(o):
    """The line with NaN / infinite numbers (legs not run) as null."""
    import math
    if isinstance(o, dict):
        return {k: finite(v) for k, v in o.items()}
    if isinstance(o, (list, tuple)):
        return [finite(v) for v in o]
    if isinstance(o, float) and not math.isfinite(o):
        return None
    return o


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
