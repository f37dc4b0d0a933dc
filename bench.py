"""Throughput benchmark of the fused isotropic phase-field step on GB300.

Workload (one "step"): one explicit time step of every instance of the 2D
orientation sweep -- ten 1024 x 1024 free-dendrite runs at alpha0 = 0, 5,
..., 45 degrees (h = 0.8, dt = 0.02, k = 0.15, eps4 = 0.02, lambda = 10,
D = 0.6267 lambda, U0 = -0.55, seed r = 10 h), scheme S-bar_{2,1}, FP32
fields, batched in one persistent launch per step replayed from a CUDA
graph, with the FP64 observe reductions every 100 steps.  Synthetic data.

Prints one JSON line (rank 0).  `value` is aggregate cell updates per
second (GLUPS) over all ranks; `roofline` reports the dominant kernel's
algorithmic HBM bandwidth against the measured copy bandwidth;
`cpu_baseline` times the FP64 CPU oracle on a bounded sample; `e2e` is the
same job through the public API with the state uploaded from and returned to
pinned host buffers inside the timed region.

--impl reference times the FP64 CPU oracle itself (the only baseline: the
paper ships no code), one instance-step of the same workload per step.
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
sys.path.insert(0, ROOT)

METRIC = "GLUPS & %HBM peak, batched FP32 vs plain FP64 at stated error; p50/p99 latency"
THETAS = tuple(range(0, 50, 5))
PHYS_STEPS = 20000
DS_THETAS = (0, 10, 20, 30, 40)
DS_VP, DS_LT = 0.1, 2000.0
OBS_EVERY = 100
# algorithmic bytes per cell update: read psi, U; write psi', U' (f32c: hi
# and lo halves of psi and U); the two-kernel form adds the d psi/dt write
# and read and the U pass's second read of psi and U.  Plus the int16 grain
# index where it is read: in 3D always, in 2D only for instances with cells
# outside grain 0 (the 2D step reads no grain rows when every cell is in
# grain 0).
B_STATE = {"f32": 16, "f64": 32, "f32c": 32}
B_STATE_TWO = {"f32": 32, "f64": 64}
B_GRAIN = 2


def bytes_per_cell(ws, precision, two=False) -> float:
    """Algorithmic bytes per cell update of a batch, averaged over its cells."""
    cells = sum(w.n_cells for w in ws)
    graincells = sum(w.n_cells for w in ws
                     if w.dim == 3 or (len(w.seed_grain) and int(max(w.seed_grain)) > 0))
    return (B_STATE_TWO if two else B_STATE)[precision] + B_GRAIN * graincells / cells


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# DRAM traffic per step of the dominant kernel from an ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) without cache flushes between
# launches (--cache-control none: the lines a launch leaves dirty in L2 are
# written back during the next one, as in a live run), valid only while the
# kernel source is byte-identical to the one captured (sha256 of the .cu file)
# and the launch uses the captured tile (block x, block y, sweep).
TRAFFIC = {
    # one step of the orientation sweep (10 x 1024^2, tile 64 x 1 x 38): the two
    # k_step2d<float, S-bar_21> launches of the two five-instance groups, summed (ncu runs them one
    # after the other, so each group's half of the state partly stays in L2)
    "sweep2d": {"source": "paper_2110_12448_gb300/csrc/step2d.cu", "tile": [64, 1, 38],
                "sha256": "51b2245cc8536307702969be51cd8ebcc4eef9819cb65035bf04650382af4634", "bytes": 103638016},
    # one k_step3d<float, S-bar_120, 30, 6> launch of the 256^3 free dendrite (tile 34 x 10 x 52)
    "dendrite3d": {"source": "paper_2110_12448_gb300/csrc/step3d.cu", "tile": [34, 10, 52],
                   "sha256": "1f5d22af251dade05882fb4be57c4fe582caa7ec964125d0cab5048c80b10939", "bytes": 265664000},
}


# FP32 floating-point operations per cell update of the dominant kernel, from
# an ncu capture of one launch: FADD + FMUL + 2 FFMA + 2 (FADD2 + FMUL2) +
# 4 FFMA2 thread instructions (sm__sass_thread_inst_executed_op_*_pred_on)
# over the launch's cell updates; like TRAFFIC, valid only while the kernel
# source is byte-identical to the one captured.  The FP32 peak is the unit
# count at the maximum clock: 152 SMs x 128 FP32 lanes x 2 (FMA) x 2.07 GHz.
# (3D: executed per output cell, including the ring-1 recompute of the tile.)
FLOPS = {
    # k_step2d<float, S-bar_21> launch of the orientation sweep (10 x 1024^2, tile 64 x 1 x 38)
    "sweep2d": {"source": "paper_2110_12448_gb300/csrc/step2d.cu", "tile": [64, 1, 38],
                "sha256": "51b2245cc8536307702969be51cd8ebcc4eef9819cb65035bf04650382af4634", "flop_per_cell": 261.2},
    # k_step3d<float, S-bar_120, 30, 6> launch of the 256^3 free dendrite (tile 34 x 10 x 52)
    "dendrite3d": {"source": "paper_2110_12448_gb300/csrc/step3d.cu", "tile": [34, 10, 52],
                   "sha256": "1f5d22af251dade05882fb4be57c4fe582caa7ec964125d0cab5048c80b10939", "flop_per_cell": 1100.6},
}
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def _captured(table, workload, key, tile=None):
    """table[workload][key] if the kernel source still matches the capture and
    the launch uses the captured block shape, else None.  (The sweep length
    moves the per-cell figures only through the halo rows or planes of each
    work item's prologue: well under 1 % between neighbouring sweeps.)  The
    DRAM bytes were captured at depth 1 (one launch per step); a depth-2 tile
    (two steps per wavefront of band launches) runs the same work items, so
    its FLOP per cell carry over, its DRAM bytes do not."""
    import hashlib
    t = table.get(workload)
    if not t or not t["sha256"]:
        return None
    if tile is None or list(tile)[:2] != list(t["tile"])[:2]:
        return None
    if key == "bytes" and len(tile) > 3 and int(tile[3]) != 1:
        return None
    with open(os.path.join(ROOT, t["source"]), "rb") as f:
        if hashlib.sha256(f.read()).hexdigest() != t["sha256"]:
            return None
    return t[key]


def traffic_for(workload, tile=None):
    return _captured(TRAFFIC, workload, "bytes", tile)


def aggregate(ms_local: float, cells_per_rank: int, steps: int, world: int, device=None) -> tuple:
    """Whole-job throughput: every rank runs its own replica of the workload
    (weak scaling, no data-path collective); the job time is the slowest
    rank's.  Returns (max ms over ranks, aggregate GLUPS)."""
    ms = ms_local
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, cells_per_rank * steps * world / (ms / 1e3) / 1e9


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap,utilization.gpu")

    def __init__(self, index, window="the timed region"):
        self.index = index
        self.window = window
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        self.edges = []  # one-shot samples taken right before and right after

    def once(self):
        """One synchronous sample (a row in the sampler's format), or None."""
        try:
            r = subprocess.run(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=10)
            row = r.stdout.strip().splitlines()[0]
            return row if row.count(",") >= 9 else None
        except Exception:
            return None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def mark(self):
        """A synchronous sample at this point (call right before and right
        after the timed region, so that short timed regions still carry one)."""
        row = self.once()
        if row:
            self.edges.append(row)

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        try:
            self.f.flush()
            sampled = [r for r in open(self.f.name).read().strip().splitlines() if r.strip()]
            rows = [r.split(",") for r in sampled + self.edges]
            sm = [float(r[1]) for r in rows]
            mx = max(float(r[2]) for r in rows)
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
            # utilisation from the sampler only: the edge samples are taken
            # with the device synchronised, idle by construction
            util = [float(r[9]) for r in (x.split(",") for x in sampled)
                    if len(r) > 9 and r[9].strip().replace(".", "", 1).isdigit()]
            return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": reasons,
                    # NVML's utilisation is an average over its own sampling period: a
                    # median of a handful of samples around a sub-second timed region
                    # says nothing, so it is reported from five samples up
                    "gpu_util_pct_median": statistics.median(util) if len(util) >= 5 else None,
                    "samples": len(sampled), "edge_samples": len(self.edges),
                    "edge_sm_mhz": [float(r.split(",")[1]) for r in self.edges],
                    "window": f"200 ms sampler over {self.window}, plus one sample right before and one right "
                              f"after the timed region"}
        except Exception as e:  # pragma: no cover
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "error": str(e)}


def workloads(n, scheme, mode="sweep2d"):
    from paper_2110_12448_gb300 import synth
    if mode == "dendrite3d":
        return [synth.free_dendrite_3d(n, scheme=scheme)]
    if mode == "poly2d":
        return [w for w in synth.polycrystal_batch_2d(64)]
    if mode == "directional2d":
        return [synth.directional_2d(n, 2 * n, float(t), scheme, Vp=DS_VP, lT=DS_LT, steps=20000) for t in DS_THETAS]
    return [synth.free_dendrite_2d(n, float(t), scheme, steps=20000) for t in THETAS]


WORKLOAD_TEXT = {
    "sweep2d": "orientation sweep 2D, 10 x {n}^2 instances (alpha0 = 0..45 deg), {scheme}",
    "dendrite3d": "3D free dendrite {n}^3, random ZXZ orientation, {scheme}",
    "poly2d": "batched 2D polycrystal, 64 instances 256^2..1536^2, 3-12 grains each, {scheme}",
    "directional2d": "directional solidification 2D, 5 x {n}x{n2} instances (alpha0 = 0..40 deg), frozen gradient "
                     "Vp = 0.1 W/tau0, lT = 2000 W, periodic x, {scheme}",
}


def cpu_baseline(n, scheme, max_seconds=15.0, max_steps=400):
    """FP64 oracle on the host cores, bounded sample: one instance, a few steps."""
    import numpy as np
    from oracle import oracle as O
    ws = workloads(n, scheme)
    w = ws[3]
    p = O.params(nx=w.nx, ny=w.ny, scheme=O.SBAR21 if scheme == "SBAR21" else {"S21": 1, "S10": 0}[scheme], h=w.h,
                 dt=w.dt, k=w.k, eps4=w.eps4, lam=w.lam, D=w.D)
    psi, U, g = O.init_seeds(p, w.U0, w.seeds, w.seed_grain)
    O.step(p, w.rots, g, psi, U, 1)  # warm
    steps = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < max_seconds and steps < max_steps:
        psi, U = O.step(p, w.rots, g, psi, U, 1)
        steps += 1
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": w.n_cells * steps / dt / 1e9, "unit": "GLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{steps} steps of one {w.nx}x{w.ny} instance (alpha0={THETAS[3]} deg) of the 10, FP64, {dt:.1f} s",
            "single_thread": cpu_baseline_1thread(n, scheme)}


def cpu_baseline_1thread(n, scheme, steps=2):
    """The same oracle sample on one host thread (a fresh process, so that
    OpenMP starts with OMP_NUM_THREADS=1): `steps` steps of the same instance."""
    import subprocess
    import sys
    code = ("import sys, time; sys.path.insert(0, {root!r}); import bench; from oracle import oracle as O; "
            "w = bench.workloads({n}, {scheme!r})[3]; "
            "p = O.params(nx=w.nx, ny=w.ny, scheme={code}, h=w.h, dt=w.dt, k=w.k, eps4=w.eps4, lam=w.lam, D=w.D); "
            "psi, U, g = O.init_seeds(p, w.U0, w.seeds, w.seed_grain); O.step(p, w.rots, g, psi, U, 1); "
            "t0 = time.perf_counter(); O.step(p, w.rots, g, psi, U, {steps}); "
            "print(w.n_cells * {steps} / (time.perf_counter() - t0) / 1e9)").format(
        root=ROOT, n=n, scheme=scheme, steps=steps, code={"SBAR21": 2, "S21": 1, "S10": 0}[scheme])
    try:
        r = subprocess.run([sys.executable, "-c", code], env=dict(os.environ, OMP_NUM_THREADS="1"),
                           capture_output=True, text=True, timeout=120, check=True)
        v = float(r.stdout.strip().splitlines()[-1])
    except Exception as e:  # reported, not fatal: the all-core figure stands
        return {"error": str(e)[:200]}
    return {"value": v, "unit": "GLUPS", "cores": 1, "sample": f"{steps} steps of the same instance, one thread"}


def at_stated_error(stream, ws, steps, n_streams=2):
    """The same batch on the compensated FP32 state (PF_F32C), the precision
    that meets the accuracy contract: max |d phi|, |d U| <= 1e-4 against the
    FP64 oracle after 10^4 steps of the 200^2 free dendrite, tip speed within
    0.5 % (checked by tests/test_gpu_contract.py, not here).  Autotuned tile,
    persistent launches replayed from CUDA graphs, the batch as `n_streams`
    groups on their own streams like the main measurement, device time of
    `steps` steps after a warm-up; no observe inside the timed region."""
    import torch

    from paper_2110_12448_gb300 import autotune
    from paper_2110_12448_gb300 import native as N
    from paper_2110_12448_gb300.batch import Batch
    tile, _ = autotune.tune(ws, "f32c", n_streams=n_streams)
    batch = Batch(ws, "f32c", n_streams=n_streams, tile=tile)
    batch.step(32, stream=stream)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    batch.step(steps, stream=stream)
    b.record(stream)
    b.synchronize()
    ms = a.elapsed_time(b)
    cells = batch.n_cells
    batch.close()
    return {"value": cells * steps / (ms / 1e3) / 1e9, "unit": "GLUPS", "precision": "f32c",
            "ms_per_step": ms / steps, "steps": steps, "tile": list(tile),
            "contract": "max |d phi|, |d U| <= 1e-4 vs the FP64 oracle after 10^4 steps of the 200^2 free dendrite, "
                        "tip speed within 0.5 % (tests/test_gpu_contract.py)",
            "bytes_per_cell": bytes_per_cell(ws, "f32c"),
            "hbm_frac": cells * bytes_per_cell(ws, "f32c") / (ms / steps / 1e3) / 1e9 / peaks()[0]}


def fp64_plain(stream, n=200, steps=2000):
    """Comparator: the plain single-instance FP64 step (200 x 200 free
    dendrite, one launch per step through pf_step), GLUPS and us/step (mean,
    and p50/p99 over individually timed steps); and the same instance stepped
    through a one-member group replayed from a CUDA graph."""
    import statistics

    import torch

    from paper_2110_12448_gb300 import native as N
    from paper_2110_12448_gb300 import synth
    w = synth.free_dendrite_2d(n)
    s = N.Sim.from_workload(w, "f64", stream=stream)
    s.set_tile(64, 1, 16)
    s.step(10)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    s.step(steps)
    b.record(stream)
    b.synchronize()
    ms = a.elapsed_time(b)
    o = s.observe(0)
    # per-step times: one event pair around each of 200 single steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(200)]
    for e0, e1 in ev:
        e0.record(stream)
        s.step(1)
        e1.record(stream)
    ev[-1][1].synchronize()
    per = sorted(e0.elapsed_time(e1) * 1e3 for e0, e1 in ev)
    # the same instance through a one-member group (persistent launch + CUDA graph)
    g = N.Group(1, N.Group.work_items(s), stream=stream)
    g.add(s)
    g.step(10)
    a.record(stream)
    g.step(steps)
    b.record(stream)
    b.synchronize()
    ms_graph = a.elapsed_time(b)
    g.close()
    s.close()
    return {"value": w.n_cells * steps / (ms / 1e3) / 1e9, "unit": "GLUPS", "us_per_step": ms * 1e3 / steps,
            "us_per_step_p50": statistics.median(per), "us_per_step_p99": per[int(0.99 * (len(per) - 1))],
            "graph_us_per_step": ms_graph * 1e3 / steps,
            "workload": f"free dendrite 2D {n}x{n}, SBAR21, FP64, {steps} steps, one launch per step "
                        f"(graph: the same instance in a one-member group, replayed from a CUDA graph)",
            "tip_y": o["tip"][1]}


# tip operating state of the orientation sweep: all three 2D schemes, FP32,
# run to the sweep's full length; an FP64 run of one angle states the FP32 error
PHYS_SCHEMES = ("S10", "S21", "SBAR21")
PHYS_FP64_THETA = 30.0
PHYS_FP64_BATCH_STEPS = 200  # timed steps of each scheme's ten-instance batch in FP64
# Table 1: seconds per isothermal run of Sec. 4.3.2 on one Tesla P100 (context)
PAPER_TABLE1_S = {"S10": 1359.0, "S21": 4612.0, "SBAR21": 3883.0}


def run_batch(stream, ws, precision, obs_back=1000, keep=()):
    """Step a batch of workloads (one group, autotuned tile) to ws[0].steps.
    Returns (device ms of the steps, per-instance tip state at the end,
    tile, {index: (psi, U)} for the indices in `keep`).  The tip state: growth
    angle of the tip seen from the seed centre and of the tip's track over the
    second half of the run (the direction of its displacement, measured like the
    paper's alpha by tracking the tip), tip velocity over the last `obs_back`
    steps, tip radius, sigma* and the tip Peclet number rho V / (2 D)."""
    import math

    import torch

    from paper_2110_12448_gb300 import autotune
    from paper_2110_12448_gb300 import native as N
    tile, _ = autotune.tune(ws, precision)
    sims = []
    with torch.cuda.stream(stream):
        for w in ws:
            sims.append(N.Sim.from_workload(w, precision, stream=stream))
            sims[-1].set_tile(*autotune.split(tile)[0])
    group = N.Group(len(sims), sum(N.Group.work_items(s) for s in sims), stream=stream)
    for s in sims:
        group.add(s)
    group.set_depth(*autotune.split(tile)[1])
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    ms = 0.0
    half = ws[0].steps // 2
    mid = None
    for k in (half, ws[0].steps - half - obs_back, obs_back):
        a.record(stream)
        group.step(k)
        b.record(stream)
        b.synchronize()
        ms += a.elapsed_time(b)
        obs = [s.observe(0, allow_nonfinite=True) for s in sims]
        if mid is None:
            mid = [o["tip"] for o in obs]
    rows = []
    for w, s, o, t1 in zip(ws, sims, obs, mid):
        ok = o["found"] and not o["nonfinite"]
        tr = s.tip_radius(o, 0) if ok else {"rho": float("nan"), "sigma_star": float("nan")}
        track = math.degrees(math.atan2(-(o["tip"][0] - t1[0]), o["tip"][1] - t1[1])) if ok else float("nan")
        rows.append({"alpha_deg": o["angle_xy_deg"] if ok else float("nan"), "alpha_track_deg": track,
                     "v_tip": o["v_tip"] if ok else float("nan"),
                     "rho": tr["rho"], "sigma_star": tr["sigma_star"],
                     "peclet": tr["rho"] * o["v_tip"] / (2 * w.D) if ok else float("nan"),
                     "nonfinite": o["nonfinite"]})
    fields = {i: sims[i].get_fields() for i in keep}
    group.close()
    for s in sims:
        s.close()
    return ms, rows, tile, fields


def ivantsov_peclet_2d(omega):
    """Peclet number P = rho V / (2 D) of the 2D Ivantsov needle at
    supersaturation omega: omega = sqrt(pi P) exp(P) erfc(sqrt(P)), by
    bisection (the left side increases with P)."""
    import math
    lo, hi = 1e-9, 50.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if math.sqrt(math.pi * mid) * math.exp(mid) * math.erfc(math.sqrt(mid)) < omega:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def batch_rate(stream, ws, precision, steps, warm=5):
    """GLUPS of one batch of workloads (one group, autotuned tile) over `steps`
    timed steps after `warm` untimed ones."""
    import torch

    from paper_2110_12448_gb300 import autotune
    from paper_2110_12448_gb300 import native as N
    tile, _ = autotune.tune(ws, precision)
    sims = []
    with torch.cuda.stream(stream):
        for w in ws:
            sims.append(N.Sim.from_workload(w, precision, stream=stream))
            sims[-1].set_tile(*autotune.split(tile)[0])
    group = N.Group(len(sims), sum(N.Group.work_items(s) for s in sims), stream=stream)
    for s in sims:
        group.add(s)
    group.set_depth(*autotune.split(tile)[1])
    group.step(warm)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    group.step(steps)
    b.record(stream)
    b.synchronize()
    ms = a.elapsed_time(b)
    group.close()
    for s in sims:
        s.close()
    return sum(w.n_cells for w in ws) * steps / ms / 1e6


def _table(thetas, rows):
    r6 = lambda v: None if v != v else round(float(v), 6)  # noqa: E731
    t = {"theta_deg": [float(x) for x in thetas]}
    for key in ("alpha_deg", "alpha_track_deg", "v_tip", "rho", "sigma_star", "peclet"):
        t[key] = [r6(r[key]) for r in rows]
    t["alpha_over_alpha0"] = [None if (x == 0 or r["alpha_track_deg"] != r["alpha_track_deg"]) else
                              r6(r["alpha_track_deg"] / x) for x, r in zip(thetas, rows)]
    t["nonfinite_instances"] = sum(1 for r in rows if r["nonfinite"])
    return t


def orientation_physics(stream, n, steps):
    """The orientation sweep's physical output (growth angle and tip velocity
    vs crystal angle) for the three 2D schemes, FP32, after `steps` steps, and
    FP32 against FP64 for one angle of S-bar_{2,1}."""
    import math

    import numpy as np

    from paper_2110_12448_gb300 import synth
    w0 = synth.free_dendrite_2d(n, 0.0, "SBAR21", steps=steps)
    out = {"grid": f"10 x {n}^2", "steps": steps, "ivantsov_peclet": ivantsov_peclet_2d(-w0.U0), "schemes": {}}
    i30 = THETAS.index(int(PHYS_FP64_THETA))
    for scheme in PHYS_SCHEMES:
        ws = [synth.free_dendrite_2d(n, float(t), scheme, steps=steps) for t in THETAS]
        ms, rows, tile, f32 = run_batch(stream, ws, "f32", keep=(i30,) if scheme == "SBAR21" else ())
        out["schemes"][scheme] = dict(_table(THETAS, rows), glups=round(len(ws) * ws[0].n_cells * steps / ms / 1e6, 3),
                                      device_s=round(ms / 1e3, 3), tile=list(tile),
                                      fp64_batch_glups=round(batch_rate(stream, ws, "f64", PHYS_FP64_BATCH_STEPS), 3))
        if scheme == "SBAR21":
            w64 = [synth.free_dendrite_2d(n, PHYS_FP64_THETA, scheme, steps=steps)]
            ms64, rows64, _, f64 = run_batch(stream, w64, "f64", keep=(0,))
            (p32, u32), (p64, u64) = f32[i30], f64[0]
            s2 = math.sqrt(2.0)
            r32 = rows[i30]
            out["fp32_vs_fp64"] = {
                "scheme": scheme, "theta_deg": PHYS_FP64_THETA, "steps": steps,
                "max_abs_dphi": float(np.max(np.abs(np.tanh(p32.astype(np.float64) / s2) - np.tanh(p64 / s2)))),
                "max_abs_dU": float(np.max(np.abs(u32.astype(np.float64) - u64))),
                "v_tip_f32": r32["v_tip"], "v_tip_f64": rows64[0]["v_tip"],
                "v_tip_rel_err": abs(r32["v_tip"] - rows64[0]["v_tip"]) / abs(rows64[0]["v_tip"]),
                "alpha_deg_f32": r32["alpha_deg"], "alpha_deg_f64": rows64[0]["alpha_deg"],
                "fp64_glups": round(w64[0].n_cells * steps / ms64 / 1e6, 3)}
    return out


def run_paper2d(args):
    """The isothermal runs of Sec. 4.3.2 (781^2, h/W = 1.2, W/d0* = 16,
    eps4 = 0.014, Omega = 0.43, k = 0.1, 20 345 steps): for each 2D scheme the
    ten crystal angles as one batch, and one run alone, timed on the device;
    with the tip state (growth angle, tip velocity, tip radius, sigma*) at the
    paper's measuring time and the paper's seconds per run on a P100 beside."""
    import torch

    from paper_2110_12448_gb300 import synth
    stream = torch.cuda.Stream()
    clocks = Clocks(0)
    res = {}
    cells = 0
    total_ms = 0.0
    with clocks:
        for scheme in PHYS_SCHEMES:
            ws = [synth.paper_isothermal_2d(float(t), scheme) for t in THETAS]
            ms, rows, tile, _ = run_batch(stream, ws, "f32")
            one = [synth.paper_isothermal_2d(30.0, scheme)]
            ms1, _, tile1, _ = run_batch(stream, one, "f32")
            cells += len(ws) * ws[0].n_cells * ws[0].steps
            total_ms += ms
            res[scheme] = dict(_table(THETAS, rows), s_per_run_in_batch=round(ms / 1e3 / len(ws), 4),
                               s_per_run_alone=round(ms1 / 1e3, 4), paper_p100_s_per_run=PAPER_TABLE1_S[scheme],
                               tile_batch=list(tile), tile_alone=list(tile1),
                               glups_batch=round(len(ws) * ws[0].n_cells * ws[0].steps / ms / 1e6, 3))
    w = synth.paper_isothermal_2d(0.0, "SBAR21")
    line = {"metric": METRIC, "value": cells / (total_ms / 1e3) / 1e9, "unit": "GLUPS", "n_gpus": 1,
            "steps": w.steps, "warmup": 0, "ms_per_step": total_ms / (len(PHYS_SCHEMES) * w.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"isothermal runs of Sec. 4.3.2: {w.nx}^2, h/W = {w.h}, W/d0* = 16, eps4 = "
                                   f"{w.eps4}, Omega = {-w.U0}, k = {w.k}, {w.steps} steps; 10 crystal angles x "
                                   f"{len(PHYS_SCHEMES)} schemes (one batch per scheme), FP32 fields",
                       "cells_per_gpu": 10 * w.n_cells},
            "clocks": clocks.summary(), "ivantsov_peclet": ivantsov_peclet_2d(-w.U0), "paper_runs": res}
    print(json.dumps(line), flush=True)
    return 0


# Table 2: seconds per isothermal 3D run of Sec. 6.2.2 on one Tesla P100 (context)
PAPER_TABLE2_S = {"S100": 5445.0, "SBAR120": 25155.0}
PAPER3D_THETAS = (0.0, 15.0, 30.0)


def run_paper3d(args):
    """The isothermal 3D runs of Sec. 6.2.2 (h/W = 1.2, W/d0* = 16,
    eps4 = 0.014, Omega = 0.25, k = 0.1, crystal turned about z by
    alpha0 = 0, 15, 30 deg, to t = 1.5e6 d0*^2 / D) in a 320^3 cube (the
    paper's cube of side 9.6e4 d0* does not fit one GPU), one run at a time:
    growth angle by tip tracking, tip radii, sigma*, seconds per run beside
    Table 2."""
    import torch

    from paper_2110_12448_gb300 import synth
    stream = torch.cuda.Stream()
    clocks = Clocks(0)
    n = args.n
    res = {}
    cells = 0
    total_ms = 0.0
    with clocks:
        for scheme in ("S100", "SBAR120"):
            ws = [synth.paper_isothermal_3d(t, scheme, n=n) for t in PAPER3D_THETAS]
            rows, secs = [], []
            for w in ws:
                ms, r, tile, _ = run_batch(stream, [w], "f32")
                rows += r
                secs.append(round(ms / 1e3, 3))
                cells += w.n_cells * w.steps
                total_ms += ms
            res[scheme] = dict(_table(PAPER3D_THETAS, rows), s_per_run=secs,
                               paper_p100_s_per_run=PAPER_TABLE2_S[scheme], tile=list(tile))
    w = synth.paper_isothermal_3d(0.0, "SBAR120", n=n)
    line = {"metric": METRIC, "value": cells / (total_ms / 1e3) / 1e9, "unit": "GLUPS", "n_gpus": 1,
            "steps": w.steps, "warmup": 0, "ms_per_step": total_ms / (2 * len(PAPER3D_THETAS) * w.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"isothermal 3D runs of Sec. 6.2.2 in a {n}^3 cube: h/W = {w.h}, W/d0* = 16, "
                                   f"eps4 = {w.eps4}, Omega = {-w.U0}, k = {w.k}, {w.steps} steps; alpha0 = 0, 15, "
                                   f"30 deg about z x S_100, S-bar_120, FP32 fields", "cells_per_gpu": w.n_cells},
            "clocks": clocks.summary(), "paper_runs": res}
    print(json.dumps(line), flush=True)
    return 0


PAPER_DS_THETAS = (0.0, 30.0)
PAPER_DS_STEPS = 4000000


def run_paper_ds2d(args):
    """The 2D directional runs of Sec. 4.3.3 in model units (synth.
    paper_directional_2d): one dendrite per box at alpha0 = 0 and 30 deg for
    the three 2D schemes, the box following the tip (pf_shift_frame keeps the
    most advanced interface along +y, observed with pf_observe(-2), between 50
    and 60% of its height).  Reports the steady tip undercooling
    Delta = 1 - zeta_tip (mean and spread over the last quarter of the run),
    the tip speed against Vp, and delta(alpha0) = (Delta(alpha0) - Delta(0)) lT,
    the distance between the tips that Fig. 2D_DS compares across schemes."""
    import torch

    from paper_2110_12448_gb300 import native as N
    from paper_2110_12448_gb300 import synth
    stream = torch.cuda.Stream()
    steps = args.steps if args.steps != 2000 else PAPER_DS_STEPS
    chunk = min(100000, max(1, steps // 20))  # observations (and frame moves) per run: about 20 or more
    clocks = Clocks(0)
    res = {}
    cells = 0
    total_ms = 0.0
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    with clocks:
        for scheme in ("SBAR21", "S21", "S10"):
            res[scheme] = {}
            for th in PAPER_DS_THETAS:
                w = synth.paper_directional_2d(th, scheme)
                with torch.cuda.stream(stream):
                    s = N.Sim.from_workload(w, "f32", stream=stream)
                s.set_tile(64, 1, 8)  # one instance: short sweeps fill the GPU
                off, done, hist = 0.0, 0, []
                while done < steps:
                    k = min(chunk, steps - done)
                    a.record(stream)
                    s.step(k)
                    b.record(stream)
                    b.synchronize()
                    total_ms += a.elapsed_time(b)
                    done += k
                    o = s.observe(-2)
                    yt = o["tip"][1]
                    zeta = (yt - (w.yT - off) - w.Vp * done * w.dt) / w.lT
                    hist.append((done, yt + off, 1.0 - zeta))
                    if yt > 0.6 * w.ny * w.h:
                        rows = int((yt - 0.5 * w.ny * w.h) / w.h)
                        s.shift_frame(rows)
                        off += rows * w.h
                cells += w.n_cells * steps
                q = max(1, len(hist) // 4)  # the last quarter of the observations
                last = [d for _, _, d in hist[-q:]]
                (n1, y1, _), (n2, y2, _) = hist[max(0, len(hist) - q - 1)], hist[-1]
                v = (y2 - y1) / ((n2 - n1) * w.dt) if n2 > n1 else float("nan")
                res[scheme][f"{th:g}"] = {"Delta": statistics.fmean(last), "Delta_spread": max(last) - min(last),
                                          "v_tip": v, "Vp": w.Vp,
                                          "frame_moved_W": off}
                s.close()
            base = res[scheme]["0"]["Delta"]
            for th in PAPER_DS_THETAS[1:]:
                r = res[scheme][f"{th:g}"]
                r["delta_W"] = (r["Delta"] - base) * w.lT
                r["delta_um"] = r["delta_W"] * math.sqrt(1270.0 * (1e-5 / w.dt) / w.D)  # W in um (synth's mapping)
    w = synth.paper_directional_2d(0.0)
    line = {"metric": METRIC, "value": cells / (total_ms / 1e3) / 1e9, "unit": "GLUPS", "n_gpus": 1, "steps": steps,
            "warmup": 0, "ms_per_step": total_ms / (3 * len(PAPER_DS_THETAS) * steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"directional runs of Sec. 4.3.3 in model units: {w.nx}x{w.ny}, Vp = {w.Vp:.4f} "
                                   f"W/tau0, lT = {w.lT:.0f} W, h/W = {w.h}, eps4 = {w.eps4}, k = {w.k}, periodic x, "
                                   f"box following the tip, alpha0 = 0 and 30 deg x three schemes, {steps} steps each, "
                                   f"FP32 fields", "cells_per_gpu": w.n_cells},
            "clocks": clocks.summary(), "paper_ds_runs": res}
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    """Served stream: Poisson arrivals of mixed 2D/3D runs (sizes and step
    counts scaled by --serve-scale), continuous batching by an 80 % HBM
    budget; reports aggregate GLUPS and p50/p99 time-to-result."""
    import torch

    from paper_2110_12448_gb300 import serve, synth
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    reqs = synth.request_stream(rate_per_s=args.rate, window_s=args.window, size_scale=args.serve_scale,
                                steps_scale=args.serve_scale)
    rq = [serve.Request(i, r.workload, r.workload.steps, "f32", r.arrival_s) for i, r in enumerate(reqs)]
    srv = serve.Server(budget_frac=0.8, chunk=100, n_streams=args.streams)
    with Clocks(local) as clocks:
        srv.run(rq)
    summ = srv.summary()
    srv.close()
    if rank == 0:
        line = {"metric": METRIC, "value": summ["glups"], "unit": "GLUPS", "n_gpus": world, "steps": len(rq),
                "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"served mixed stream: Poisson {args.rate}/s over {args.window} s, 2D "
                                       f"128..2048 and 3D 64..192 scaled by {args.serve_scale}, 1-16 seeds, U0 in "
                                       f"[-0.7,-0.4], 1000..20000 steps scaled by {args.serve_scale}, 80% HBM budget"},
                "latency_s": {"p50": summ["p50_s"], "p99": summ["p99_s"], "of": "time to result"},
                "requests": summ["requests"], "wall_s": summ["wall_s"], "clocks": clocks.summary(),
                "cell_updates": {"2d": summ["cell_updates_2d"], "3d": summ["cell_updates_3d"]},
                "max_running": summ["max_running"], "peak_bytes": summ["peak_bytes"],
                "budget_bytes": summ["budget_bytes"]}
        print(json.dumps(line), flush=True)
    return 0


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    from oracle import oracle as O
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
    ws = workloads(args.n, args.scheme)
    states = []
    for w in ws:
        p = O.params(nx=w.nx, ny=w.ny, scheme={"SBAR21": 2, "S21": 1, "S10": 0}[args.scheme], h=w.h, dt=w.dt, k=w.k,
                     eps4=w.eps4, lam=w.lam, D=w.D)
        psi, U, g = O.init_seeds(p, w.U0, w.seeds, w.seed_grain)
        states.append([p, w, psi, U, g])

    def one(i):
        p, w, psi, U, g = states[i % len(states)]
        psi, U = O.step(p, w.rots, g, psi, U, 1)
        states[i % len(states)][2:4] = [psi, U]
        return w.n_cells

    for i in range(args.warmup):
        one(i)
    t0 = time.perf_counter()
    cells = 0
    for i in range(args.steps):
        cells += one(args.warmup + i)
    dt = time.perf_counter() - t0
    v = cells / dt / 1e9
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"metric": METRIC, "value": v, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"orientation sweep 2D, 10 x {args.n}^2, {args.scheme}", "sample":
                       "one instance-step per step, cycling alpha0", "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": v, "unit": "GLUPS", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} instance-steps of {args.n}^2"},
            "e2e": {"value": v, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_native(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2110_12448_gb300 import native as N

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    stream = torch.cuda.Stream()
    ws = workloads(args.n, args.scheme, args.workload)
    for w in ws:
        if args.time_level == "t0" or args.kernels == "two":
            w.time_level = 1
        if args.kernels == "two":
            w.kernels = 1
    # the clock sampler runs from before the autotuner (seconds of load on a
    # fresh box) to the end of the timed region
    clocks = Clocks(local, window="the autotuner, the warm-up and the timed region")
    clocks.__enter__()
    tile, tune_times = None, {}
    if args.tile:
        from paper_2110_12448_gb300 import autotune
        tile = tuple(int(x) for x in args.tile.split(","))
    elif not args.no_tune:
        from paper_2110_12448_gb300 import autotune
        tile, tune_times = autotune.tune(ws, args.precision, n_streams=args.streams)
    # the batch as `args.streams` groups on their own streams (forked from and
    # joined to `stream` around every run of steps): one group's launches fill
    # the tail of the other's persistent launch
    from paper_2110_12448_gb300.batch import Batch
    batch = Batch(ws, args.precision, n_streams=args.streams, tile=tile)
    sims = batch.members
    cells = batch.n_cells
    observes = [0]

    def steps(k):
        """k steps with the FP64 observe of every instance every OBS_EVERY
        steps and after the last one; returns event pairs around the step
        launches alone (fork to join), without the observes."""
        done = 0
        pairs = []
        while done < k:
            chunk = min(OBS_EVERY - (batch.steps_done % OBS_EVERY), k - done)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            batch.step(chunk, use_graph=True, stream=stream)
            b.record(stream)
            pairs.append((a, b, chunk))
            done += chunk
            if batch.steps_done % OBS_EVERY == 0 or done == k:
                batch.observe(0)  # every instance, one synchronisation per group
                observes[0] += 1
        return pairs

    steps(args.warmup)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    observes[0] = 0
    clocks.mark()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    pairs = steps(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks.mark()
    clocks.__exit__()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    kern_ms = sum(a.elapsed_time(b) for a, b, _ in pairs)
    n_launch = sum(c for _, _, c in pairs)
    n_observe = observes[0]
    ms, value = aggregate(ms, cells, args.steps, world, device="cuda")

    # per-step latency after the timed region: 200 single steps of the batch,
    # each launched directly and bracketed by its own events
    lat = []
    for _ in range(200):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        batch.step(1, use_graph=False, stream=stream)
        b.record(stream)
        lat.append((a, b))
    torch.cuda.synchronize()
    per_step = sorted(a.elapsed_time(b) for a, b in lat)

    # latency of the device tip-radius fit (pf_tip_radius, host round trip
    # included) on the sweep's instances after the timed region; the physical
    # tip state is measured by orientation_physics at the sweep's full length
    sweep = None
    if args.workload == "sweep2d" and rank == 0:
        tr_s = []
        for s in sims:
            ob = s.observe(0)
            t0 = time.perf_counter()
            s.tip_radius(ob, 0)
            tr_s.append(time.perf_counter() - t0)
        sweep = {"tip_radius_call_ms_p50": statistics.median(tr_s) * 1e3, "at_step": sims[0].steps_done}

    # directional solidification: most advanced tip of each misorientation relative to
    # the isotherm T0 and the distance to the well-oriented grain's tip (Sec. 4.2)
    if args.workload == "directional2d" and rank == 0:
        tips = []
        for s in sims:
            ob = s.observe(0)
            tips.append(ob["tip"][1] if ob["found"] else float("nan"))
        t_now = sims[0].steps_done * ws[0].dt
        sweep = {"theta_deg": list(DS_THETAS), "tip_y": [round(v, 4) for v in tips],
                 "isotherm_y": round(ws[0].yT + DS_VP * t_now, 4),
                 "delta": [round(tips[0] - v, 4) for v in tips], "at_step": sims[0].steps_done}

    # roofline of the fused step kernel: algorithmic bytes per launch / mean launch time
    peak, peak_kind = peaks()
    bpc = bytes_per_cell(ws, args.precision, two=args.kernels == "two")
    achieved = cells * bpc / (kern_ms / n_launch / 1e3) / 1e9
    tname = {"f32": "float", "f64": "double", "f32c": "float, compensated state"}[args.precision]
    kname = ("k_step2d" if ws[0].dim == 2 else "k_step3d") + f"<{tname},{args.scheme}>"
    if args.kernels == "two":
        kname += " psi pass + U pass (two-kernel form, T0)"
    elif args.time_level == "t0":
        kname += " (T0)"
    default_path = args.precision == "f32" and args.kernels == "fused" and args.time_level == "t1"
    fpc = _captured(FLOPS, args.workload, "flop_per_cell", tile) \
        if default_path and args.scheme in ("SBAR21", "SBAR120") else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic_for(args.workload, tile) if default_path else None, "peak_source": peak_kind,
            "bytes_per_cell": bpc, "kernel": kname,
            "timing": "step launches of the whole batch, fork to join of its group streams, observes excluded"}
    roof_alu = None
    if fpc:
        tf = cells * fpc / (kern_ms / n_launch / 1e3) / 1e12
        roof_alu = {"bound": "alu", "achieved": tf, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": tf / FP32_PEAK_TFLOPS, "flop_per_cell": fpc, "kernel": kname,
                    "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
                    "flop_source": "ncu thread-instruction counts of one launch (FADD, FMUL, FFMA and packed pairs)"}

    # end to end through the public API, as a client pipelines a batch: the
    # instances split into `args.e2e_parts` parts, each a group on its own
    # stream; per part, its state queued in from pinned host buffers
    # (pf_set_fields_async), the K steps with their observes
    # (pf_group_observe), the state queued back out (pf_get_fields_async)
    # right after the part's last observe.  One part's copies overlap the
    # other parts' steps; all inside the timed region, from the first upload
    # to the last download.
    e2e = None
    if not args.no_e2e:
        dt_np = np.float32 if args.precision == "f32" else np.float64
        host = []
        for s in sims:
            hp = torch.empty(s.shape, dtype=torch.float32 if dt_np == np.float32 else torch.float64).pin_memory()
            hu = torch.empty_like(hp).pin_memory()
            s.get_fields(out=(hp.numpy(), hu.numpy()))
            host.append((hp, hu))
        n_parts = max(1, min(args.e2e_parts, len(ws)))
        parts = [list(range(len(ws)))[k::n_parts] for k in range(n_parts)]
        pipes = []
        for idx in parts:
            if not idx:
                continue
            st_ = torch.cuda.Stream()
            ss = []
            with torch.cuda.stream(st_):
                for i in idx:
                    ss.append(N.Sim.from_workload(ws[i], args.precision, stream=st_, init=False))
                    # the grain map is part of the problem, not of the per-step state: the
                    # same map as the measured instance, set before the timed region
                    ss[-1].set_grain_index(sims[i].get_grain_index())
                    if tile:
                        ss[-1].set_tile(*autotune.split(tile)[0])
            g_ = N.Group(len(ss), sum(N.Group.work_items(x) for x in ss), stream=st_)
            for x in ss:
                g_.add(x)
            if tile:
                g_.set_depth(*autotune.split(tile)[1])
            pipes.append((st_, ss, g_, [host[i] for i in idx]))
        for st_, ss, g_, hh in pipes:  # untimed warm-up of the new groups (graph capture)
            for x, (hp, hu) in zip(ss, hh):
                x.set_fields_async(hp.numpy(), hu.numpy())
            g_.step(max(args.warmup, 16), use_graph=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for st_, ss, g_, hh in pipes:
            for x, (hp, hu) in zip(ss, hh):
                x.set_fields_async(hp.numpy(), hu.numpy())
        done = 0
        while done < args.steps:
            at = pipes[0][1][0].steps_done
            chunk = min(OBS_EVERY - (at % OBS_EVERY), args.steps - done)
            for st_, ss, g_, hh in pipes:
                g_.step(chunk, use_graph=True)
            done += chunk
            last = done == args.steps
            if (at + chunk) % OBS_EVERY == 0 or last:
                for st_, ss, g_, hh in pipes:
                    g_.observe(0)
                    if last:  # this part's state back out while the other parts still step
                        for x, (hp, hu) in zip(ss, hh):
                            x.get_fields_async(hp.numpy(), hu.numpy())  # straight into the pinned buffers
        h2d = d2h = 0
        for st_, ss, g_, hh in pipes:
            for x, (hp, hu) in zip(ss, hh):
                h2d += hp.numel() * hp.element_size() * 2
                d2h += hp.numel() * hp.element_size() * 2
        for st_, ss, g_, hh in pipes:
            st_.synchronize()
        e2e_s = time.perf_counter() - t0
        for st_, ss, g_, hh in pipes:
            g_.close()
            for x in ss:
                x.close()
        e2e = {"value": cells * args.steps * world / e2e_s / 1e9, "unit": "GLUPS",
               "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps,
               "copies": f"{len(pipes)} parts of the batch on their own streams, each: pf_set_fields_async from "
                         "pinned host buffers, the steps and observes, pf_get_fields_async into them after its last "
                         "observe; one part's copies overlap the other parts' steps"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
                "config": {"workload": WORKLOAD_TEXT[args.workload].format(n=args.n, n2=2 * args.n, scheme=args.scheme) +
                                       (", T0 time level" if args.time_level == "t0" or args.kernels == "two" else "") +
                                       (", two-kernel form (psi kernel stores d psi/dt, then the U kernel)"
                                        if args.kernels == "two" else "") +
                                       f", {args.precision.upper()} fields, batched persistent launches + CUDA graphs as "
                                       f"{len(batch.groups)} group(s) on their own streams, "
                                       f"FP64 observe of every instance every {OBS_EVERY} steps and after the last "
                                       f"timed step ({n_observe} inside the timed region)",
                           "cells_per_gpu": cells,
                           "l2": f"state {cells * 2 * (4 if args.precision == 'f32' else 8) / 1e6:.0f} MB per step "
                                 f"> 129 MB L2, no flush"},
                "roofline": roof, "roofline_alu": roof_alu, "e2e": e2e, "clocks": clocks.summary(),
                "latency_ms_per_step": {"p50": statistics.median(per_step),
                                        "p99": per_step[min(len(per_step) - 1, int(0.99 * len(per_step)))],
                                        "over": f"{len(per_step)} single steps of the whole batch after the timed "
                                                f"region, each launched directly with its own events"},
                "tile": list(tile) if tile else None,
                # a depth-2 step is one launch per band (one class per group here)
                "gpu_launches": (n_launch * (autotune.bands(ws, tile) if tile else 1) + 2 * n_observe)
                                * len(batch.groups)}
        if tune_times:
            # temporal-blocking depth as the autotuner raced it (ms per step of the batch)
            line["depth_race"] = autotune.depth_race(tune_times)
        if sweep:
            line["directional" if args.workload == "directional2d" else "tip_radius_call"] = sweep
        if world == 1 and not args.no_fp64:
            line["fp64_plain"] = fp64_plain(stream)
        if world == 1 and args.workload == "sweep2d" and args.precision == "f32" and not args.no_fp64:
            line["at_stated_error"] = at_stated_error(stream, ws, max(200, args.steps), args.streams)
        if world == 1 and not args.no_physics and args.workload == "sweep2d":
            line["orientation_physics"] = orientation_physics(stream, args.n, PHYS_STEPS)
        if world == 1 and not args.no_cpu and args.workload == "sweep2d":
            line["cpu_baseline"] = cpu_baseline(args.n, args.scheme)
        print(json.dumps(line), flush=True)
    batch.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="f32", choices=["f32", "f64", "f32c"],
                    help="f32c: FP32 arithmetic on the compensated (hi + lo) state, 2D")
    ap.add_argument("--time-level", default="t1", choices=["t1", "t0"])
    ap.add_argument("--e2e-parts", type=int, default=2,
                    help="parts of the batch in the end-to-end measurement, each on its own stream")
    ap.add_argument("--streams", type=int, default=2,
                    help="groups the batch is split into, each on its own CUDA stream (fewer for fewer instances)")
    ap.add_argument("--kernels", default="fused", choices=["fused", "two"],
                    help="two: the psi kernel stores d psi/dt, then the U kernel (2D, T0)")
    ap.add_argument("--scheme", default="SBAR21", choices=["SBAR21", "S21", "S10", "SBAR120", "S100"])
    ap.add_argument("--n", type=int, default=None,
                    help="grid side (default 1024 in 2D, 256 for dendrite3d, 320 for paper3d)")
    ap.add_argument("--workload", default="sweep2d", choices=["sweep2d", "dendrite3d", "poly2d", "directional2d", "serve", "paper2d", "paper3d", "paper_ds2d"])
    ap.add_argument("--rate", type=float, default=20.0, help="serve: arrivals per second")
    ap.add_argument("--window", type=float, default=20.0, help="serve: arrival window in seconds")
    ap.add_argument("--serve-scale", type=float, default=0.25, help="serve: scale of sides and step counts")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end host-buffer run")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparator")
    ap.add_argument("--no-tune", action="store_true", help="use the default tile instead of the autotuner's")
    ap.add_argument("--tile", default=None,
                    help="force a tile instead of the autotuner's: block_x,block_y,sweep[,depth,band_sweeps]")
    ap.add_argument("--no-physics", action="store_true",
                    help="skip the orientation sweep's tip-state runs (three schemes to 2e4 steps, FP64 check)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.n is None:
        args.n = {"dendrite3d": 256, "paper3d": 320}.get(args.workload, 1024)
    if args.workload == "dendrite3d" and args.scheme in ("SBAR21", "S21", "S10"):
        args.scheme = {"S10": "S100"}.get(args.scheme, "SBAR120")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "paper2d":
        return run_paper2d(args)
    if args.workload == "paper3d":
        return run_paper3d(args)
    if args.workload == "paper_ds2d":
        return run_paper_ds2d(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
