"""Benchmark of the LOSS time step on one GB300 (or N replicas, one per GPU).

Workload: the 2-D acoustic layered model on 2049 x 2049 points in 8 x 8 patches (M = 256), PMBC halo width 20,
h = 10 m, 3-layer velocity (1500/2500/3500 m/s) times a 5 % Gaussian-correlated perturbation (seed 2002),
Ricker 20 Hz at the centre, CFL 0.4, a 40-point ADE-PML layer on every side.  One step = one Strang step of
the whole hot path (PMBC closures, local spline solves, derivatives, velocity-stress update, PML memory
variables, source, receivers on the top row).  Headline precision: FP32 fields with Kahan-compensated updates
(PMBC sums in FP64); the FP64 form is measured alongside.

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events on the library's stream, with an L2
flush (write + read of a buffer larger than L2) between timed steps; barrier + synchronize around the timed
region; the max over ranks is reported.  value = whole-job grid-point updates per second (sum over ranks).
Per-kernel launch durations (roofline) come from a second pass of K flushed steps with a CUDA event pair around
every launch; those events cost ~2 us per launch on the GPU and are kept out of the headline steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import datetime
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grid-pt updates/s per step on 1 GB300 (FP32 vs FP64) at stated L2 err; HBM GB/s frac"
UNIT = "pt-upd/s"
WORKLOAD = "acoustic2d_layered 2049x2049 pts, 8x8 patches (M=256), n_nb=20, PML 40, 3-layer + 5% noise, Ricker 20 Hz"


# Source files of the FP32 step's kernels; a DRAM-traffic figure from ncu is valid only for the sources it was taken on.
KERNEL_SOURCES = ("paper_2301_05127_gb300/csrc/loss_kernels_tiled.cu", "paper_2301_05127_gb300/csrc/loss_fir.cuh",
                  "paper_2301_05127_gb300/csrc/loss_line.cuh", "paper_2301_05127_gb300/csrc/loss_block.cuh",
                  "paper_2301_05127_gb300/csrc/loss_types.h")
KERNEL_OF = {"acoustic_x": "k_xp", "acoustic_z": "k_tz<1", "acoustic_z2": "k_tz<2"}


def kernel_sources_digest():
    """Digest of the kernel sources without comments and whitespace (a comment edit leaves the kernels as they
    were captured)."""
    import hashlib
    import re

    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p)) as f:
            code = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
        code = re.sub(r"//[^\n]*", "", code)
        h.update("".join(code.split()).encode())
    return h.hexdigest()[:16]


def _traffic(kernel):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of one ncu capture of the kernel, from
    profiles/dram_traffic.txt (lines: <kernel> <bytes per launch> <sources digest>), or None when no capture of the
    current sources exists."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    digest = kernel_sources_digest()
    for line in open(path):
        f = line.split()
        if len(f) >= 3 and not line.startswith("#") and f[0] == kernel and f[2] == digest:
            return float(f[1])
    return None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def max_over_ranks(x, ws, device):
    """The largest x over the ranks of the process group (x itself for one process)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(ws, points, ms_per_step):
    """Whole-job grid-point updates per second: every rank advances its own replica of the workload, and the step
    time is the slowest rank's."""
    return ws * points / (ms_per_step * 1e-3)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, window=None):
        """Median SM clock and the throttle reasons seen; window = (t0, t1) in time.time() seconds keeps only the
        samples taken inside it (all samples when none falls inside)."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                ts = None
            try:
                rows.append((ts, float(parts[2]), float(parts[3]), parts[6:10]))
            except ValueError:
                continue
        if window is not None:
            inside = [r for r in rows if r[0] is not None and window[0] - 0.25 <= r[0] <= window[1] + 0.25]
            rows = inside or rows
        sm = [r[1] for r in rows]
        smax = [r[2] for r in rows]
        reasons = set()
        for r in rows:
            for nm, v in zip(names, r[3]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _flusher(torch, dev):
    """Write then read a 512 MiB buffer (L2 is ~129 MiB): evicts our data and leaves clean lines."""
    a = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device=dev)
    b = torch.ones(128 * 1024 * 1024, dtype=torch.float32, device=dev)

    def flush():
        a.fill_(1.0)
        b.sum()

    return flush


def _timed_steps(torch, g, steps, flush):
    st = torch.cuda.current_stream()
    times = []
    for _ in range(steps):
        flush()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        g.step(1)
        e1.record(st)
        times.append((e0, e1))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in times]


KERNELS = ("acoustic_x", "acoustic_z", "acoustic_z2")

# Algorithmic bytes per point-step of one whole step (FP32): every state array and the model read once and every
# state array written once.  2-D acoustic: sigma, v1, v3 read and written, kappa read (the benchmark's density
# is constant, so the buoyancy is a scalar): 7 x 4 = 28 B; the FP32 compensation arrays of the three fields
# add 3 x 2 x 4 = 24 B.  3-D elastic, constant model: nine fields read and written, 18 x 4 = 72 B.
STEP_ALG_BYTES, STEP_COMP_BYTES = 28, 24
ELASTIC_ALG_BYTES = 72


def _alg_bytes_per_point(kernel, esize, kahan, b_array):
    """Algorithmic DRAM bytes per grid point of one launch of the FP32 step's kernels: every array the kernel must
    touch, once (the density of the benchmark model is constant, so the buoyancy is a scalar and no b array is
    read)."""
    if kernel == "acoustic_x":
        # read v1, sigma, kappa, d_z v3; write sigma, v1 (+ compensation of sigma and v1, read and written)
        n = 4 + 2 + (4 if kahan else 0) + (1 if b_array else 0)
    elif kernel == "acoustic_z":
        # read sigma, v3; write v3 (+ compensation of v3, read and written)
        n = 2 + 1 + (2 if kahan else 0) + (1 if b_array else 0)
    else:
        # read v3; write d_z v3
        n = 2
    return n * esize


def _batched_leg(torch, pkg, units, warmup_units, k):
    """The 64-shot survey (n_s from 512 to 2048, M = 128, FP32): tile shapes from the library's autotuner, then
    timed replays of a captured graph of k batched steps (one persistent launch per kernel per step).  The shots
    hold ~4.5 GB, far more than L2, so no flush is needed between replays."""
    from synth import batched_shots

    ws = batched_shots(steps=k)
    pts = sum(w.points for w in ws)
    g = pkg.Grid.from_workloads(ws)
    g.set_schedule(True, k)
    tune = g.autotune(steps=2)
    st = torch.cuda.current_stream()
    for _ in range(warmup_units):
        g.step(k)
    g.sync()
    ev = []
    for _ in range(units):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        g.step(k)
        e1.record(st)
        ev.append((e0, e1))
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev) / (units * k)
    launches = g.profile_read(-1)[1]
    conv = g.profile_read("acoustic_z2")[1] > 0  # the convolution kernels split z into Z1 and Z2
    g.close()
    peak, kind = _peaks()
    # Algorithmic bytes per point-step: the step's 28 B (sigma, v1, v3 read and written, kappa read).  The kernels
    # themselves touch 44 B (convolution: x 24, Z1 12, Z2 8, with the d_z v3 temporary) or 40 B (line kernels).
    alg = STEP_ALG_BYTES
    own = 44 if conv else 40
    value = pts / (ms * 1e-3)
    return {"workload": f"{len(ws)} shots, n from {min(w.n[0] for w in ws)} to {max(w.n[0] for w in ws)}, M=128, "
                        f"n_nb=20, PML 40, FP32, graph of {k} steps",
            "kernels": "truncated-convolution" if conv else "line",
            "points_per_step": pts, "value": value, "unit": UNIT, "ms_per_step": ms,
            "alg_bytes_per_point": alg, "alg_frac_of_peak": value * alg / (peak * 1e9),
            "kernel_bytes_per_point": own, "kernel_bytes_frac_of_peak": value * own / (peak * 1e9),
            "peak_kind": peak_kind_note(kind),
            "autotune": tune, "launches": launches, "l2": "working set 4.5 GB, no flush"}


# GB300's FP64 FMA rate, from its unit counts and clock: 152 SMs x 2 DFMA per clock x 2.07 GHz (1.26 TFLOP/s, the
# nominal 1.25 TFLOP/s of the part).
FP64_DFMA_PER_S = 152 * 2 * 2.07e9


def _junction_taps(n, c, radius):
    """FP64 FMAs of one junction sum at position c of an n-interval line (taps m in [-radius, radius], clipped to
    the line)."""
    return min(radius, c) + min(radius, n - c) + 1


def elastic_dfma_per_point_step(n, p, n_nb, K=16):
    """FP64 FMAs per point-step of the FP32 elastic step on an n^3 grid with p patches per axis: the x passes sum
    every junction of a line once for each of their 6 derivatives (PMBC sums, radius n_nb); the y / z tiles sum
    both junctions of their patch for each of their 12 derivatives (junction corrections, radius max(n_nb, K))."""
    M = n // p
    line = sum(_junction_taps(n, j * M, n_nb) for j in range(p + 1))
    rd = max(n_nb, K)
    tiles = sum(_junction_taps(n, l * M, rd) + _junction_taps(n, (l + 1) * M, rd) for l in range(p))
    return (6 * line + 12 * tiles) / (n + 1)


def _elastic_leg(torch, pkg, steps, warmup, flush):
    """The homogeneous 3-D elastic workload (257^3 points, 4 x 4 x 4 patches, n_nb = 20, 20-point layers,
    explosive + shear source, v1..v3 receivers on z = 20), FP32 with compensated updates, tile shapes from the
    library's autotuner, per-step events with an L2 flush in between; per-kernel times from the library's
    events."""
    from synth import elastic3d_homogeneous

    w = elastic3d_homogeneous(precision="fp32_kahan")
    g = pkg.Grid.from_workloads([w])
    tune = g.autotune(steps=2)
    g.step(warmup)
    g.sync()
    g.profile(True)
    ms = _timed_steps(torch, g, steps, flush)
    kern = {k: g.profile_read(k) for k in ("elastic_x", "elastic_y", "elastic_z")}
    g.close()
    ms_step = sum(ms) / len(ms)
    peak, kind = _peaks()
    # Algorithmic bytes per point-step of the elastic step with a constant model: the nine FP32 fields read and
    # written once, 72 B; the compensation arrays of the nine fields add another 72 B (read and written once).
    # Derivative temporaries are not algorithmic.
    alg, alg_comp = ELASTIC_ALG_BYTES, 2 * ELASTIC_ALG_BYTES
    value = w.points / (ms_step * 1e-3)
    # The PMBC sums stay in FP64, and GB300's FP64 rate is low: their FMAs set a floor above the HBM one.
    dfma = elastic_dfma_per_point_step(w.n[0], w.p[0], w.n_nb)
    fp64_floor_ms = 1e3 * w.points * dfma / FP64_DFMA_PER_S
    return {"workload": "elastic3d_homogeneous 257^3 pts, 4x4x4 patches (M=64), n_nb=20, PML 20, FP32 + Kahan",
            "value": value, "unit": UNIT, "ms_per_step": ms_step,
            "fp64": {"bound": "alu", "dfma_per_point_step": dfma, "floor_ms": fp64_floor_ms,
                     "frac": fp64_floor_ms / ms_step, "peak_tflops": 2e-12 * FP64_DFMA_PER_S,
                     "peak_kind": "derived: 152 SMs x 2 FP64 FMA per clock x 2.07 GHz"},
            "kernels_ms_per_step": {k: v[0] / steps for k, v in kern.items()},
            "alg_bytes_per_point": alg, "alg_frac_of_peak": value * alg / (peak * 1e9),
            "alg_bytes_per_point_with_compensation": alg_comp,
            "alg_frac_of_peak_with_compensation": value * alg_comp / (peak * 1e9),
            "peak_kind": peak_kind_note(kind), "l2": "flushed between timed steps", "autotune": tune}


def _adjoint_leg(steps):
    """Misfit gradient on the heterogeneous 3-D elastic geometry (193^3 points, 4 x 4 x 4 patches, n_nb = 20,
    FP32 + Kahan) at the homogeneous start model: forward with checkpoints, segment recomputation and the adjoint,
    timed around the library call (includes its host work: residual, chain rule)."""
    import paper_2301_05127_gb300 as pkg
    from synth import elastic3d_heterogeneous

    w = elastic3d_heterogeneous(steps=steps, true_model=False)
    g = pkg.Grid.from_workloads([w])
    obs = np.zeros((steps, len(w.receivers["v3"])))
    g.gradient(0, obs, 4)  # warm-up (allocations)
    g.sync()
    t0 = time.perf_counter()
    J, _ = g.gradient(0, obs, steps)
    wall = time.perf_counter() - t0
    g.close()
    return {"workload": f"elastic3d_heterogeneous start model 193^3 pts, 4x4x4 patches, {steps} steps, FP32 + Kahan, "
                        f"checkpoints every {int(math.ceil(math.sqrt(steps)))} steps",
            "ms_per_step": 1e3 * wall / steps, "value": w.points * steps / wall, "unit": UNIT + " (forward+adjoint)",
            "misfit": J}


def _accuracy_leg(pkg):
    """The benchmark workload over its whole length (2000 steps) in the headline precision (FP32 + compensation,
    the timed kernels) and in FP64, compared with the FP64 oracle's golden run of the same workload
    (tests/golden/full_acoustic2d_layered.npz, written by tests/golden/make_full_runs.py from the oracle):
    pressure traces after every step on lines through the source, and every field at four checkpoints on a
    sub-grid of stride 16.  Errors: max |gpu - ref| / max |ref| (traces) and ||gpu - ref||_2 over the largest
    ||ref||_2 of the run (fields)."""
    import importlib.util

    path = os.path.join(ROOT, "tests", "golden", "make_full_runs.py")
    spec = importlib.util.spec_from_file_location("make_full_runs", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    name = "acoustic2d_layered"
    if not os.path.exists(mod.path_of(name)):
        return {"unavailable": f"golden run {os.path.relpath(mod.path_of(name), ROOT)} missing"}
    gold = dict(np.load(mod.path_of(name)))
    w, stride = mod.golden_workload(name)
    sl = tuple(slice(None, None, stride) for _ in range(w.dim))
    res = {"reference": "FP64 oracle, golden run tests/golden/full_acoustic2d_layered.npz", "steps": w.steps}
    for prec in ("fp32_kahan", "fp64"):
        g = pkg.Grid.from_workloads([w], precision=prec)
        done, worst, peak = 0, {}, {}
        for i, c in enumerate(gold["ckpt_steps"]):
            g.step(int(c) - done)
            done = int(c)
            for f in ("sigma", "v1", "v3"):
                ref = gold[f"snap_{f}"][i]
                got = g.get_field(0, f).astype(np.float64)[sl]
                worst[f] = max(worst.get(f, 0.0), float(np.linalg.norm(got - ref)))
                peak[f] = max(peak.get(f, 0.0), float(np.linalg.norm(ref)))
        tr = g.record(0)["sigma"].astype(np.float64)
        g.close()
        ref_tr = gold["trace_sigma"]
        res[prec] = {"trace_rel_max": float(np.abs(tr - ref_tr).max() / np.abs(ref_tr).max()),
                     "field_rel_l2_max": max(worst[f] / peak[f] for f in worst)}
    return res


def peak_kind_note(kind):
    return "of measured" if kind == "measured" else "of fallback"


def run_ours(args):
    import torch
    import paper_2301_05127_gb300 as pkg
    from synth import acoustic2d_layered

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    flush = _flusher(torch, dev)

    def barrier():
        if ws > 1:
            import torch.distributed as dist

            dist.barrier()
        torch.cuda.synchronize()

    def slowest(x):
        return max_over_ranks(x, ws, dev)

    w = acoustic2d_layered(precision="fp32_kahan")
    pts = w.points

    # --- headline: FP32 + Kahan -------------------------------------------------------------------------
    g = pkg.Grid.from_workloads([w])
    # the clock sampler starts before the warm-up steps: starting a process inside the timed region would delay
    # the first timed step's launches
    clk = Clocks(local)
    clk.start()
    time.sleep(0.5)
    # warm-up steps, each after a flush as in the timed region (the flush's kernels load on first use)
    for _ in range(args.warmup):
        flush()
        g.step(1)
    g.sync()
    g.profile(False)  # counts launches, records no per-launch events
    barrier()
    t_wall, t_start = time.perf_counter(), time.time()
    step_ms = _timed_steps(torch, g, args.steps, flush)
    barrier()
    t_wall = time.perf_counter() - t_wall
    clocks = clk.stop(window=(t_start, time.time()))
    launches = g.profile_read(-1)[1]
    # kernel durations: K more steps, flushed the same way, with a CUDA event pair around every launch on the
    # library's stream (the events cost ~2 us per launch, so they are kept out of the headline steps)
    g.profile(True)
    prof_ms = _timed_steps(torch, g, args.steps, flush)
    kern = {k: g.profile_read(k) for k in KERNELS + ("gather",)}
    g.profile(False)
    sum_ms = slowest(sum(step_ms))
    ms_per_step = sum_ms / args.steps
    value = job_value(ws, pts, ms_per_step)

    # dominant kernel roofline: the step's algorithmic bytes (28 B per point) over one launch of the dominant
    # kernel, which processes every point of the grid once per step
    dom = max(KERNELS, key=lambda k: kern[k][0])
    dom_ms = kern[dom][0] / max(kern[dom][1], 1)
    alg = STEP_ALG_BYTES * pts
    peak, peak_kind = _peaks()
    achieved = alg / (dom_ms * 1e-3) / 1e9
    traffic = _traffic(dom)
    own = _alg_bytes_per_point(dom, 4, True, False) * pts  # every array the kernel itself reads or writes, once

    # --- FP64 form ---------------------------------------------------------------------------------------
    g64 = pkg.Grid.from_workloads([w], precision="fp64")
    g64.step(args.warmup)
    g64.sync()
    n64 = max(1, min(args.steps, max(3, args.steps // 2)))
    ms64 = _timed_steps(torch, g64, n64, flush)
    fp64_ms = slowest(sum(ms64)) / len(ms64)
    g64.close()
    g.close()

    # --- accuracy over the whole run against the FP64 oracle's golden run -------------------------------------
    accuracy = _accuracy_leg(pkg) if not args.no_accuracy else None

    # --- batched multi-shot survey, 3-D elastic step, misfit gradient ---------------------------------------
    batched = _batched_leg(torch, pkg, units=3, warmup_units=1, k=10) if not args.no_batched else None
    elastic = _elastic_leg(torch, pkg, steps=5, warmup=3, flush=flush) if not args.no_batched else None
    adjoint = _adjoint_leg(steps=60) if not args.no_batched else None

    # --- end to end through the public API with host buffers ---------------------------------------------
    # three runs on fresh handles (the timed region holds host round trips: the median is reported)
    shape = w.shape
    host_in = [torch.zeros(shape, dtype=torch.float32).pin_memory() for _ in range(3)]
    host_in[0].copy_(torch.from_numpy(np.zeros(shape, np.float32)))
    host_out = torch.empty(shape, dtype=torch.float32).pin_memory()
    e2e_runs = []
    for _ in range(3):
        ge = pkg.Grid.from_workloads([w])
        ge.step(1)  # kernels loaded and tables built; the staggered start is paid in the timed region anyway
        ge.sync()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for f, hb in zip(("sigma", "v1", "v3"), host_in):
            ge.set_field(0, f, hb)
        ge.step(args.steps)
        tr = ge.record(0)["_all"]
        ge.get_field(0, "sigma", out=host_out)
        e1.record()
        e1.synchronize()
        e2e_runs.append(slowest(e0.elapsed_time(e1)))
        ge.close()
    e2e_ms = sorted(e2e_runs)[1]
    h2d = 3 * pts * 4
    d2h = pts * 4 + tr.nbytes

    out = None
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "points": pts, "precision": "fp32 + Kahan compensation, PMBC sums fp64",
                       "l2": "flushed between timed steps (512 MiB write + read)", "parallelism": f"replicas x{ws}"},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
                         "alg_bytes_per_point": STEP_ALG_BYTES, "alg_bytes_per_launch": alg, "avg_launch_ms": dom_ms,
                         "traffic_over_alg": None if traffic is None else traffic / alg,
                         "kernel_own_bytes_per_launch": own, "kernel_own_frac": own / (dom_ms * 1e-3) / 1e9 / peak,
                         "step_frac": STEP_ALG_BYTES * pts / (ms_per_step * 1e-3) / 1e9 / peak,
                         "step_frac_with_compensation": (STEP_ALG_BYTES + STEP_COMP_BYTES) * pts
                         / (ms_per_step * 1e-3) / 1e9 / peak,
                         "durations": "CUDA events around each launch in a second pass of K flushed steps"},
            "ms_per_step_with_launch_events": sum(prof_ms) / len(prof_ms),
            "step_ms_min_median_max": [min(step_ms), statistics.median(step_ms), max(step_ms)],
            "kernels_ms_per_launch": {k: (v[0] / max(v[1], 1)) for k, v in kern.items()},
            "kernels_frac_of_peak": {k: _alg_bytes_per_point(k, 4, True, False) * pts / (kern[k][0] / kern[k][1] * 1e-3)
                                     / (peak * 1e9) for k in KERNELS if kern[k][1]},
            "fp64": {"value": job_value(ws, pts, fp64_ms), "ms_per_step": fp64_ms, "unit": UNIT},
            "accuracy": accuracy,
            "e2e": {"value": ws * pts * args.steps / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d / args.steps,
                    "d2h_bytes_per_step": d2h / args.steps, "ms_total": e2e_ms, "runs_ms": e2e_runs},
            "batched": batched,
            "elastic": elastic,
            "adjoint": adjoint,
            "gpu_launches": launches,
            "clocks": clocks,
            "wall_s_timed_region": t_wall,
        }
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return out


def _oracle_steps(steps, warmup):
    """Time the FP64 oracle on the benchmark workload: each step a full Strang step of the full grid.  The oracle
    runs as it stands, with the derivative terms of each sub-step spread over one worker process per host core
    but one (oracle.parallel, equal to the serial oracle bit for bit).  Returns (pt-upd/s, cores used, wall s,
    workers): cores = CPU seconds of the parent and the workers over the timed steps / their wall time."""
    from oracle.parallel import ParallelSimulation
    from synth import acoustic2d_layered

    w = acoustic2d_layered(precision="fp64")
    workers = max(1, (os.cpu_count() or 2) - 1)
    with ParallelSimulation(w, workers=workers) as sim:
        sim.step(max(1, warmup), record=False)
        c0, t0 = sim.cpu_time(), time.perf_counter()
        sim.step(steps, record=False)
        wall = time.perf_counter() - t0
        cpu = sim.cpu_time() - c0
    return w.points * steps / wall, max(1, round(cpu / wall)), wall, workers


def cpu_baseline():
    v, cores, wall, workers = _oracle_steps(steps=20, warmup=1)
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"20 full Strang steps of the 2049^2 FP64 oracle ({wall:.1f} s), derivative terms spread over "
                      f"{workers} worker processes; host {os.cpu_count()} cores"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return None
    v, cores, wall, workers = _oracle_steps(args.steps, args.warmup)
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "points": 2049 * 2049, "precision": "fp64 oracle"},
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": v,
                             "sample": f"{args.steps} full Strang steps of the 2049^2 FP64 oracle, derivative terms "
                                       f"spread over {workers} worker processes"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched, elastic and gradient legs")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the full-run comparison with the golden run")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        out = run_reference(args)
    else:
        out = run_ours(args)
        if out is not None:
            ws = _dist()[0]
            out["cpu_baseline"] = None if (args.no_cpu_baseline or ws > 1) else cpu_baseline()
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
