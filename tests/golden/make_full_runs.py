"""Writes the full-length FP64 oracle runs of the benchmark workloads to tests/golden/full_<name>.npz.

Calls only ``oracle`` (through ``oracle.parallel.ParallelSimulation``, which equals the serial oracle bit for
bit) and the seeded input generators in ``synth``; nothing here comes from the CUDA path.  Each file holds,
for one workload run over its whole length:

* ``rcv_<field>``: flat receiver indices, and ``trace_<field>``: the oracle's values there after every step
  (shape [steps, receivers]);
* ``ckpt_steps``: the checkpoint steps (a quarter, half, three quarters and all of the run);
* ``snap_<field>``: every field at the checkpoints, sampled with stride ``stride`` along every axis (shape
  [checkpoints, *sampled shape]);
* ``norm_<field>``: the full-field L2 norm of every field at the checkpoints.

The receivers sit where the wavefield is: lines through the source (2-D; for the survey shots the receiver row and
the source column) or lines on the receiver plane (3-D: the top of the physical domain, z = pml_width), 33 points
each; the workloads' own receiver sets are whole planes or rows and too large to store for every step.

Usage: python tests/golden/make_full_runs.py [name ...]     (default: every name of golden_names(); the 3-D runs
take hours of CPU time on 8 cores)
"""
from __future__ import annotations

import dataclasses
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from synth import workloads as W  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def _line_points(n: int, count: int = 33) -> np.ndarray:
    return np.unique(np.linspace(0, n, count).round().astype(np.int64))


def _rcv_2d_through_source(w) -> np.ndarray:
    """33 points along x on the source row and 33 along z on the source column."""
    nz, nx = w.n
    zs, xs = w.src_index
    row = zs * (nx + 1) + _line_points(nx)
    col = _line_points(nz) * (nx + 1) + xs
    return np.unique(np.concatenate([row, col])).astype(np.int64)


def _rcv_plane_lines(w, z: int = 0) -> np.ndarray:
    """33 points along x and 33 along y on the plane of axis-0 index z, through the source's (y, x)."""
    _, ny, nx = w.n
    _, ys, xs = w.src_index
    a = ys * (nx + 1) + _line_points(nx)
    b = _line_points(ny) * (nx + 1) + xs
    return (z * (ny + 1) * (nx + 1) + np.unique(np.concatenate([a, b]))).astype(np.int64)


def survey_shot_indices(shots) -> tuple:
    """The smallest and the largest shot of the survey and the two whose sizes lie nearest one and two thirds
    of the way between them."""
    sizes = np.array([s.n[0] for s in shots])
    lo, hi = int(np.argmin(sizes)), int(np.argmax(sizes))
    picks = [lo]
    for frac in (1.0 / 3.0, 2.0 / 3.0):
        target = sizes[lo] + frac * (sizes[hi] - sizes[lo])
        order = np.argsort(np.abs(sizes - target), kind="stable")
        picks.append(int(next(i for i in order if int(i) not in picks and int(i) != hi)))
    picks.append(hi)
    return tuple(picks)


def golden_workload(name: str):
    """(workload, stride) of a golden run, with its stored receivers."""
    if name == "acoustic2d_small":
        w = W.acoustic2d_small()
        return dataclasses.replace(w, receivers={"sigma": _rcv_2d_through_source(w)}), 8
    if name == "acoustic2d_layered":
        w = W.acoustic2d_layered(precision="fp64")
        return dataclasses.replace(w, receivers={"sigma": _rcv_2d_through_source(w)}), 16
    if name == "elastic3d_homogeneous":
        w = W.elastic3d_homogeneous(precision="fp64")
        r = _rcv_plane_lines(w, w.pml_width)
        return dataclasses.replace(w, receivers={"v1": r, "v2": r, "v3": r}), 16
    if name == "elastic3d_heterogeneous":
        w = W.elastic3d_heterogeneous(precision="fp64")
        return dataclasses.replace(w, receivers={"v3": _rcv_plane_lines(w, w.pml_width)}), 12
    if name.startswith("survey_shot"):
        s = int(name[len("survey_shot"):])
        w = W.batched_shots()[s]
        nz, nx = w.n
        row = w.pml_width * (nx + 1) + _line_points(nx)  # the receiver row, the top of the physical domain
        col = _line_points(nz) * (nx + 1) + w.src_index[1]
        return dataclasses.replace(w, receivers={"sigma": np.unique(np.concatenate([row, col]))}), 32
    raise KeyError(name)


def golden_names():
    return (["acoustic2d_small", "acoustic2d_layered", "elastic3d_homogeneous", "elastic3d_heterogeneous"]
            + [f"survey_shot{s}" for s in survey_shot_indices(W.batched_shots())])


def checkpoints(steps: int):
    return sorted({max(1, steps // 4), max(1, steps // 2), max(1, (3 * steps) // 4), steps})


def path_of(name: str) -> str:
    return os.path.join(HERE, f"full_{name}.npz")


def run(name: str, workers: int):
    from oracle.parallel import ParallelSimulation

    w, stride = golden_workload(name)
    ck = checkpoints(w.steps)
    sl = tuple(slice(None, None, stride) for _ in range(w.dim))
    snaps, norms = {}, {}
    t0 = time.time()
    with ParallelSimulation(w, workers=workers) as sim:
        done = 0
        for c in ck:
            sim.step(c - done)
            done = c
            for f, v in sim.state.items():
                snaps.setdefault(f, []).append(np.array(v[sl]))
                norms.setdefault(f, []).append(float(np.linalg.norm(v)))
            print(f"{name}: step {done}/{w.steps}, {time.time() - t0:.0f} s", flush=True)
        out = {"ckpt_steps": np.asarray(ck, np.int64), "stride": np.int64(stride)}
        for f, idx in w.receivers.items():
            out[f"rcv_{f}"] = np.asarray(idx, np.int64)
            out[f"trace_{f}"] = sim.trace_array(f)
    for f in snaps:
        out[f"snap_{f}"] = np.stack(snaps[f])
        out[f"norm_{f}"] = np.asarray(norms[f])
    np.savez_compressed(path_of(name), **out)
    print(f"{name}: wrote {path_of(name)} in {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    names = sys.argv[1:] or golden_names()
    workers = int(os.environ.get("ORACLE_WORKERS", max(1, (os.cpu_count() or 2) - 1)))
    for nm in names:
        run(nm, workers)
