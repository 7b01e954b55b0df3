"""Full-length parity of every benchmark workload against the FP64 oracle's golden runs
(tests/golden/full_<name>.npz, written by tests/golden/make_full_runs.py, which calls only the oracle).

Each workload runs over its whole length on the GPU, in the launch configuration the benchmark uses, and is
compared with the oracle element by element:

* receiver traces after every step: max |gpu - ref| over the run / max |ref| over the run, per field, at the
  receivers outside the absorbing layers, and over every receiver;
* every field at four checkpoints, sampled on a regular sub-grid, on the physical domain (the points outside
  the absorbing layers): ||gpu - ref||_2 / (largest ||ref||_2 over the checkpoints), per field (the run error of
  the paper's normalisation by the reference maximum, Sec. 4), and element by element, max |gpu - ref| /
  max |ref| over the run, so that a defect confined to a few points (one tile's edge, one patch) cannot hide in
  the norm;
* the same L2 error over the whole sampled grid, absorbing layers included;
* the full-field L2 norms at the checkpoints, relative to the largest norm of the run.

Tolerances: 1e-12 for the FP64 path, 1e-5 for the FP32 forms (FP32 fields, FP32 with compensated updates); the
element-wise field bound is ten times those (a maximum over many points of a rounding-level difference).  The
whole-grid error and the traces of every receiver, the ones inside the absorbing layers included, are held to ten
times the tolerance: on the outermost row of an absorbing layer the damping
profile's alpha vanishes, every static field profile there is an equilibrium of the layer's equations, and
rounding differences accumulate undamped (two FP64 implementations that differ only in the rounding order of
the layer update differ there by about a thousand times their difference elsewhere)."""
import dataclasses
import importlib.util
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
TOL = {"fp64": 1e-12, "fp32": 1e-5, "fp32_kahan": 1e-5}
POINT = 10.0  # element-wise field errors: POINT * TOL
LAYERS = 10.0  # whole-grid field errors, absorbing layers included: LAYERS * TOL


def _golden_module():
    spec = importlib.util.spec_from_file_location("make_full_runs", os.path.join(HERE, "golden", "make_full_runs.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


G = _golden_module()


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as ge

    ge.build()
    import paper_2301_05127_gb300 as p

    return p


def _load(name):
    path = G.path_of(name)
    assert os.path.exists(path), f"golden run {path} is missing: python tests/golden/make_full_runs.py {name}"
    return dict(np.load(path))


def _inner(shape, stride, width):
    """Slices of the sampled grid (stride `stride`) that keep the points outside absorbing layers `width` wide."""
    return tuple(slice(-(-width // stride), (n - 1 - width) // stride + 1) for n in shape)


def _outside_layers(idx, shape, width):
    """Which of the flat indices idx of a grid of `shape` points lie outside absorbing layers `width` wide."""
    coords = np.unravel_index(np.asarray(idx, dtype=np.int64), shape)
    ok = np.ones(len(idx), dtype=bool)
    for c, n in zip(coords, shape):
        ok &= (c >= width) & (c <= n - 1 - width)
    return ok


def _errors(gold, fields, snaps, norms, traces, inner, shape, width):
    """Relative errors per field of the GPU run against the golden run; `inner` selects the physical domain of
    the sampled grid, `shape` and `width` place the receivers."""
    errs = {}
    for f in fields:
        ref = gold[f"snap_{f}"]
        peak = max(float(np.linalg.norm(r[inner])) for r in ref)
        if peak > 0:
            errs[f"snap_{f}"] = max(float(np.linalg.norm((a - r)[inner])) for a, r in zip(snaps[f], ref)) / peak
            amax = max(float(np.abs(r[inner]).max()) for r in ref)
            errs[f"point_{f}"] = max(float(np.abs((a - r)[inner]).max()) for a, r in zip(snaps[f], ref)) / amax / POINT
            whole = max(float(np.linalg.norm(r)) for r in ref)
            errs[f"layers_{f}"] = max(float(np.linalg.norm(a - r)) for a, r in zip(snaps[f], ref)) / whole / LAYERS
        nref = gold[f"norm_{f}"]
        if nref.max() > 0:
            errs[f"norm_{f}"] = float(np.abs(np.asarray(norms[f]) - nref).max() / nref.max())
    for f, tr in traces.items():
        ref = gold[f"trace_{f}"]
        peak = np.abs(ref).max()
        ok = _outside_layers(gold[f"rcv_{f}"], shape, width)
        errs[f"trace_{f}"] = float(np.abs(tr - ref)[:, ok].max() / peak)
        errs[f"tlayers_{f}"] = float(np.abs(tr - ref).max() / peak) / LAYERS
    return errs


def _run_grid(g, shots, gold_by_shot, stride_by_shot, steps, fields):
    """Advance g to each checkpoint and collect sampled snapshots and full norms of the given shots."""
    ck = list(gold_by_shot[shots[0]]["ckpt_steps"])
    snaps = {s: {f: [] for f in fields} for s in shots}
    norms = {s: {f: [] for f in fields} for s in shots}
    done = 0
    for c in ck:
        g.step(int(c) - done)
        done = int(c)
        for s in shots:
            sl = tuple(slice(None, None, int(stride_by_shot[s])) for _ in range(len(g.shape(s))))
            for f in fields:
                v = g.get_field(s, f).astype(np.float64)
                snaps[s][f].append(v[sl])
                norms[s][f].append(float(np.linalg.norm(v)))
    assert done == steps
    return snaps, norms


def _single(pkg, name, prec, fields, family=None):
    gold = _load(name)
    w, stride = G.golden_workload(name)
    g = pkg.Grid.from_workloads([w], precision=prec)
    if family:
        g.set_kernels(family)
    snaps, norms = _run_grid(g, [0], {0: gold}, {0: stride}, w.steps, fields)
    rec = g.record(0)
    traces = {f: rec[f].astype(np.float64) for f in w.receivers}
    g.close()
    errs = _errors(gold, fields, snaps[0], norms[0], traces, _inner(g.shape(0), stride, w.pml_width), g.shape(0),
                   w.pml_width)
    _report(f"{name} {prec}{'/' + family if family else ''}", errs)
    return errs


def _report(label, errs):
    worst = lambda key: max((v for k, v in errs.items() if k.startswith(key)), default=0.0)  # noqa: E731
    print(f"[full run] {label}: fields {worst('snap'):.2e}, points {POINT * worst('point'):.2e}, "
          f"whole grid {LAYERS * worst('layers'):.2e}, norms {worst('norm'):.2e}, traces {worst('trace'):.2e}, "
          f"all receivers {LAYERS * worst('tlayers'):.2e}")


ACOUSTIC = ("sigma", "v1", "v3")
ELASTIC = ("v1", "v2", "v3", "s11", "s22", "s33", "s12", "s13", "s23")


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_kahan"])
def test_small_2d_full_run(pkg, prec):
    """129^2 points, 2 x 2 patches, n_nb = 12, 300 steps."""
    errs = _single(pkg, "acoustic2d_small", prec, ACOUSTIC)
    assert max(errs.values()) < TOL[prec], errs


@pytest.mark.parametrize("prec", ["fp64", "fp32_kahan"])
def test_layered_2049_full_run(pkg, prec):
    """2049^2 points, 8 x 8 patches (M = 256), n_nb = 20, layered model with correlated noise, 2000 steps: the
    benchmark workload over its whole length, FP32 + compensation on the convolution kernels the benchmark times."""
    errs = _single(pkg, "acoustic2d_layered", prec, ACOUSTIC)
    assert max(errs.values()) < TOL[prec], errs


def test_layered_2049_full_run_line_kernels(pkg):
    """The same run on the line-kernel family (FP32 + compensation)."""
    errs = _single(pkg, "acoustic2d_layered", "fp32_kahan", ACOUSTIC, family="line")
    assert max(errs.values()) < TOL["fp32_kahan"], errs


def test_layered_2049_full_run_item_kernels(pkg):
    """The same run with the x part on (row, patch) items, the form rows too long for the pipelined x kernel take
    (FP32 + compensation)."""
    errs = _single(pkg, "acoustic2d_layered", "fp32_kahan", ACOUSTIC, family="convolution_items")
    assert max(errs.values()) < TOL["fp32_kahan"], errs


@pytest.mark.parametrize("prec", ["fp64", "fp32_kahan"])
def test_elastic_257_full_run(pkg, prec):
    """257^3 points, 4 x 4 x 4 patches, homogeneous, explosive + shear source, 1000 steps; v1, v2, v3 on the top
    plane of the physical domain (z = 20) and all nine fields at the checkpoints."""
    errs = _single(pkg, "elastic3d_homogeneous", prec, ELASTIC)
    assert max(errs.values()) < TOL[prec], errs


@pytest.mark.parametrize("prec", ["fp64", "fp32_kahan"])
def test_elastic_heterogeneous_193_full_run(pkg, prec):
    """193^3 points, 4 x 4 x 4 patches, smooth random vp / vs / rho, 1500 steps: the forward run of the
    gradient workload; v3 on the top plane of the physical domain (z = 20) and all nine fields at the checkpoints."""
    errs = _single(pkg, "elastic3d_heterogeneous", prec, ELASTIC)
    assert max(errs.values()) < TOL[prec], errs


def _survey_names():
    return [n for n in G.golden_names() if n.startswith("survey_shot")]


@pytest.mark.parametrize("prec,graph", [("fp32", 25), ("fp64", 0)])
def test_survey_full_run(pkg, prec, graph):
    """The 64-shot survey, 1500 steps.  FP32: all 64 shots in one batched schedule replayed from a captured CUDA
    graph (the benchmark's launch configuration), compared on the smallest, the largest and two shots between.
    FP64: those four shots in one batched handle."""
    from synth import batched_shots

    names = _survey_names()
    picks = [int(n[len("survey_shot"):]) for n in names]
    gold = {s: _load(n) for s, n in zip(picks, names)}
    stride = {s: int(gold[s]["stride"]) for s in picks}
    ws = batched_shots()
    golden_ws = {s: G.golden_workload(n)[0] for s, n in zip(picks, names)}
    if prec == "fp32":
        shots = [golden_ws.get(s, dataclasses.replace(w, receivers={})) for s, w in enumerate(ws)]
        idx = {s: s for s in picks}
    else:
        shots = [golden_ws[s] for s in picks]
        idx = {s: i for i, s in enumerate(picks)}
    g = pkg.Grid.from_workloads(shots, precision=prec)
    g.set_schedule(True, graph)
    steps = ws[0].steps
    snaps, norms = _run_grid(g, [idx[s] for s in picks], {idx[s]: gold[s] for s in picks},
                             {idx[s]: stride[s] for s in picks}, steps, ACOUSTIC)
    worst = {}
    for s in picks:
        rec = g.record(idx[s])
        errs = _errors(gold[s], ACOUSTIC, snaps[idx[s]], norms[idx[s]], {"sigma": rec["sigma"].astype(np.float64)},
                       _inner(g.shape(idx[s]), stride[s], ws[s].pml_width), g.shape(idx[s]), ws[s].pml_width)
        _report(f"survey shot {s} ({ws[s].n[0]}^2) {prec}", errs)
        worst[s] = max(errs.values())
        assert worst[s] < TOL[prec], (s, errs)
    g.close()
