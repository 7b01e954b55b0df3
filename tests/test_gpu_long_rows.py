"""GPU parity of the 2-D FP32 step on rows that the whole-row x kernel does not take: rows longer than 2049
points, and patches whose length is not a multiple of 8.  Their x part runs on (row, x patch) items in two
launches (sub-step B, then the x part of A), each warp staging its patch plus the junction halo.  Compared with
the FP64 oracle as in tests/test_gpu_acoustic.py: every field at checkpoints along the run, relative to the
largest reference norm, and the receiver traces."""
import dataclasses

import numpy as np
import pytest

from oracle.wave import Simulation
from synth import Workload

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp32_kahan": 1e-5}


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as ge

    ge.build()
    import paper_2301_05127_gb300 as p

    return p


def _wide(nz, nx, pz, px, steps, pml=12, n_nb=12):
    """nz x nx intervals, two layers (2000 m/s above the middle row, 2600 below, 1000 kg/m^3), a 15 Hz Ricker
    at the centre, receivers on the top row of the physical domain."""
    shape = (nz + 1, nx + 1)
    h = 10.0

    def model():
        v = np.where(np.arange(nz + 1)[:, None] < nz // 2, 2000.0, 2600.0) * np.ones(shape)
        return v, None, np.full(shape, 1000.0)

    return Workload(name=f"wide_{nz}x{nx}", dim=2, physics="acoustic", n=(nz, nx), p=(pz, px), h=(h, h),
                    n_nb=n_nb, dt=0.4 * h / 2600.0, steps=steps, model_fn=model, src_index=(nz // 2, nx // 2),
                    src_kinds=("pressure",), f0=15.0, t0=0.08,
                    receivers={"sigma": pml * (nx + 1) + np.arange(nx + 1, dtype=np.int64)}, pml_width=pml)


_REF = {}


def _reference(w, every):
    """The oracle's fields at every checkpoint and its traces (computed once per workload)."""
    if w.name not in _REF:
        sim = Simulation(w)
        snaps = []
        done = 0
        while done < w.steps:
            k = min(every, w.steps - done)
            sim.step(k)
            done += k
            snaps.append({f: sim.state[f].copy() for f in ("sigma", "v1", "v3")})
        _REF[w.name] = (snaps, sim.trace_array("sigma"))
    return _REF[w.name]


def _compare(pkg, w, prec, every=20):
    snaps, ref_tr = _reference(w, every)
    g = pkg.Grid.from_workloads([w], precision=prec)
    fields = ("sigma", "v1", "v3")
    peak = {f: 0.0 for f in fields}
    worst = {f: 0.0 for f in fields}
    smax = 0.0
    done = 0
    for ref in snaps:
        k = min(every, w.steps - done)
        g.step(k)
        done += k
        for f in fields:
            peak[f] = max(peak[f], np.linalg.norm(ref[f]))
            worst[f] = max(worst[f], np.linalg.norm(g.get_field(0, f).astype(np.float64) - ref[f]))
        smax = max(smax, np.abs(ref["sigma"]).max())
    errs = {f: worst[f] / max(peak[f], 1e-300) for f in fields}
    tr = g.record(0)["sigma"].astype(np.float64)
    errs["trace"] = np.abs(tr - ref_tr).max() / smax
    g.close()
    return errs


@pytest.mark.parametrize("prec", ["fp32", "fp32_kahan"])
def test_rows_of_4097_points(pkg, prec):
    """65 x 4097 points, 1 x 16 patches (M = 256 along x), 120 steps: the wave crosses patch junctions along x."""
    w = _wide(64, 4096, 1, 16, 120)
    errs = _compare(pkg, w, prec)
    assert max(errs.values()) < TOL[prec], errs


@pytest.mark.parametrize("prec", ["fp32", "fp32_kahan"])
def test_patches_of_ragged_length(pkg, prec):
    """97 x 301 points, 2 x 4 patches (M = 75 along x: chunks of 8 end short, the last patch owns the line's end),
    and 129 x 3301 points, 2 x 12 patches (M = 275, two rounds of chunks per lane), 100 steps."""
    for w in (_wide(96, 300, 2, 4, 100, pml=10, n_nb=10), _wide(128, 3300, 2, 12, 100)):
        errs = _compare(pkg, w, prec)
        assert max(errs.values()) < TOL[prec], (w.name, errs)


def test_layer_and_source_on_item_boundaries(pkg):
    """The absorbing layer spans whole and partial patches (M = 16 < layer width 20), and the source's 25-point
    profile crosses a patch junction: 65 x 2113 points, 1 x 132 patches, FP32 with compensation, 80 steps."""
    w = _wide(64, 2112, 1, 132, 80, pml=20, n_nb=12)
    w = dataclasses.replace(w, src_index=(32, 16 * 66 + 3))
    errs = _compare(pkg, w, "fp32_kahan")
    assert max(errs.values()) < TOL["fp32_kahan"], errs


def test_batched_schedule_with_a_long_row_shot(pkg):
    """A batch holding a shot with 4097-point rows runs it on the per-shot schedule: every shot equals its own
    single-shot run bit for bit."""
    wide = _wide(64, 4096, 1, 16, 30)
    small = _wide(64, 512, 1, 4, 30)
    g = pkg.Grid.from_workloads([wide, small], precision="fp32_kahan")
    g.set_schedule(True, 0)
    g.step(30)
    both = [{f: g.get_field(i, f) for f in ("sigma", "v1", "v3")} for i in range(2)]
    g.close()
    for i, w in enumerate((wide, small)):
        g = pkg.Grid.from_workloads([w], precision="fp32_kahan")
        g.step(30)
        for f in ("sigma", "v1", "v3"):
            assert np.array_equal(g.get_field(0, f), both[i][f]), (w.name, f)
        g.close()
