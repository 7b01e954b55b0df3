"""GPU parity of the 3-D elastic LOSS step (nine velocity-stress fields, PMBC closures and local solves on all
three axes, Strang splitting with the ADE-PML layer, explosive/shear/force sources, receivers) against the FP64
oracle, through the C ABI.  Run error as in test_gpu_acoustic: ||u_gpu - u_ref|| / max over the run of
||u_ref||, at checkpoints, for every field."""
import dataclasses

import numpy as np
import pytest

from oracle.wave import ELASTIC_FIELDS, Simulation
from synth import elastic3d_heterogeneous, elastic3d_homogeneous, scaled

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-11, "fp32": 1e-5, "fp32_kahan": 1e-5}


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as ge

    ge.build()
    import paper_2301_05127_gb300 as p

    return p


def _compare(pkg, w, prec, steps, every=20, fields=ELASTIC_FIELDS, traces=True, family=None):
    g = pkg.Grid.from_workloads([w], precision=prec)
    if family:
        g.set_kernels(family)
    sim = Simulation(w)
    peak = {f: 0.0 for f in fields}
    worst = {f: 0.0 for f in fields}
    vmax = 0.0
    done = 0
    while done < steps:
        k = min(every, steps - done)
        g.step(k)
        sim.step(k)
        done += k
        for f in fields:
            ref = sim.state[f]
            peak[f] = max(peak[f], np.linalg.norm(ref))
            worst[f] = max(worst[f], np.linalg.norm(g.get_field(0, f).astype(np.float64) - ref))
        vmax = max(vmax, max(np.abs(sim.state[f]).max() for f in ("v1", "v2", "v3")))
    errs = {f: worst[f] / max(peak[f], 1e-300) for f in fields}
    if traces and w.receivers:
        rec = g.record(0)
        for f in w.receivers:
            errs["trace_" + f] = np.abs(rec[f].astype(np.float64) - sim.trace_array(f)).max() / max(vmax, 1e-300)
    g.close()
    return errs


@pytest.mark.parametrize("prec,family", [("fp64", None), ("fp32", "convolution"), ("fp32", "line"),
                                         ("fp32_kahan", "convolution"), ("fp32_kahan", "line")])
def test_homogeneous_small(pkg, prec, family):
    """33^3 points in 2 x 2 x 2 patches, explosive + shear source, 6-point layer, 60 steps; FP32 on both kernel
    families (y / z passes on one-patch tiles in the truncated-convolution form, or on whole lines)."""
    w = elastic3d_homogeneous(n=32, p=2, n_nb=8, steps=60, pml_width=6, precision=prec)
    w = dataclasses.replace(w, f0=40.0, t0=1.2 / 40.0)
    errs = _compare(pkg, w, prec, w.steps, family=family)
    assert max(errs.values()) < TOL[prec], errs


@pytest.mark.parametrize("prec,family", [("fp64", None), ("fp32_kahan", "convolution"), ("fp32_kahan", "line")])
def test_heterogeneous_model(pkg, prec, family):
    """Smooth random vp / vs / rho (arrays for lambda, mu and b), 4 x 4 x 4 patches of M = 12, 40 steps."""
    w = scaled(elastic3d_heterogeneous(), n=48, p=4, steps=40, n_nb=12, pml_width=8)
    w = dataclasses.replace(w, f0=40.0, t0=1.2 / 40.0)
    errs = _compare(pkg, w, prec, w.steps, family=family)
    assert max(errs.values()) < TOL[prec], errs


def test_anisotropic_grid_force_source(pkg):
    """Different n and p on every axis and a vertical body force (FORCE_Z), FP64."""
    w = elastic3d_homogeneous(n=32, p=2, n_nb=8, steps=30, pml_width=6, precision="fp64")
    shape = (25, 33, 41)

    def model():
        return np.full(shape, 3000.0), np.full(shape, 1730.0), np.full(shape, 2000.0)

    w = dataclasses.replace(w, n=(24, 32, 40), p=(2, 2, 4), model_fn=model, src_index=(12, 16, 20),
                            src_kinds=("force_z", "explosive"), f0=40.0, t0=1.2 / 40.0,
                            receivers={"v3": np.arange(33 * 41, dtype=np.int64)})
    errs = _compare(pkg, w, "fp64", w.steps)
    assert max(errs.values()) < TOL["fp64"], errs


@pytest.mark.parametrize("prec", ["fp32", "fp32_kahan"])
def test_anisotropic_grid_three_forces_tiles(pkg, prec):
    """Uneven n and p per axis (patches of 12, 16 and 10 points, shorter than the 20-point tile halo), the body
    force along x, y and z plus the explosive source, 30 steps, on the FP32 tile passes."""
    w = elastic3d_homogeneous(n=32, p=2, n_nb=8, steps=30, pml_width=4, precision=prec)
    shape = (25, 33, 41)

    def model():
        return np.full(shape, 3000.0), np.full(shape, 1730.0), np.full(shape, 2000.0)

    w = dataclasses.replace(w, n=(24, 32, 40), p=(2, 2, 4), model_fn=model, src_index=(12, 16, 20),
                            src_kinds=("force_x", "force_y", "force_z", "explosive"), f0=40.0, t0=1.2 / 40.0,
                            receivers={"v1": np.arange(33 * 41, dtype=np.int64)})
    errs = _compare(pkg, w, prec, w.steps, family="convolution")
    assert max(errs.values()) < TOL[prec], errs


@pytest.mark.parametrize("prec,family", [("fp64", None), ("fp32_kahan", "convolution"), ("fp32_kahan", "line")])
def test_one_patch_per_axis(pkg, prec, family):
    """25^3 points in one patch per axis (only the one-sided end closures, no interior junction), explosive +
    shear source, 5-point layer, 40 steps."""
    w = elastic3d_homogeneous(n=24, p=1, n_nb=8, steps=40, pml_width=5, precision=prec)
    w = dataclasses.replace(w, f0=40.0, t0=1.2 / 40.0)
    errs = _compare(pkg, w, prec, w.steps, family=family)
    assert max(errs.values()) < TOL[prec], errs


def test_full_size_homogeneous_one_step(pkg):
    """257^3 points in 4 x 4 x 4 patches (the homogeneous 3-D benchmark geometry), FP32 + Kahan, after the
    staggered start and one step, every field element-wise against the oracle."""
    w = elastic3d_homogeneous(steps=2)
    errs = _compare(pkg, w, "fp32_kahan", 2, every=2, traces=False)
    assert max(errs.values()) < TOL["fp32_kahan"], errs
