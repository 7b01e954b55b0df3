"""GPU parity of the 2-D acoustic LOSS step (PMBC closure, local solves, derivatives, velocity-stress update,
Strang integrator with the ADE-PML layer, source and receivers) against the FP64 oracle, through the C ABI.

Run error (the paper's normalisation by the reference maximum, Sec. 4): at checkpoints along the run,
||u_gpu - u_ref||_2 divided by the largest ||u_ref||_2 seen over the run, maximised over checkpoints and
fields; traces: max |trace_gpu - trace_ref| / max |sigma_ref| over the run."""
import dataclasses

import numpy as np
import pytest

from oracle.wave import Simulation
from synth import acoustic2d_small, acoustic2d_layered, scaled

pytestmark = pytest.mark.gpu

# Relative L2 tolerances of the path: FP64 to the oracle's rounding, FP32 forms over the run.
TOL = {"fp64": 1e-12, "fp32": 1e-5, "fp32_kahan": 1e-5}


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as ge

    ge.build()
    import paper_2301_05127_gb300 as p

    return p


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300)


def _compare(pkg, w, prec, steps, every=50, family=None):
    g = pkg.Grid.from_workloads([w], precision=prec)
    if family:
        g.set_kernels(family.split("/")[0])
        if family.endswith("/z8"):  # convolution z tiles with 8 positions per warp row
            g.set_tile("acoustic_z", 0, 3)
            g.set_tile("acoustic_z2", 0, 3)
    sim = Simulation(w)
    fields = ("sigma", "v1", "v3")
    peak = {f: 0.0 for f in fields}
    worst = {f: 0.0 for f in fields}
    smax = 0.0
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
        smax = max(smax, np.abs(sim.state["sigma"]).max())
    errs = {f: worst[f] / max(peak[f], 1e-300) for f in fields}
    tr = g.record(0)["sigma"].astype(np.float64)
    errs["trace"] = np.abs(tr - sim.trace_array("sigma")).max() / smax
    g.close()
    return errs


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_kahan"])
def test_small_grid_full_run(pkg, prec):
    """129^2 points in 2 x 2 patches, constant model, Ricker at the centre, n_nb = 12, 300 steps (the small 2-D
    benchmark case) -- whole run, every field at checkpoints and the top-row pressure traces."""
    w = acoustic2d_small()
    errs = _compare(pkg, w, prec, w.steps)
    assert max(errs.values()) < TOL[prec], errs


@pytest.mark.parametrize("prec", ["fp64", "fp32_kahan"])
def test_layered_model_scaled(pkg, prec):
    """Layered + correlated-noise model on 513^2 points in 2 x 2 patches of M = 256 (the benchmark patch size),
    200 steps."""
    w = scaled(acoustic2d_layered(), n=512, p=2, steps=200)
    errs = _compare(pkg, w, prec, w.steps)
    assert max(errs.values()) < TOL[prec], errs


@pytest.mark.parametrize("prec", ["fp32_kahan", "fp64"])
def test_layered_model_full_size_short(pkg, prec):
    """Full 2049^2 grid in 8 x 8 patches, the launch configuration of the benchmark, 4 steps."""
    w = acoustic2d_layered(steps=4)
    errs = _compare(pkg, w, prec, 4)
    assert max(errs.values()) < TOL[prec], errs


def test_reading_velocities_midway_does_not_change_the_run(pkg):
    """Reading v (which brings the staggered velocities back to the integer time level) between steps gives the
    same result as an uninterrupted run, up to rounding."""
    w = acoustic2d_small(n=64, p=2, steps=40, n_nb=12)
    a = pkg.Grid.from_workloads([w])
    a.step(40)
    b = pkg.Grid.from_workloads([w])
    for _ in range(4):
        b.step(10)
        b.get_field(0, "v1")
    for f in ("sigma", "v1", "v3"):
        assert rel(b.get_field(0, f), a.get_field(0, f).astype(np.float64)) < 1e-12
    assert b.get_step(0) == 40
    a.close()
    b.close()


def test_state_round_trip_and_initial_fields(pkg):
    """set_field initial conditions (the paper's Gaussian pulse, no source), checkpoint after 20 steps, restore
    into a fresh handle, continue: equal to the oracle over the whole run."""
    from synth import gaussian_pulse_2d

    w, s0 = gaussian_pulse_2d(64, p=2, n_nb=16, dt=2.5e-4, steps=40)
    w = dataclasses.replace(w, pml_width=12, f0=20.0)
    g = pkg.Grid.from_workloads([w])
    g.set_field(0, "sigma", s0)
    g.step(20)
    blob = g.get_state()
    h = pkg.Grid.from_workloads([w])
    h.set_state(blob)
    h.step(20)
    sim = Simulation(w, state={"sigma": s0, "v1": 0 * s0, "v3": 0 * s0}).step(40, record=False)
    for f in ("sigma", "v1", "v3"):
        assert rel(h.get_field(0, f), sim.state[f]) < 1e-11
    assert h.get_step(0) == 40
    g.close()
    h.close()


def test_zero_steps_and_no_receivers(pkg):
    w = dataclasses.replace(acoustic2d_small(n=32, p=2, n_nb=8, pml_width=8), receivers={})
    g = pkg.Grid.from_workloads([w])
    g.step(0)
    assert np.all(g.get_field(0, "sigma") == 0)
    g.step(3)
    assert g.record(0)["_all"].shape == (0, 0)
    g.close()


def test_multiple_shots_in_one_handle(pkg):
    """Several independent grids of different sizes advanced by one loss_step call."""
    ws = [acoustic2d_small(n=32, p=2, n_nb=8, steps=15, pml_width=8),
          acoustic2d_small(n=48, p=3, n_nb=12, steps=15, pml_width=10)]
    g = pkg.Grid.from_workloads(ws)
    g.step(15)
    for s, w in enumerate(ws):
        sim = Simulation(w).step(15)
        assert rel(g.get_field(s, "sigma"), sim.state["sigma"]) < 1e-11
    g.close()


def test_velocity_receivers_inside_the_layer(pkg):
    """Velocity traces on the top row (inside the absorbing layer) at integer time levels: the staggered state is
    corrected for the non-linear exponential sub-flow, so they equal the literal Strang values."""
    w = acoustic2d_small(n=64, p=2, n_nb=12, steps=150, pml_width=12)
    top = np.arange(65, dtype=np.int64)
    w = dataclasses.replace(w, receivers={"v1": top, "v3": top, "sigma": top})
    g = pkg.Grid.from_workloads([w])
    g.step(150)  # the direct wave reaches the top row after ~90 steps
    rec = g.record(0)
    sim = Simulation(w).step(150)
    for f in ("v1", "v3", "sigma"):
        ref = sim.trace_array(f)
        assert np.abs(rec[f] - ref).max() <= 1e-11 * np.abs(ref).max(), f
    g.close()


@pytest.mark.parametrize("family", ["line", "convolution", "convolution/z8"])
@pytest.mark.parametrize("geom", [
    # (n_z, n_x, p_z, p_x, n_nb, layer): patch lengths shorter than the convolution's truncation length (16),
    # not multiples of 8 (x falls back to the line kernel), a single-warp z tile, x extents that are not multiples
    # of 32, halo widths above 16, one patch per axis
    (24, 24, 2, 2, 6, 5),
    (36, 40, 3, 5, 8, 6),
    (48, 70, 4, 5, 10, 8),
    (64, 96, 2, 3, 20, 10),
    (80, 48, 1, 1, 24, 8),
    # sources inside the absorbing layers: at a corner (z and x layers, the line's last chunk) and at the left end
    (64, 96, 2, 3, 20, 10, (3, 95)),
    (48, 64, 2, 2, 12, 12, (40, 1)),
])
def test_fp32_kernel_families_on_uneven_geometries(pkg, family, geom):
    """Both kernel families of the FP32 step against the oracle on geometries chosen to reach the edge cases of
    the convolution kernels (tiles of one warp, ragged column groups, patch ends within the truncation length,
    line ends reached by the recursions' warm-up from both sides)."""
    nz, nx, pz, px, n_nb, layer = geom[:6]
    src = geom[6] if len(geom) > 6 else (nz // 2, nx // 3)
    w = acoustic2d_small(n=max(nz, nx), p=2, n_nb=n_nb, steps=60, pml_width=layer)
    shape = (nz + 1, nx + 1)

    def model():
        z = np.arange(nz + 1)[:, None] * np.ones((1, nx + 1))
        return np.where(z < nz / 2, 2000.0, 2600.0), None, np.full(shape, 1000.0)

    top = np.arange(nx + 1, dtype=np.int64)
    w = dataclasses.replace(w, n=(nz, nx), p=(pz, px), model_fn=model, src_index=src,
                            receivers={"sigma": top}, f0=60.0, t0=1.2 / 60.0, dt=0.4 * 10.0 / 2600.0)
    errs = _compare(pkg, w, "fp32_kahan", 60, every=20, family=family)
    assert max(errs.values()) < TOL["fp32_kahan"], errs


@pytest.mark.parametrize("prec", ["fp64", "fp32_kahan"])
def test_pinned_host_buffers(pkg, prec):
    """Fields set from and read into pinned host tensors (the pitch kernels read and write the mapped host memory
    directly) equal the copies through pageable numpy arrays, on a grid whose 101-point rows are padded in HBM."""
    import torch

    w = acoustic2d_small(n=100, p=4, steps=10, n_nb=10, pml_width=10)
    g = pkg.Grid.from_workloads([w], precision=prec)
    dt = g.dtype
    tdt = torch.float64 if dt == np.float64 else torch.float32
    rng = np.random.default_rng(11)
    a = rng.standard_normal(w.shape).astype(dt)
    g.set_field(0, "sigma", torch.from_numpy(a.copy()).pin_memory())
    assert np.array_equal(g.get_field(0, "sigma"), a)
    out = torch.empty(w.shape, dtype=tdt).pin_memory()
    g.get_field(0, "sigma", out=out)
    assert np.array_equal(out.numpy(), a)
    g.step(5)
    for f in ("sigma", "v1", "v3"):
        ref = g.get_field(0, f)
        out = torch.full(w.shape, float("nan"), dtype=tdt).pin_memory()
        g.get_field(0, f, out=out)
        assert np.array_equal(out.numpy(), ref), f
    g.close()
