"""The double-layer experiment of the paper (Sec. 4.3) on the GPU.

* Parity: the double-layer model on a small z-refined grid (nz = 2n), with the paper's body force along all three
  axes, against the FP64 oracle: every field at checkpoints and the v3 traces on the vertical line x = y = 0.
* Order reduction at the interface: a GPU self-convergence series on grids n, 2n, 4n (nz = 2n each) started from
  an explosive Gaussian stress blob above the interface, with the same time step on every grid.  The differences
  between consecutive grids on the vertical line through the blob give the observed order
  log2(|u_n - u_2n| / |u_2n - u_4n|).  The same series on the upper layer's homogeneous model gives the scheme's
  order without the interface; the paper reports that the material discontinuity lowers it.
  An initial condition is used instead of the body force because the source's spatial profile is a fixed number
  of cells wide, so it changes with the grid and a self-convergence series would measure that change."""
import dataclasses

import numpy as np
import pytest

from oracle.wave import Simulation
from synth import DOUBLE_LAYER_UPPER, elastic3d_double_layer

pytestmark = pytest.mark.gpu

ELASTIC = ("v1", "v2", "v3", "s11", "s22", "s33", "s12", "s13", "s23")
TOL = {"fp64": 1e-12, "fp32_kahan": 1e-5}


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as ge

    ge.build()
    import paper_2301_05127_gb300 as p

    return p


def _small_case():
    """33 x 17 x 17 points (nz = 2n), 2 x 2 x 2 patches, n_nb = 8, 4-point layers, the three-axis body force with
    a 1 Hz Ricker (the grid resolves none of the paper's frequencies; this case checks the arithmetic), 300 steps
    of 5 ms."""
    w = elastic3d_double_layer(n=16, nz=32, p=2, pz=2, steps=300, n_nb=8, pml_width=4, precision="fp64")
    return dataclasses.replace(w, f0=1.0, t0=1.2)


@pytest.mark.parametrize("prec", ["fp64", "fp32_kahan"])
def test_double_layer_parity_with_three_axis_force(pkg, prec):
    w = _small_case()
    assert set(w.src_kinds) == {"force_x", "force_y", "force_z"}
    g = pkg.Grid.from_workloads([w], precision=prec)
    sim = Simulation(w)
    worst, peak, smax = {f: 0.0 for f in ELASTIC}, {f: 0.0 for f in ELASTIC}, 0.0
    for _ in range(3):
        g.step(100)
        sim.step(100)
        for f in ELASTIC:
            ref = sim.state[f]
            peak[f] = max(peak[f], float(np.linalg.norm(ref)))
            worst[f] = max(worst[f], float(np.linalg.norm(g.get_field(0, f).astype(np.float64) - ref)))
        smax = max(smax, float(np.abs(sim.state["v3"]).max()))
    errs = {f: worst[f] / peak[f] for f in ELASTIC if peak[f] > 0}
    assert all(peak[f] > 0 for f in ("v1", "v2", "v3")), peak  # the force drives every component
    tr = g.record(0)["v3"].astype(np.float64)
    errs["trace"] = float(np.abs(tr - sim.trace_array("v3")).max() / smax)
    g.close()
    assert max(errs.values()) < TOL[prec], errs


def _blob_run(pkg, n, homogeneous, steps, prec="fp64", width=5000.0):
    """v3 on the line x = y = 0 after `steps` steps of 5 ms from an explosive Gaussian stress blob of std `width`
    centred 10 km above the interface; no source.  The absorbing layers are n / 8 points wide, the same physical
    thickness on every grid of the series."""
    w = elastic3d_double_layer(n=n, nz=2 * n, p=2, pz=4, steps=steps, n_nb=16, pml_width=n // 8, precision=prec)
    w = dataclasses.replace(w, src_kinds=(), amp=0.0)
    if homogeneous:
        shape = w.shape
        w = dataclasses.replace(w, model_fn=lambda: tuple(np.full(shape, v) for v in DOUBLE_LAYER_UPPER))
    nz = 2 * n
    z = -40000.0 + (80000.0 / nz) * np.arange(nz + 1)
    x = -40000.0 + (80000.0 / n) * np.arange(n + 1)
    r2 = (z[:, None, None] - 10000.0) ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2
    s0 = 1e6 * np.exp(-r2 / (2.0 * width**2))
    g = pkg.Grid.from_workloads([w])
    for f in ("s11", "s22", "s33"):
        g.set_field(0, f, s0)
    g.step(steps)
    v3 = g.get_field(0, "v3").astype(np.float64)[:, n // 2, n // 2]
    g.close()
    return v3  # nz + 1 points along z


def _orders(pkg, homogeneous, n0=64, steps=1200):
    u = [_blob_run(pkg, n0 * k, homogeneous, steps) for k in (1, 2, 4)]
    # common points: the points of the coarsest line with -25 km <= z <= 20 km, away from the absorbing layers
    # (5 km thick at each end of z) and from anything they reflect within 6 s
    z = -40000.0 + (80000.0 / (2 * n0)) * np.arange(2 * n0 + 1)
    keep = (z >= -25000.0) & (z <= 20000.0)
    c = [u[0][keep], u[1][::2][keep], u[2][::4][keep]]
    e1 = np.linalg.norm(c[0] - c[1])
    e2 = np.linalg.norm(c[1] - c[2])
    return float(np.log2(e1 / e2)), float(e1 / np.linalg.norm(c[2])), float(e2 / np.linalg.norm(c[2]))


def test_order_reduction_at_the_interface(pkg):
    """Self-convergence on n = 64, 128, 256 (z-refined, 0.5 to 33.9 million points), 6 s of propagation: the P
    wave crosses the interface at about 3.8 s."""
    p_hom, a_hom, b_hom = _orders(pkg, True)
    p_int, a_int, b_int = _orders(pkg, False)
    print(f"homogeneous: order {p_hom:.2f} (rel. differences {a_hom:.2e}, {b_hom:.2e}); "
          f"double layer: order {p_int:.2f} ({a_int:.2e}, {b_int:.2e})")
    assert p_hom > 3.0, (p_hom, a_hom, b_hom)
    assert p_int < p_hom - 0.5, (p_int, p_hom)
    assert p_int > 0.5, (p_int, a_int, b_int)  # still converging
