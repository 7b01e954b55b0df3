"""GPU parity of the LOSS derivative on non-uniform grids (loss_set_coordinates; the paper's Sec. 3 remark and its
conclusion) against the oracle's B-spline collocation on the same knots (oracle/nonuniform.py), element by
element: first and second derivatives, their transpose and PMBC junction values, 2-D and 3-D, FP64 and FP32, several
axes and patch counts; and the 2-D acoustic step on such grids, with absorbing layers and pressure sources."""
import numpy as np
import pytest

from oracle import nonuniform as nu

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-5}


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as ge

    ge.build()
    import paper_2301_05127_gb300 as p

    return p


def _knots(n, seed, ratio=2.0, scale=10.0):
    rng = np.random.default_rng(seed)
    h = np.exp(rng.uniform(0.0, np.log(ratio), size=n)) * scale
    return np.concatenate([[0.0], np.cumsum(h)])


CASES = [
    # dim, n, p, n_nb, non-uniform axes
    (2, (64, 96), (2, 3), 12, (0, 1)),
    (2, (120, 48), (4, 2), 10, (1,)),
    (3, (24, 32, 40), (2, 2, 4), 8, (0, 1, 2)),
    (3, (48, 36, 30), (3, 2, 1), 12, (1,)),
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_nonuniform_derivative_and_phi_match_oracle(pkg, case, prec):
    dim, n, p, n_nb, axes = case
    d = pkg.make_desc(dim, pkg.LOSS_ACOUSTIC, pkg.PRECISIONS[prec], n_nb, n, p, (10.0,) * dim, 1e-3)
    g = pkg.Grid([d])
    knots = {}
    for a in axes:
        knots[a] = _knots(n[a], 100 + a)
        g.set_coordinates(0, a, knots[a])
    rng = np.random.default_rng(7)
    f = rng.standard_normal(g.shape()).astype(g.dtype)
    for a in range(dim):
        x = knots.get(a, 10.0 * np.arange(n[a] + 1))
        ref = nu.derivative(f.astype(np.float64), a, x, p[a], n_nb)
        got = g.derivative(0, a, f).astype(np.float64)
        assert np.abs(got - ref).max() <= TOL[prec] * np.abs(ref).max(), (a, prec)
        if a in knots:
            _, ref2 = nu.derivative(f.astype(np.float64), a, x, p[a], n_nb, second=True)
            got1, got2 = g.derivative(0, a, f, second=True)
            assert np.array_equal(got1, g.derivative(0, a, f)), (a, prec)
            tol2 = 1e-10 if prec == "fp64" else 5e-4
            assert np.abs(got2.astype(np.float64) - ref2).max() <= tol2 * np.abs(ref2).max(), (a, prec)
            fm = np.moveaxis(f.astype(np.float64), a, -1).reshape(-1, n[a] + 1)
            ref_phi = nu.pmbc_phi(fm, x, p[a], n_nb)
            got_phi = g.pmbc_phi(0, a, f)
            assert np.abs(got_phi - ref_phi).max() <= TOL[prec] * np.abs(ref_phi).max(), (a, prec)
    g.close()


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_nonuniform_derivative_adjoint_matches_the_oracles_transpose(pkg, case, prec):
    """loss_derivative_adjoint on axes with knots against the transpose of the oracle's derivative operator, built
    column by column from unit vectors: D^T g along every line, element by element."""
    dim, n, p, n_nb, axes = case
    d = pkg.make_desc(dim, pkg.LOSS_ACOUSTIC, pkg.PRECISIONS[prec], n_nb, n, p, (10.0,) * dim, 1e-3)
    g = pkg.Grid([d])
    knots = {a: _knots(n[a], 200 + a) for a in axes}
    for a, x in knots.items():
        g.set_coordinates(0, a, x)
    G = np.random.default_rng(9).standard_normal(g.shape()).astype(g.dtype)
    for a, x in knots.items():
        D = nu.derivative_1d(np.eye(n[a] + 1), x, p[a], n_nb).T  # D[:, c] = D e_c
        ref = np.moveaxis(np.moveaxis(G.astype(np.float64), a, -1) @ D, -1, a)
        got = g.derivative_adjoint(0, a, G).astype(np.float64)
        assert np.abs(got - ref).max() <= TOL[prec] * np.abs(ref).max(), (a, prec)
    g.close()


def test_uniform_knots_equal_the_uniform_path(pkg):
    """Knots with equal spacing through the non-uniform kernel give the uniform LOSS derivative (to rounding)."""
    n, p, n_nb, h = (40, 56), (2, 4), 10, (2.5, 4.0)
    d = pkg.make_desc(2, pkg.LOSS_ACOUSTIC, pkg.LOSS_FP64, n_nb, n, p, h, 1e-3)
    a, b = pkg.Grid([d]), pkg.Grid([d])
    for ax in range(2):
        b.set_coordinates(0, ax, h[ax] * np.arange(n[ax] + 1) + 3.0)
    f = np.random.default_rng(3).standard_normal(a.shape())
    for ax in range(2):
        ra, rb = a.derivative(0, ax, f), b.derivative(0, ax, f)
        assert np.abs(ra - rb).max() < 1e-12 * np.abs(ra).max()
    b.set_coordinates(0, 1, None)  # back to uniform spacing
    assert np.array_equal(a.derivative(0, 1, f), b.derivative(0, 1, f))
    a.close()
    b.close()


def test_nonuniform_rejections(pkg):
    d = pkg.make_desc(2, pkg.LOSS_ACOUSTIC, pkg.LOSS_FP64, 8, (32, 32), (2, 2), (1.0, 1.0), 1e-3)
    g = pkg.Grid([d])
    bad = np.arange(33, dtype=np.float64)
    bad[5] = bad[4]
    with pytest.raises(pkg.LossError) as e:
        g.set_coordinates(0, 0, bad)
    assert e.value.status == pkg.LOSS_E_ARG
    g.set_coordinates(0, 0, _knots(32, 1))
    with pytest.raises(pkg.LossError) as e:  # gradients through the step on knots are not built
        g.gradient(0, np.zeros((1, 1)), 1)
    assert e.value.status == pkg.LOSS_E_UNSUPPORTED
    g.set_model(0, np.full(g.shape(), 2000.0), None, np.full(g.shape(), 1000.0))
    g.set_source(0, [16, 0, 16], pkg.LOSS_SRC_PRESSURE, 1.0, 20.0, 0.06)
    g.step(1)  # a pressure source is taken on the knots
    assert np.abs(g.get_field(0, "sigma")).max() > 0
    g.close()


def _stretched(n, eps=0.3, half=5.0):
    xi = np.linspace(-half, half, n + 1)
    return xi + eps * (half / np.pi) * np.sin(np.pi * xi / half)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_kahan"])
@pytest.mark.parametrize("axes", [(0, 1), (1,)])
def test_nonuniform_step_matches_oracle(pkg, prec, axes):
    """The paper's Gaussian pulse (Sec. 4.1) on 65^2 points (2 x 4 patches, n_nb = 16) with stretched knots on one
    or both axes (spacings varying by a factor 1.86), 300 steps of 1e-4 s: every field at three checkpoints element
    by element, and pressure and v3 traces on a row, against the oracle's literal Strang steps on the same knots."""
    import dataclasses

    from synth import gaussian_pulse_2d

    n = 64
    w, _ = gaussian_pulse_2d(n, p=2, n_nb=16, dt=1e-4, steps=300)
    w = dataclasses.replace(w, p=(2, 4), receivers={"sigma": 40 * 65 + np.arange(65), "v3": 40 * 65 + np.arange(65)})
    knots = {a: _stretched(n) for a in axes}
    xs = [knots.get(a, np.linspace(-5.0, 5.0, n + 1)) for a in (0, 1)]
    s0 = np.exp(-5.0 * (xs[0][:, None] ** 2 + xs[1][None, :] ** 2))
    st = {"sigma": s0, "v1": np.zeros(w.shape), "v3": np.zeros(w.shape)}
    sim = nu.simulation(w, knots, state=st)
    g = pkg.Grid.from_workloads([w], precision=prec)
    for a, x in knots.items():
        g.set_coordinates(0, a, x)
    g.set_field(0, "sigma", s0)
    tol = TOL[prec] if prec == "fp64" else 1e-5
    for _ in range(3):
        g.step(100)
        sim.step(100)
        for f in ("sigma", "v1", "v3"):
            ref = sim.state[f]
            got = g.get_field(0, f).astype(np.float64)
            assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref), (f, prec)
            assert np.abs(got - ref).max() <= 10 * tol * np.abs(ref).max(), (f, prec)
    rec = g.record(0)
    for f in ("sigma", "v3"):
        ref = sim.trace_array(f)
        assert np.abs(rec[f] - ref).max() <= 10 * tol * np.abs(ref).max(), f
    g.close()


_REF = {}


def _padded_stretched(nt, h, pad, eps=0.3):
    xi = -5.0 + h * (np.arange(nt + 1) - pad)
    half = xi[-1]
    return xi + eps * (half / np.pi) * np.sin(np.pi * xi / half)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_kahan"])
@pytest.mark.parametrize("order", ["layer first", "knots first"])
def test_nonuniform_step_with_absorbing_layers_matches_oracle(pkg, prec, order):
    """The Gaussian pulse on 65^2 points with stretched knots on both axes and 8-interval absorbing layers outside
    [-5, 5]^2, their profiles on the physical distance into the layer: 1200 steps of 1e-4 s, through the time the
    pulse enters the layers, every field at three checkpoints against the oracle.  The layer is set before the
    knots (its tables are rebuilt for them) or after."""
    import dataclasses

    from synth import gaussian_pulse_2d

    n, pad = 48, 8
    w, _ = gaussian_pulse_2d(n, p=2, n_nb=12, dt=1e-4, steps=1200, pad=pad)
    w = dataclasses.replace(w, pml_width=pad)
    x = _padded_stretched(n + 2 * pad, 10.0 / n, pad)
    knots = {0: x, 1: x}
    s0 = np.exp(-5.0 * (x[:, None] ** 2 + x[None, :] ** 2))
    if "layered" not in _REF:
        sim = nu.simulation(w, knots, state={"sigma": s0, "v1": np.zeros(w.shape), "v3": np.zeros(w.shape)})
        snaps = []
        for _ in range(3):
            sim.step(400)
            snaps.append({f: sim.state[f].copy() for f in ("sigma", "v1", "v3")})
        _REF["layered"] = snaps
    g = pkg.Grid.from_workloads([w], precision=prec)  # sets the layer
    for a, xa in knots.items():
        g.set_coordinates(0, a, xa)
    if order == "knots first":
        g.set_pml(0, pad, w.pml_R, w.pml_kmax, w.f0)
    g.set_field(0, "sigma", s0)
    tol = TOL[prec] if prec == "fp64" else 1e-5
    for snap in _REF["layered"]:
        g.step(400)
        for f in ("sigma", "v1", "v3"):
            ref = snap[f]
            got = g.get_field(0, f).astype(np.float64)
            assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref), (f, prec)
            assert np.abs(got - ref).max() <= 10 * tol * np.abs(ref).max(), (f, prec)
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_kahan"])
def test_nonuniform_step_with_a_source_matches_oracle(pkg, prec):
    """A 15 Hz Ricker pressure source at the centre of 97^2 knots stretched by 1.86 along both axes (1.3 h at the
    source), with 12-point absorbing layers and pressure receivers on row 30: its amplitude is the Gaussian of width
    2 h on the physical distance from the source knot, normalised with the knots' cell volumes.  120 steps, every
    field at three checkpoints and the traces against the oracle."""
    import dataclasses

    from synth import acoustic2d_small

    n = 96
    w = acoustic2d_small(n=n, p=2, n_nb=12, steps=120, pml_width=12)
    w = dataclasses.replace(w, receivers={"sigma": 30 * (n + 1) + np.arange(n + 1, dtype=np.int64)})
    h = w.h[0]
    xi = h * np.arange(n + 1) - h * n / 2
    x = xi + 0.3 * (xi[-1] / np.pi) * np.sin(np.pi * xi / xi[-1]) + h * n / 2
    knots = {0: x, 1: x}
    key = "source"
    if key not in _REF:
        sim = nu.simulation(w, knots)
        snaps = []
        for _ in range(3):
            sim.step(40)
            snaps.append({f: sim.state[f].copy() for f in ("sigma", "v1", "v3")})
        _REF[key] = (snaps, sim.trace_array("sigma"))
    snaps, ref_tr = _REF[key]
    g = pkg.Grid.from_workloads([w], precision=prec)
    for a, xa in knots.items():
        g.set_coordinates(0, a, xa)
    tol = TOL[prec] if prec == "fp64" else 1e-5
    smax = 0.0
    for snap in snaps:
        g.step(40)
        for f in ("sigma", "v1", "v3"):
            ref = snap[f]
            got = g.get_field(0, f).astype(np.float64)
            assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref), (f, prec)
            assert np.abs(got - ref).max() <= 10 * tol * np.abs(ref).max(), (f, prec)
        smax = max(smax, np.abs(snap["sigma"]).max())
    tr = g.record(0)["sigma"].astype(np.float64)
    assert np.abs(tr - ref_tr).max() <= 10 * tol * smax, prec
    assert np.abs(ref_tr).max() > 1e-3 * smax  # the wave has reached the receivers
    g.close()


def test_nonuniform_derivative_throughput(pkg):
    """257^3 FP32, 4 x 4 x 4 patches, n_nb = 20, non-uniform knots on every axis: one derivative per axis on device
    arrays, timed with CUDA events after a warm-up (reported, and a floor against a pathological slowdown)."""
    import torch

    n = 256
    d = pkg.make_desc(3, pkg.LOSS_ACOUSTIC, pkg.LOSS_FP32, 20, (n,) * 3, (4,) * 3, (10.0,) * 3, 1e-3)
    g = pkg.Grid([d])
    for a in range(3):
        g.set_coordinates(0, a, _knots(n, 200 + a))
    f = torch.randn((n + 1,) * 3, device="cuda", dtype=torch.float32)
    res = {}
    for a in range(3):
        g.derivative(0, a, f)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            g.derivative(0, a, f)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / 5
        res[a] = ((n + 1) ** 3 / (ms * 1e-3), 8 * (n + 1) ** 3 / (ms * 1e-3) / 1e9)
    print("non-uniform derivative 257^3 FP32, pt/s and GB/s (read f + write d) per axis z, y, x:", res)
    assert min(v[0] for v in res.values()) > 1e9
    g.close()
