"""Pins of the oracle's absorbing layer (ADE-PML with the exponential Strang splitting, paper Sec. 3.3)."""
import dataclasses

import numpy as np

from oracle.exact import pulse_on_grid
from oracle.wave import PML, Simulation
from synth import acoustic2d_small, gaussian_pulse_2d
from synth.workloads import Workload


def test_exponential_flow_is_exact_for_frozen_gradient():
    """For a frozen derivative g the memory ODE dPsi/dt = -beta Psi - (d/k^2) g has the closed form used by the
    splitting; two half steps equal one full step (so consecutive half A steps merge exactly)."""
    pml = PML((40,), (1.0,), 10, 1e-6, 1.5, 5.0, 3.0)
    rng = np.random.default_rng(0)
    g = rng.standard_normal(41)
    m1 = rng.standard_normal(41) * (pml.prof[0][0] > 0)
    m2 = m1.copy()
    x_full = pml.advance(m1, g, 0, 0.2)
    x_half = pml.advance(m2, g, 0, 0.1) + pml.advance(m2, g, 0, 0.1)
    assert np.allclose(m1, m2, rtol=0, atol=1e-14)
    assert np.allclose(x_full, x_half, rtol=0, atol=1e-14)
    # Reference: integrate the ODE pair (Psi, integral) with a fine explicit RK4.
    d, k, a = pml.prof[0]
    i = 3
    beta = d[i] / k[i] + a[i]
    psi, acc, h = m1[i] * 0 + 0.7, 0.0, 1e-4
    psi0 = psi
    f = lambda p: -beta * p - d[i] / k[i] ** 2 * g[i]
    for _ in range(2000):
        k1 = f(psi); k2 = f(psi + 0.5 * h * k1); k3 = f(psi + 0.5 * h * k2); k4 = f(psi + h * k3)
        acc += h / 6 * (psi + 2 * (psi + 0.5 * h * k1) + 2 * (psi + 0.5 * h * k2) + (psi + h * k3))
        psi += h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    mem = np.zeros(41); mem[i] = psi0
    x = pml.advance(mem, g, 0, 0.2)
    assert abs(mem[i] - psi) < 1e-10
    # field increment = -tau g / k - integral of Psi
    assert abs(x[i] - (-0.2 * g[i] / k[i] - acc)) < 1e-8


def test_layer_absorbs_outgoing_wave():
    """Energy leaves through the layer: after the wave has crossed it, less than 1 % of the peak energy remains,
    whereas the reflecting box keeps it."""
    w = acoustic2d_small(n=64, p=2, n_nb=12, steps=0, pml_width=16)
    w0 = dataclasses.replace(w, pml_width=0)
    a, b = Simulation(w), Simulation(w0)
    ea, eb = [], []
    for _ in range(24):
        a.step(10, record=False)
        b.step(10, record=False)
        ea.append(a.energy())
        eb.append(b.energy())
    assert ea[-1] < 0.01 * max(ea)
    assert eb[-1] > 0.3 * max(eb)


def test_layer_reflection_is_small():
    """Interior field with a 20-point layer vs. the same interior cut from a twice larger reflecting grid
    before its boundary echo returns: the layer's reflection stays at the percent level of the peak."""
    small = acoustic2d_small(n=128, p=2, n_nb=12, steps=0, pml_width=20)
    big = acoustic2d_small(n=256, p=4, n_nb=12, steps=0, pml_width=0)
    a, b = Simulation(small), Simulation(big)
    steps = 150  # 0.3 s: the pulse has entered the layer of the small grid; no echo from the big grid's ends yet
    a.step(steps, record=False)
    b.step(steps, record=False)
    inner = a.state["sigma"][20:109, 20:109]
    ref = b.state["sigma"][64 + 20:64 + 109, 64 + 20:64 + 109]
    peak = np.abs(ref).max()
    assert np.abs(inner - ref).max() < 0.03 * peak


def _fp32_floor(pml_width, steps=300):
    w = acoustic2d_small(steps=steps, pml_width=pml_width)
    a, b = Simulation(w), Simulation(w)
    peak, worst = 0.0, 0.0
    for _ in range(steps):
        a.step(1, record=False)
        b.step(1, record=False)
        for f in b.state:
            b.state[f] = b.state[f].astype(np.float32).astype(np.float64)
        peak = max(peak, np.linalg.norm(a.state["sigma"]))
        worst = max(worst, np.linalg.norm(a.state["sigma"] - b.state["sigma"]))
    return worst / peak


def test_layer_bounds_rounding_growth():
    """Rounding the state to float32 every step (a model of FP32 storage) stays at the float32 level with the
    layer, while the reflecting box lets zero-frequency polynomial modes amplify it by many orders."""
    assert _fp32_floor(20) < 1e-6
    assert _fp32_floor(0) > 1e-3


def test_elastic_layer_absorbs():
    """3-D elastic: with the layer the radiated P and S energy leaves the grid; without it, it stays."""
    from synth import elastic3d_homogeneous

    w = elastic3d_homogeneous(n=32, p=2, n_nb=8, steps=0, pml_width=8)
    w = dataclasses.replace(w, receivers={}, f0=40.0, t0=1.2 / 40.0, dt=0.4 * 10.0 / 3000.0)
    w0 = dataclasses.replace(w, pml_width=0)
    a, b = Simulation(w), Simulation(w0)
    ea, eb = [], []
    for _ in range(16):
        a.step(10, record=False)
        b.step(10, record=False)
        ea.append(a.energy())
        eb.append(b.energy())
    assert ea[-1] < 0.05 * max(ea), (ea[-1], max(ea))
    assert eb[-1] > 0.3 * max(eb)


def test_layer_absorbs_the_gaussian_pulse_over_the_papers_time_range():
    """Sec. 4.1 up to t = 0.2 s: the pulse on [-5, 5]^2 (64 intervals) padded by 20 points on every side.  With a
    20-point layer in the padding (R = 1e-6, k_max = 1) the v3 error inside [-5, 5]^2 against the free-space
    solution of the time-discrete scheme stays at the discretisation level it has before the wave leaves the
    domain.  Without the layer, the echo from the grid's ends, back inside by 0.2 s, makes it larger than the
    field itself."""
    n, pad = 64, 20
    errs = {}
    for width in (pad, 0):
        w, s0 = gaussian_pulse_2d(n, p=2, n_nb=20, dt=1e-4, steps=2000, pad=pad)
        w = dataclasses.replace(w, pml_width=width)
        sim = Simulation(w, state={"sigma": s0, "v1": 0 * s0, "v3": 0 * s0})
        done = 0
        for steps in (1000, 2000):
            sim.step(steps - done, record=False)
            done = steps
            ref = pulse_on_grid(n, steps, 1e-4)[1]
            v3 = sim.state["v3"][pad:pad + n + 1, pad:pad + n + 1]
            errs[width, steps] = np.linalg.norm(v3 - ref) / np.linalg.norm(ref)
    # by 0.1 s only the pulse's Gaussian tail has reached the layer
    assert abs(errs[pad, 1000] / errs[0, 1000] - 1.0) < 1e-3, errs
    assert errs[pad, 2000] < 1.2 * errs[pad, 1000], errs
    assert errs[0, 2000] > 1.0, errs


def _normal_incidence_reflection(L, R, n=400, h=10.0, c=2000.0, rho=1000.0, width=6.0):
    """Largest |v3| left in the interior after a plane packet (6-cell Gaussian, sigma = rho c v3 so that it moves to
    +z) has entered an L-point layer at the z end and had time to come back to its start."""
    shape = (n + 1, 5)
    w = Workload(name="pml_column", dim=2, physics="acoustic", n=(n, 4), p=(1, 1), h=(h, h), n_nb=20,
                 dt=0.4 * h / c, steps=0, model_fn=lambda: (np.full(shape, c), None, np.full(shape, rho)),
                 src_index=(0, 0), src_kinds=(), f0=1.0, t0=0.0, amp=0.0, precision="fp64", pml_width=L, pml_R=R)
    z = np.arange(n + 1)
    g = np.exp(-(((z - n // 2) / width) ** 2))[:, None] * np.ones(shape)
    sim = Simulation(w, state={"sigma": rho * c * g, "v1": 0 * g, "v3": g.copy()})
    sim.step(int(round(2 * (n - n // 2) * h / c / w.dt)), record=False)
    return float(np.abs(sim.state["v3"][L:n + 1 - L, 2]).max())


def test_layer_meets_its_design_reflection_at_normal_incidence():
    """d0 = -3 c log(R) / (2 L) makes the round trip through a continuous layer attenuate by exactly R (Sec. 3.3).
    The discrete layer of 50 points returns 1.7e-6 of a unit packet for R = 1e-6 and 1.6e-7 for R = 1e-9.  A
    20-point layer adds discretisation reflection (1.2e-5 for R = 1e-6)."""
    assert _normal_incidence_reflection(50, 1e-6) < 3e-6
    assert _normal_incidence_reflection(50, 1e-9) < 3e-7
    assert _normal_incidence_reflection(20, 1e-6) > 5e-6


def test_pml_study_reproduces_the_papers_findings():
    """The oracle's ADE-PML study on 512^2 (tests/golden/pml_tables_oracle.txt, written by make_pml_tables.py from
    oracle/ only) shows what Sec. 4.1 reports: every layer gives the same error until the wave reaches it; at
    0.2 s the error falls with the thickness L and the reflection coefficient R; k_max = 1 is the best cut-off;
    and up to 0.10 s the error falls by 2^4 per doubling of N (Table 2d_error).  Errors are eps_2 = h ||e|| / A
    (one amplitude for the run)."""
    import collections
    import os

    path = os.path.join(os.path.dirname(__file__), "golden", "pml_tables_oracle.txt")
    e = collections.defaultdict(dict)
    for line in open(path):
        if line.startswith("#"):
            continue
        N, L, R, k, steps, _, _, eps2a = line.split()
        e[int(N), int(L), float(R), float(k)][int(steps)] = float(eps2a)
    study = [c for c in e if c[0] == 512]
    for steps in (200, 400, 600):
        vals = [e[c][steps] for c in study]
        assert max(vals) < 1.01 * min(vals), steps
    t = 2000
    assert e[512, 10, 1e-6, 1.0][t] > e[512, 20, 1e-6, 1.0][t] > e[512, 50, 1e-6, 1.0][t]
    assert e[512, 50, 1e-1, 1.0][t] > e[512, 50, 1e-3, 1.0][t] > e[512, 50, 1e-6, 1.0][t] > e[512, 50, 1e-9, 1.0][t]
    late = lambda c: max(e[c][s] for s in range(1000, 2001, 200))
    assert late((512, 50, 1e-6, 1.0)) < 0.2 * min(late((512, 50, 1e-6, 0.5)), late((512, 50, 1e-6, 6.0)))
    for steps in (200, 400, 600, 1000):
        for n in (64, 128, 256):
            order = np.log2(e[n, 50, 1e-6, 1.0][steps] / e[2 * n, 50, 1e-6, 1.0][steps])
            assert 3.9 < order < 4.4, (n, steps, order)
