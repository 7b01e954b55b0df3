"""Pins of the oracle's non-uniform-grid LOSS derivative (oracle/nonuniform.py; the paper's Sec. 3 remark that the
construction carries over to non-uniform grids)."""
import numpy as np
import pytest
from scipy.interpolate import CubicSpline

from oracle import nonuniform as nu
from oracle import spline


def _knots(N, seed, ratio=2.0):
    """Strictly increasing knots with neighbouring spacings within a factor `ratio` of each other overall."""
    rng = np.random.default_rng(seed)
    h = np.exp(rng.uniform(0.0, np.log(ratio), size=N))
    return np.concatenate([[0.0], np.cumsum(h)]) * 7.0


@pytest.mark.parametrize("N,p,seed", [(48, 4, 1), (36, 3, 2), (40, 1, 3)])
def test_complete_sums_equal_natural_cubic_spline(N, p, seed):
    """With n_nb >= N every PMBC sum is complete, so the patched derivative is the global natural spline's: it
    must equal an independent natural cubic spline (scipy CubicSpline) at every knot, first and second
    derivative."""
    x = _knots(N, seed)
    f = np.random.default_rng(seed + 10).standard_normal((3, N + 1))
    d1, d2 = nu.derivative_1d(f, x, p, N, second=True)
    for r in range(3):
        cs = CubicSpline(x, f[r], bc_type="natural")
        scale1 = np.abs(cs(x, 1)).max()
        scale2 = np.abs(cs(x, 2)).max()
        assert np.abs(d1[r] - cs(x, 1)).max() < 1e-11 * scale1
        assert np.abs(d2[r] - cs(x, 2)).max() < 1e-10 * scale2


@pytest.mark.parametrize("n,p,n_nb", [(32, 2, 6), (48, 4, 12)])
def test_uniform_knots_reduce_to_the_uniform_oracle(n, p, n_nb):
    """On equally spaced knots the B-splines are the paper's (rows (1, 4, 1)/6, derivative +-1/(2h)): the result
    equals the uniform-grid oracle with the same truncated sums."""
    h = 2.5
    x = h * np.arange(n + 1)
    f = np.random.default_rng(5).standard_normal((4, n + 1))
    a1, a2 = nu.derivative_1d(f, x, p, n_nb, second=True)
    b1, b2 = spline.derivative_1d(f, n, p, h, n_nb, second=True)
    assert np.abs(a1 - b1).max() < 1e-12 * np.abs(b1).max()
    assert np.abs(a2 - b2).max() < 1e-11 * np.abs(b2).max()


def test_truncation_error_decays_exponentially():
    """The weights of the global inverse decay geometrically away from the junction, so the error of the truncated
    PMBC sums falls geometrically with n_nb (rate near |sqrt(3) - 2| = 0.268 for mild spacing variations)."""
    N, p = 96, 4
    x = _knots(N, 7, ratio=1.5)
    f = np.random.default_rng(8).standard_normal((2, N + 1))
    full = nu.derivative_1d(f, x, p, N)
    errs = [np.abs(nu.derivative_1d(f, x, p, k) - full).max() for k in (4, 8, 12, 16)]
    for a, b in zip(errs, errs[1:]):
        assert b < a * 0.06  # four more terms: at most 0.06 of the error (0.268^4 = 5.2e-3 for uniform knots)
    assert errs[-1] < 1e-8 * np.abs(full).max()


def test_slope_equations_hold_inside_every_patch():
    """C^2 continuity of the local spline at an interior knot i of a patch gives, whatever the junction values,
    h_i d_{i-1} + 2 (h_{i-1} + h_i) d_i + h_{i-1} d_{i+1} = 3 (h_i (f_i - f_{i-1}) / h_{i-1}
    + h_{i-1} (f_{i+1} - f_i) / h_i), with h_i = x_{i+1} - x_i (the non-uniform form of the compact identity)."""
    N, p, n_nb = 60, 3, 5
    x = _knots(N, 9)
    f = np.random.default_rng(10).standard_normal((2, N + 1))
    d = nu.derivative_1d(f, x, p, n_nb)
    h = np.diff(x)
    M = N // p
    for l in range(p):
        for i in range(l * M + 1, (l + 1) * M):
            lhs = h[i] * d[:, i - 1] + 2 * (h[i - 1] + h[i]) * d[:, i] + h[i - 1] * d[:, i + 1]
            rhs = 3 * (h[i] * (f[:, i] - f[:, i - 1]) / h[i - 1] + h[i - 1] * (f[:, i + 1] - f[:, i]) / h[i])
            assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(rhs).max() + 1e-13


def test_junction_values_equal_phi_and_linear_fields_are_exact():
    N, p, n_nb = 48, 4, 8
    x = _knots(N, 11)
    f = np.random.default_rng(12).standard_normal((3, N + 1))
    d = nu.derivative_1d(f, x, p, n_nb)
    phi = nu.pmbc_phi(f, x, p, n_nb)
    M = N // p
    for j in range(p + 1):
        assert np.abs(d[:, j * M] - phi[:, j]).max() < 1e-12 * np.abs(phi).max()
    lin = 3.0 - 0.7 * x  # with complete sums the natural spline reproduces linear data exactly
    d_lin = nu.derivative_1d(lin[None, :], x, p, N)
    assert np.abs(d_lin + 0.7).max() < 1e-12


def _stretched(n, eps=0.3, half=5.0):
    """n + 1 knots on [-half, half]: x = xi + eps (half / pi) sin(pi xi / half) for uniform xi, a smooth map with
    spacings varying by a factor (1 + eps) / (1 - eps)."""
    xi = np.linspace(-half, half, n + 1)
    return xi + eps * (half / np.pi) * np.sin(np.pi * xi / half)


def test_pulse_on_stretched_grids_converges_to_the_exact_solution():
    """The paper's Gaussian pulse (Sec. 4.1) stepped on grids whose spacing varies smoothly by a factor 1.86 along
    both axes: against the exact solution of the same Strang time stepping (oracle/exact.py) at the knots, the error
    falls at high order with refinement and stays within a small factor of the uniform grid's."""
    import dataclasses

    from oracle.exact import pulse_solution
    from oracle.wave import Simulation
    from synth import gaussian_pulse_2d

    steps, dt = 200, 1e-4
    errs, errs_u = [], []
    for n in (32, 64):
        w, s0u = gaussian_pulse_2d(n, p=2, n_nb=16, dt=dt, steps=steps)
        x = _stretched(n)
        s0 = np.exp(-5.0 * (x[:, None] ** 2 + x[None, :] ** 2))
        sim = nu.simulation(w, {0: x, 1: x}, state={"sigma": s0, "v1": np.zeros(w.shape), "v3": np.zeros(w.shape)})
        sim.step(steps, record=False)
        ref_s, ref_v3 = pulse_solution(x[None, :], x[:, None], steps, dt)
        errs.append(np.abs(sim.state["v3"] - ref_v3).max() / np.abs(ref_v3).max())
        xu = np.linspace(-5.0, 5.0, n + 1)
        u = Simulation(dataclasses.replace(w), state={"sigma": s0u, "v1": np.zeros(w.shape),
                                                      "v3": np.zeros(w.shape)}).step(steps, record=False)
        ref_u = pulse_solution(xu[None, :], xu[:, None], steps, dt)[1]
        errs_u.append(np.abs(u.state["v3"] - ref_u).max() / np.abs(ref_u).max())
    order = np.log2(errs[0] / errs[1])
    assert order > 3.0, (errs, order)
    assert errs[1] < 4.0 * errs_u[1], (errs, errs_u)


def test_uniform_knots_step_like_the_uniform_oracle():
    from oracle.wave import Simulation
    from synth import gaussian_pulse_2d

    w, s0 = gaussian_pulse_2d(32, p=2, n_nb=12, dt=1e-4, steps=20)
    st = {"sigma": s0, "v1": np.zeros(w.shape), "v3": np.zeros(w.shape)}
    a = Simulation(w, state=st).step(20, record=False)
    x = np.linspace(-5.0, 5.0, 33)
    b = nu.simulation(w, {0: x, 1: x}, state=st).step(20, record=False)
    for f in ("sigma", "v1", "v3"):
        assert np.abs(a.state[f] - b.state[f]).max() < 1e-12 * np.abs(a.state[f]).max()


def test_layer_profiles_on_equal_knots_are_the_uniform_layers():
    """On equally spaced knots the physical-distance profiles are wave.PML's, value for value."""
    from oracle.wave import PML

    for n, W, h in ((64, 12, 10.0), (40, 8, 0.25)):
        x = h * np.arange(n + 1)
        ref = PML((n,), (h,), W, 1e-6, 1.0, 15.0, 2000.0).prof[0]
        got = nu.layer_profiles(x, W, 1e-6, 1.0, 15.0, 2000.0)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)


def _padded_stretched(nt, h, pad, eps=0.3):
    xi = -5.0 + h * (np.arange(nt + 1) - pad)
    half = xi[-1]
    return xi + eps * (half / np.pi) * np.sin(np.pi * xi / half)


def test_uniform_knots_with_a_layer_step_like_the_uniform_oracle():
    import dataclasses

    from oracle.wave import Simulation
    from synth import gaussian_pulse_2d

    w, s0 = gaussian_pulse_2d(32, p=2, n_nb=12, dt=1e-4, steps=60, pad=8)
    w = dataclasses.replace(w, pml_width=8)
    st = {"sigma": s0, "v1": np.zeros(w.shape), "v3": np.zeros(w.shape)}
    a = Simulation(w, state=st).step(60, record=False)
    x = w.h[0] * np.arange(w.n[0] + 1)
    b = nu.simulation(w, {0: x, 1: x}, state=st).step(60, record=False)
    for f in ("sigma", "v1", "v3"):
        assert np.abs(a.state[f] - b.state[f]).max() < 1e-10 * np.abs(a.state[f]).max()


def test_layer_absorbs_on_stretched_knots():
    """The Gaussian pulse on knots stretched by a factor 1.86, with 8-interval layers outside [-5, 5]^2 (2.5 m
    thick): after 0.36 s (900 steps of 4e-4 s) the pressure energy left on the grid is below 1 % of the initial
    one and within a factor 3 of the uniform grid's with the same layers (measured 2.6e-3 and 4.7e-3, as with
    steps of 1e-4 s), while without layers the natural-spline end modes make it grow past the initial energy."""
    import dataclasses

    from oracle.wave import Simulation
    from synth import gaussian_pulse_2d

    n, pad, steps = 32, 8, 900
    w, s0u = gaussian_pulse_2d(n, p=2, n_nb=12, dt=4e-4, steps=steps, pad=pad)
    x = _padded_stretched(n + 2 * pad, 10.0 / n, pad)
    s0 = np.exp(-5.0 * (x[:, None] ** 2 + x[None, :] ** 2))
    zero = np.zeros(w.shape)

    def left(sim, init):
        sim.step(steps, record=False)
        return np.sum(sim.state["sigma"] ** 2) / np.sum(init**2)

    wl = dataclasses.replace(w, pml_width=pad)
    e_nu = left(nu.simulation(wl, {0: x, 1: x}, state={"sigma": s0, "v1": zero, "v3": zero}), s0)
    e_u = left(Simulation(wl, state={"sigma": s0u, "v1": zero, "v3": zero}), s0u)
    e_none = left(nu.simulation(w, {0: x, 1: x}, state={"sigma": s0, "v1": zero, "v3": zero}), s0)
    assert e_nu < 1e-2 and e_nu < 3.0 * e_u, (e_nu, e_u)
    assert e_none > 1.0, e_none


def _source_grid(n=96, eps=0.3):
    """The 2-D acoustic workload (2000 m/s, h = 10 m, 15 Hz Ricker pressure source at the centre knot) without
    layers or receivers, and stretched knots on its [0, n h] axes (spacing 1.3 h at the source)."""
    import dataclasses

    from synth import acoustic2d_small

    w = acoustic2d_small(n=n, p=2, n_nb=12, steps=120, pml_width=0)
    w = dataclasses.replace(w, receivers={})
    h = w.h[0]
    xi = h * np.arange(n + 1) - h * n / 2
    half = xi[-1]
    x = xi + eps * (half / np.pi) * np.sin(np.pi * xi / half) + h * n / 2
    return w, {0: x, 1: x.copy()}


def test_knot_source_on_equal_knots_is_the_uniform_source():
    """On equally spaced knots the source amplitude is wave.Source's, and a run with it steps like the uniform
    oracle."""
    import dataclasses

    from oracle.wave import Simulation, Source

    w, _ = _source_grid(n=48)
    w = dataclasses.replace(w, steps=40)
    xu = w.h[0] * np.arange(w.n[0] + 1)
    ks = nu.KnotSource(w.src_index, w.src_kinds, w.f0, w.t0, w.amp, w.h, w.shape, {0: xu, 1: xu})
    us = Source(w.src_index, w.src_kinds, w.f0, w.t0, w.amp, w.h, w.shape)
    assert np.abs(ks.profile - us.profile).max() <= 1e-14 * np.abs(us.profile).max()
    a = Simulation(w).step(40, record=False).state["sigma"]
    b = nu.simulation(w, {0: xu, 1: xu}).step(40, record=False).state["sigma"]
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_knot_source_injects_the_total_of_the_uniform_grid():
    """On stretched knots the amplitude summed with the knots' cell volumes is the source amplitude."""
    w, knots = _source_grid()
    ks = nu.KnotSource(w.src_index, w.src_kinds, w.f0, w.t0, w.amp, w.h, w.shape, knots)
    V = np.multiply.outer(nu.cell_widths(knots[0]), nu.cell_widths(knots[1]))[ks.block]
    assert abs(float(np.sum(ks.profile * V)) - w.amp) <= 1e-13 * abs(w.amp)


def test_knot_source_radiates_the_field_of_the_uniform_grid():
    """A pressure source on knots stretched by 1.86 (1.3 h at the source) radiates the field of the same source on
    the uniform grid: after 120 steps (the wave 30 cells out, before any end is reached) the pressure at the knots
    is 1.25e-2 (L2, relative) from the uniform run's, interpolated there by bicubic splines.  The same source
    amplitude taken on knot offsets instead of physical distance (a source 1.3 times wider) ends 0.33 away."""
    from scipy.interpolate import RectBivariateSpline

    from oracle.wave import Simulation, Source

    w, knots = _source_grid()
    xu = w.h[0] * np.arange(w.n[0] + 1)
    U = Simulation(w).step(w.steps, record=False).state["sigma"]
    Ui = RectBivariateSpline(xu, xu, U, kx=3, ky=3)(knots[0], knots[1])
    S = nu.simulation(w, knots).step(w.steps, record=False).state["sigma"]
    assert np.linalg.norm(S - Ui) <= 3e-2 * np.linalg.norm(Ui)
    sim = nu.simulation(w, knots)
    sim.src = Source(w.src_index, w.src_kinds, w.f0, w.t0, w.amp, w.h, w.shape)
    S2 = sim.step(w.steps, record=False).state["sigma"]
    assert np.linalg.norm(S2 - Ui) > 0.1 * np.linalg.norm(Ui)
