"""Pins of the oracle's source terms (CPU only).

* The Ricker wavelet (reading of the garbled formula of Sec. 4.2) is the normalised negative second derivative
  of the Gaussian exp(-(pi f0 (t - t0))^2), checked against a finite difference of that Gaussian. Its amplitude
  spectrum peaks at f0, which is what "peak frequency" means, and it has zero mean.
* The Gaussian spatial amplitude sums to amp over the cell volumes (sum A h^d = amp). It is symmetric about the
  source node and keeps that sum when the grid clips it.
* Injected pressure: in an acoustic run whose waves have not reached the ends, the sum of sigma h^2 grows by
  exactly what the B sub-steps add, dt amp f_r(t_n + dt / 2), because the LOSS divergence of a velocity field
  that vanishes near the ends sums to zero up to rounding.
* Elastic sources inject exactly their own components.  Explosive: sigma11, sigma22 and sigma33 each gain
  sum dt amp f_r(t_n + dt / 2).  Shear: only sigma13 gains it.  Body force along z: the momentum sum of rho v3
  gains the impulse of the two A halves, (dt / 2) amp (f_r(t_n) + f_r(t_n+1)) per step.  Every other field sum
  stays zero: no net force from a moment source, and no net stress from a force.
"""
import dataclasses
import math

import numpy as np
import pytest

from oracle.wave import Simulation, Source, ricker
from synth import acoustic2d_small, elastic3d_homogeneous


def test_ricker_is_the_normalised_second_derivative_of_a_gaussian():
    f0, t0 = 15.0, 0.08
    a = (math.pi * f0) ** 2
    gauss = lambda t: math.exp(-a * (t - t0) ** 2)
    d = 1e-5
    for t in np.linspace(0.0, 0.16, 33):
        second = (gauss(t + d) - 2.0 * gauss(t) + gauss(t - d)) / d**2
        assert abs(ricker(t, f0, t0) - (-second / (2.0 * a))) < 1e-5, t
    assert ricker(t0, f0, t0) == 1.0


def test_ricker_spectrum_peaks_at_f0_and_has_zero_mean():
    f0, t0, dt, n = 20.0, 0.5, 1e-4, 2**16
    t = dt * np.arange(n)
    w = np.array([ricker(x, f0, t0) for x in t])
    spec = np.abs(np.fft.rfft(w))
    freq = np.fft.rfftfreq(n, dt)
    assert abs(freq[np.argmax(spec)] - f0) <= freq[1]
    assert abs(w.sum() * dt) < 1e-12


def test_source_profile_normalisation_symmetry_and_clipping():
    h = (10.0, 7.0)
    full = Source((40, 40), ("pressure",), 15.0, 0.08, 2.5, h, (81, 81))
    assert abs(full.profile.sum() * h[0] * h[1] - 2.5) < 1e-12
    assert np.allclose(full.profile, full.profile[::-1, :]) and np.allclose(full.profile, full.profile[:, ::-1])
    assert full.profile.shape == (25, 25)
    edge = Source((3, 40), ("pressure",), 15.0, 0.08, 2.5, h, (81, 81))  # clipped by the z = 0 end
    assert edge.profile.shape == (16, 25)
    assert abs(edge.profile.sum() * h[0] * h[1] - 2.5) < 1e-12


def test_injected_pressure_is_conserved_before_the_waves_reach_the_ends():
    w = acoustic2d_small(n=96, p=2, n_nb=12, steps=0, pml_width=0)
    w = dataclasses.replace(w, receivers={})
    sim = Simulation(w)
    h2 = w.h[0] * w.h[1]
    # 15 Hz, t0 = 0.08 s: stop at 0.064 s, near the extremum of the wavelet's running integral (which returns to
    # 0 afterwards); the field then reaches about 25 cells from the source and the ends are 48 cells away
    steps = 32
    sim.step(steps, record=False)
    injected = sum(w.dt * w.amp * ricker((k + 0.5) * w.dt, w.f0, w.t0) for k in range(steps))
    total = sim.state["sigma"].sum() * h2
    assert abs(injected) > 1e-4
    assert abs(total - injected) < 1e-9 * abs(injected), (total, injected)


@pytest.mark.parametrize("kind", ["explosive", "shear_xz", "force_x", "force_y", "force_z"])
def test_elastic_sources_inject_exactly_their_own_components(kind):
    w = elastic3d_homogeneous(n=40, p=2, n_nb=8, steps=0, pml_width=0)
    # 60 Hz: stop at 0.016 s, near the extremum of the running integral; the field reaches about 11 cells from
    # the centre and the ends are 20 cells away
    w = dataclasses.replace(w, src_kinds=(kind,), receivers={}, f0=60.0, t0=1.2 / 60.0)
    sim = Simulation(w)
    steps, dt = 12, w.dt
    sim.step(steps, record=False)
    stress_in = sum(dt * w.amp * ricker((k + 0.5) * dt, w.f0, w.t0) for k in range(steps))
    impulse = sum(0.5 * dt * w.amp * (ricker(k * dt, w.f0, w.t0) + ricker((k + 1) * dt, w.f0, w.t0))
                  for k in range(steps))
    rho = w.model()[2]
    vol = float(np.prod(w.h))
    sums = {f: float((a * (rho if f.startswith("v") else 1.0)).sum()) * vol for f, a in sim.state.items()}
    expect = {f: 0.0 for f in sums}
    if kind == "explosive":
        expect.update(s11=stress_in, s22=stress_in, s33=stress_in)
    elif kind == "shear_xz":
        expect["s13"] = stress_in
    else:
        expect["v" + {"x": "1", "y": "2", "z": "3"}[kind[-1]]] = impulse
    scale = max(abs(v) for v in expect.values())
    assert scale > 1e-4
    for f in sums:
        assert abs(sums[f] - expect[f]) < 1e-8 * scale, (f, sums[f], expect[f])


@pytest.mark.parametrize("kind,axis", [("force_x", 2), ("force_y", 1)])
def test_body_force_axes_follow_the_grid_axes(kind, axis):
    """On a cubic homogeneous grid a body force along x (y) radiates the field of the force along z with the grid
    axes z and x (y) exchanged: v_x from force_x is v_z from force_z transposed, and so on for every component.
    Together with the Stokes pin of the z force this pins the direction and sign of the other two."""
    w = elastic3d_homogeneous(n=24, p=2, n_nb=8, steps=0, pml_width=4)
    w = dataclasses.replace(w, receivers={}, f0=60.0, t0=1.2 / 60.0)
    ref = Simulation(dataclasses.replace(w, src_kinds=("force_z",))).step(10, record=False).state
    got = Simulation(dataclasses.replace(w, src_kinds=(kind,))).step(10, record=False).state
    comp = {2: "1", 1: "2"}[axis]  # the velocity component along the exchanged axis
    swap = {"v3": "v" + comp, "v" + comp: "v3"}
    scale = max(float(np.abs(v).max()) for v in ref.values())
    assert scale > 0
    for f in ("v1", "v2", "v3"):
        expect = np.swapaxes(ref[swap.get(f, f)], 0, axis)
        assert np.abs(got[f] - expect).max() < 1e-12 * scale, f
