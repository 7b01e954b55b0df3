"""Pins of the oracle's source terms (CPU only).

* The Ricker wavelet (reading of the garbled formula of Sec. 4.2) is the normalised negative second derivative
  of the Gaussian exp(-(pi f0 (t - t0))^2), checked against a finite difference of that Gaussian. Its amplitude
  spectrum peaks at f0, which is what "peak frequency" means, and it has zero mean.
* The Gaussian spatial amplitude sums to amp over the cell volumes (sum A h^d = amp). It is symmetric about the
  source node and keeps that sum when the grid clips it.
* Injected pressure: in an acoustic run whose waves have not reached the ends, the sum of sigma h^2 grows by
  exactly what the B sub-steps add, dt amp f_r(t_n + dt / 2), because the LOSS divergence of a velocity field
  that vanishes near the ends sums to zero up to rounding.
"""
import dataclasses
import math

import numpy as np

from oracle.wave import Simulation, Source, ricker
from synth import acoustic2d_small


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
