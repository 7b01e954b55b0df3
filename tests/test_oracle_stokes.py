"""Pin of the oracle's 3-D elastic source-to-receiver path (CPU only): a body force along z in a homogeneous
medium against Stokes' exact solution for a point force, summed over the source's Gaussian profile.

For a force F(t) along x_j at the origin (rho, P speed alpha, S speed beta, gamma = x / r), the particle velocity
is the time derivative of Stokes' displacement solution:

    v_i = 1 / (4 pi rho) [ (3 gamma_i gamma_j - delta_ij) / r^3 ( (r / alpha) F(t - r / alpha) - (r / beta) F(t - r / beta)
                                                                   + int_{t - r / beta}^{t - r / alpha} F(s) ds )
                           + gamma_i gamma_j / (alpha^2 r) F'(t - r / alpha) - (gamma_i gamma_j - delta_ij) / (beta^2 r) F'(t - r / beta) ]

with F = amp f_r, the Ricker wavelet, whose antiderivative is (t - t0) exp(-(pi f0 (t - t0))^2).  Receivers sit
12 cells from the source along the force, across it, on a diagonal and off every axis, on a 49^3 grid with a
10-point absorbing layer.  The difference is the discretisation error, 0.2-0.25 % of the peak.  A wrong modulus,
buoyancy, force timing or sign would show as several percent or more.
"""
import dataclasses
import math

import numpy as np

from oracle.wave import Simulation
from synth import elastic3d_homogeneous


def _ricker(t, f0, t0):
    a = (math.pi * f0 * (t - t0)) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def _ricker_rate(t, f0, t0):
    a = (math.pi * f0 * (t - t0)) ** 2
    return -2.0 * (math.pi * f0) ** 2 * (t - t0) * np.exp(-a) * (3.0 - 2.0 * a)


def _ricker_integral(t, f0, t0):
    return (t - t0) * np.exp(-((math.pi * f0 * (t - t0)) ** 2))


def _stokes_velocity(dx, weight, t, alpha, beta, rho, f0, t0, amp, j):
    """Velocity (array-axis order z, y, x) at the receiver of the weighted point forces along array axis j at
    offsets -dx (dx = receiver - source point, metres)."""
    r = np.linalg.norm(dx, axis=1)
    keep = r > 0  # a profile point on the receiver itself carries a weight of e^-18
    dx, weight, r = dx[keep], weight[keep], r[keep]
    g = dx / r[:, None]
    ta, tb = t - r / alpha, t - r / beta
    out = np.zeros(3)
    for i in range(3):
        gij = g[:, i] * g[:, j]
        dij = 1.0 if i == j else 0.0
        near = (3.0 * gij - dij) / r**3 * ((r / alpha) * _ricker(ta, f0, t0) - (r / beta) * _ricker(tb, f0, t0)
                                            + _ricker_integral(ta, f0, t0) - _ricker_integral(tb, f0, t0))
        far = gij / (alpha**2 * r) * _ricker_rate(ta, f0, t0) - (gij - dij) / (beta**2 * r) * _ricker_rate(tb, f0, t0)
        out[i] = amp / (4.0 * math.pi * rho) * float(np.sum(weight * (near + far)))
    return out


def test_point_force_matches_stokes_solution():
    f0, h = 10.0, 10.0
    w = elastic3d_homogeneous(n=48, p=2, n_nb=8, steps=0, pml_width=10)
    w = dataclasses.replace(w, src_kinds=("force_z",), receivers={}, f0=f0, t0=1.2 / f0)
    vp, vs, rho = (float(a.flat[0]) for a in w.model())
    sim = Simulation(w)
    src = np.array(w.src_index)
    off = np.arange(-12, 13)
    O = np.stack(np.meshgrid(off, off, off, indexing="ij"), -1).reshape(-1, 3)
    A = np.exp(-(O**2).sum(1) / 8.0)  # std 2 cells, |offset| <= 12 cells per axis, normalised to the total force
    A /= A.sum()
    receivers = [np.array(r) for r in ((12, 0, 0), (0, 0, 12), (8, 0, 8), (-7, 6, 5))]
    steps = int(round(0.26 / w.dt))
    traces = {q: [] for q in range(len(receivers))}
    times = []
    for k in range(steps):
        sim.step(1, record=False)
        if (k + 1) % 4 == 0:
            times.append((k + 1) * w.dt)
            for q, r in enumerate(receivers):
                p = tuple(src + r)
                traces[q].append([sim.state["v3"][p], sim.state["v2"][p], sim.state["v1"][p]])
    for q, r in enumerate(receivers):
        exact = np.array([_stokes_velocity((r[None, :] - O) * h, A, t, vp, vs, rho, f0, w.t0, w.amp, 0)
                          for t in times])
        err = np.abs(np.array(traces[q]) - exact).max() / np.abs(exact).max()
        assert err < 1e-2, (tuple(r), err)
