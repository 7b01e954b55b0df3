"""Pins of the oracle's 3-D elastic source-to-receiver path (CPU only) against exact solutions in a homogeneous
medium, summed over the source's Gaussian profile: a body force along z against Stokes' point-force solution, the
explosive source against the pure P field it must radiate, and the shear source against its double couple.

For a force F(t) along x_j at the origin (rho, P speed alpha, S speed beta, gamma = x / r), the particle velocity
is the time derivative of Stokes' displacement solution:

    v_i = 1 / (4 pi rho) [ (3 gamma_i gamma_j - delta_ij) / r^3 ( (r / alpha) F(t - r / alpha) - (r / beta) F(t - r / beta)
                                                                   + int_{t - r / beta}^{t - r / alpha} F(s) ds )
                           + gamma_i gamma_j / (alpha^2 r) F'(t - r / alpha) - (gamma_i gamma_j - delta_ij) / (beta^2 r) F'(t - r / beta) ]

with F = amp f_r, the Ricker wavelet, whose antiderivative is (t - t0) exp(-(pi f0 (t - t0))^2).  Receivers sit
10 cells from the source along the force, across it, on a diagonal and off every axis, on a 41^3 grid with an
8-point absorbing layer.  The difference is the discretisation error, 0.15-0.31 % of the peak.  A wrong modulus,
buoyancy, force timing or sign would show as several percent or more.

The explosive source adds s(t) A(x) to the rate of each normal stress (s = amp f_r).  With S the time integral of
s, that is the body force S(t) grad A.  Its field is the gradient of a P potential phi with phi_tt - alpha^2
Laplacian phi = S A / rho, so v = grad sum_k A_k h^3 s(t - r_k / alpha) / (4 pi rho alpha^2 r_k): radial, with no S
wave.  It agrees to about 0.2-0.3 % of the peak.  At the three receivers on symmetry axes and planes of the grid
and source (along z, along x, on the x = z diagonal) the velocity components across the source-receiver
direction, which an S wave would carry, stay at rounding level (below 1e-10 of the peak); a source that broke the
isotropy of the three normal stresses would put them at the P wave's order there.

The shear source adds s A to the rate of sigma13 (x-z).  That is the body force S (d_z A, 0, d_x A), a double
couple, whose velocity is sum_k A_k h^3 (d_z U^(x) + d_x U^(z)), where U^(j) is Stokes' displacement for a force of
history s along x_j.  The tau-weighted integral in U uses the closed form of int s f_r(s) ds.  The spatial
derivatives are central differences of the closed form with a 1 cm step, against a 55 m time scale.  It agrees
to about 0.2-0.3 % of the peak.
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


def _ricker_moment(t, f0, t0):
    """An antiderivative of s f_r(s): exp(-c x^2) (x^2 + 1 / (2c)) + t0 x exp(-c x^2), x = s - t0, c = (pi f0)^2."""
    x = t - t0
    c = (math.pi * f0) ** 2
    return np.exp(-c * x * x) * (x * x + 0.5 / c) + t0 * x * np.exp(-c * x * x)


def _stokes_displacement(dx, t, alpha, beta, rho, f0, t0, amp, j):
    """Displacement [points, 3] (array-axis order) of a force amp f_r along array axis j at each offset -dx."""
    r = np.linalg.norm(dx, axis=1)
    g = dx / r[:, None]
    ta, tb = t - r / alpha, t - r / beta
    # int_{r / alpha}^{r / beta} tau F(t - tau) dtau = int_{tb}^{ta} (t - s) F(s) ds
    J = t * (_ricker_integral(ta, f0, t0) - _ricker_integral(tb, f0, t0)) - (_ricker_moment(ta, f0, t0)
                                                                             - _ricker_moment(tb, f0, t0))
    out = np.empty((len(r), 3))
    for i in range(3):
        gij = g[:, i] * g[:, j]
        dij = 1.0 if i == j else 0.0
        out[:, i] = amp / (4.0 * math.pi * rho) * ((3.0 * gij - dij) / r**3 * J + gij / (alpha**2 * r) * _ricker(ta, f0, t0)
                                                   - (gij - dij) / (beta**2 * r) * _ricker(tb, f0, t0))
    return out


def _shear_velocity(dx, weight, t, alpha, beta, rho, f0, t0, amp, step=1e-2):
    """Velocity of the weighted x-z double couples: sum of d_z U^(x) + d_x U^(z) (array axes: x = 2, z = 0)."""
    keep = np.linalg.norm(dx, axis=1) > 1.0
    dx, weight = dx[keep], weight[keep]
    total = np.zeros(3)
    for n, m in ((2, 0), (0, 2)):
        e = np.zeros(3)
        e[m] = step
        du = (_stokes_displacement(dx + e, t, alpha, beta, rho, f0, t0, amp, n)
              - _stokes_displacement(dx - e, t, alpha, beta, rho, f0, t0, amp, n)) / (2.0 * step)
        total += (weight[:, None] * du).sum(0)
    return total


def _explosion_velocity(dx, weight, t, alpha, rho, f0, t0, amp):
    """Velocity (array-axis order) of the weighted explosive sources: grad of s(t - r / alpha) / (4 pi rho alpha^2 r)."""
    r = np.linalg.norm(dx, axis=1)
    keep = r > 0
    dx, weight, r = dx[keep], weight[keep], r[keep]
    g = dx / r[:, None]
    ta = t - r / alpha
    radial = -(amp * _ricker_rate(ta, f0, t0) / (alpha * r) + amp * _ricker(ta, f0, t0) / r**2)
    return np.array([float(np.sum(weight * g[:, i] * radial)) for i in range(3)]) / (4.0 * math.pi * rho * alpha**2)


RECEIVERS = ((10, 0, 0), (0, 0, 10), (7, 0, 7), (-6, 5, 4))


def _run(kind, t_end, f0=10.0):
    """Oracle velocities (z, y, x) at the receivers every 4 steps, with the profile points and weights."""
    w = elastic3d_homogeneous(n=40, p=2, n_nb=8, steps=0, pml_width=8)
    w = dataclasses.replace(w, src_kinds=(kind,), receivers={}, f0=f0, t0=1.2 / f0)
    sim = Simulation(w)
    src = np.array(w.src_index)
    off = np.arange(-12, 13)
    O = np.stack(np.meshgrid(off, off, off, indexing="ij"), -1).reshape(-1, 3)
    A = np.exp(-(O**2).sum(1) / 8.0)  # std 2 cells, |offset| <= 12 cells per axis, normalised to the total
    A /= A.sum()
    traces = {r: [] for r in RECEIVERS}
    times = []
    for k in range(int(round(t_end / w.dt))):
        sim.step(1, record=False)
        if (k + 1) % 4 == 0:
            times.append((k + 1) * w.dt)
            for r in RECEIVERS:
                p = tuple(src + np.array(r))
                traces[r].append([sim.state["v3"][p], sim.state["v2"][p], sim.state["v1"][p]])
    return w, O, A, times, traces


def test_point_force_matches_stokes_solution():
    w, O, A, times, traces = _run("force_z", 0.22)
    vp, vs, rho = (float(a.flat[0]) for a in w.model())
    for r in RECEIVERS:
        dx = (np.array(r)[None, :] - O) * w.h[0]
        exact = np.array([_stokes_velocity(dx, A, t, vp, vs, rho, w.f0, w.t0, w.amp, 0) for t in times])
        err = np.abs(np.array(traces[r]) - exact).max() / np.abs(exact).max()
        assert err < 1e-2, (r, err)


def test_explosive_source_radiates_the_exact_p_field():
    w, O, A, times, traces = _run("explosive", 0.22)
    vp, _, rho = (float(a.flat[0]) for a in w.model())
    for r in RECEIVERS:
        dx = (np.array(r)[None, :] - O) * w.h[0]
        exact = np.array([_explosion_velocity(dx, A, t, vp, rho, w.f0, w.t0, w.amp) for t in times])
        err = np.abs(np.array(traces[r]) - exact).max() / np.abs(exact).max()
        assert err < 1e-2, (r, err)
        if r != (-6, 5, 4):  # on a symmetry axis or plane: no transverse motion
            v = np.array(traces[r])
            g = np.array(r, dtype=np.float64) / np.linalg.norm(r)
            across = v - (v @ g)[:, None] * g[None, :]
            assert np.abs(across).max() < 1e-10 * np.abs(v).max(), (r, np.abs(across).max() / np.abs(v).max())


def test_shear_source_radiates_the_exact_double_couple_field():
    w, O, A, times, traces = _run("shear_xz", 0.22)
    vp, vs, rho = (float(a.flat[0]) for a in w.model())
    for r in RECEIVERS:
        dx = (np.array(r)[None, :] - O) * w.h[0]
        exact = np.array([_shear_velocity(dx, A, t, vp, vs, rho, w.f0, w.t0, w.amp) for t in times])
        err = np.abs(np.array(traces[r]) - exact).max() / np.abs(exact).max()
        assert err < 1e-2, (r, err)
