"""Pin of the oracle's source-to-receiver path (CPU only): a pressure source in a homogeneous 2-D acoustic medium
against the exact solution built from the 2-D Green's function.

With constant rho and kappa = rho c^2, the stepper of Sec. 2 / 3.3 with a pressure source s(t) A(x) (A the
normalised Gaussian profile, s = amp f_r, the Ricker wavelet) gives sigma_tt - c^2 Laplacian sigma = s'(t) A(x).
The causal Green's function of the 2-D wave operator is H(ct - r) / (2 pi c sqrt(c^2 t^2 - r^2)), so

    sigma(x, t) = sum_k A_k h^2 (1 / (2 pi c^2)) int_0^{acosh(c t / r_k)} s'(t - (r_k / c) cosh u) du,

where r_k is the distance from source point k (the substitution c tau = r cosh u removes the singularity at the
wavefront).  Receivers 350 m from the source along both axes and along the diagonal are compared until 0.32 s,
before any echo from the grid's ends returns.  The difference is the LOSS discretisation error: it falls by
about 2^4 when h is halved (the time step, at 0.1 h / c, plays no visible part).  A wrong source normalisation,
source time, kappa or b would leave a difference that does not converge.
"""
import dataclasses
import functools
import math

import numpy as np

from oracle.wave import Simulation
from synth import acoustic2d_small


def _ricker_rate(t, f0, t0):
    """d/dt of (1 - 2 a) exp(-a), a = (pi f0 (t - t0))^2."""
    a = (math.pi * f0 * (t - t0)) ** 2
    dadt = 2.0 * (math.pi * f0) ** 2 * (t - t0)
    return -dadt * np.exp(-a) * (3.0 - 2.0 * a)


@functools.lru_cache(maxsize=4)
def _gauss_legendre(nodes):
    return np.polynomial.legendre.leggauss(nodes)


def _exact_sigma(points, t, c, f0, t0, amp, nodes=300):
    k, wq = _gauss_legendre(nodes)
    out = 0.0
    for r, weight in points:
        if c * t <= r:
            continue
        U = math.acosh(c * t / r)
        u = 0.5 * U * (k + 1.0)
        tp = t - (r / c) * np.cosh(u)
        out += weight * float((0.5 * U * wq * amp * _ricker_rate(tp, f0, t0)).sum()) / (2.0 * math.pi * c * c)
    return out


def _max_error(n, h):
    c = 2000.0
    w = acoustic2d_small(n=n, p=2, n_nb=12, steps=0, pml_width=0)
    w = dataclasses.replace(w, h=(h, h), dt=0.1 * h / c, receivers={})
    sim = Simulation(w)
    z0, x0 = w.src_index
    off = np.arange(-12, 13)
    A = np.exp(-(off[:, None] ** 2 + off[None, :] ** 2) / 8.0)  # std 2 cells, |offset| <= 12 cells per axis
    A /= A.sum()
    d, q = int(round(350.0 / h)), int(round(250.0 / h))
    receivers = [(d, 0), (0, -d), (q, q)]
    steps, every = int(round(0.32 / w.dt)), int(round(0.004 / w.dt))
    traces = {r: [] for r in receivers}
    times = []
    for k in range(steps):
        sim.step(1, record=False)
        if (k + 1) % every == 0:
            times.append((k + 1) * w.dt)
            for r in receivers:
                traces[r].append(sim.state["sigma"][z0 + r[0], x0 + r[1]])
    errs = []
    for r in receivers:
        pts = [(h * math.hypot(r[0] - i, r[1] - j), A[i + 12, j + 12]) for i in off for j in off]
        exact = np.array([_exact_sigma(pts, t, c, w.f0, w.t0, w.amp) for t in times])
        errs.append(np.abs(np.array(traces[r]) - exact).max() / np.abs(exact).max())
    return np.array(errs)


def test_point_source_matches_the_2d_greens_function_at_fourth_order():
    coarse = _max_error(120, 10.0)
    fine = _max_error(240, 5.0)
    assert (fine < 2e-3).all(), fine
    assert (np.log2(coarse / fine) > 2.5).all(), (coarse, fine)
