"""Oracle, part 4: closed-form solutions of the paper's 2-D Gaussian-pulse experiment (Sec. 4.1), FP64.
TEST INFRASTRUCTURE ONLY.

Setup of Sec. 4.1: constant c = 50 m/s and rho = 1 on [-5, 5]^2, zero initial velocity and the initial pressure
sigma(x, z, 0) = exp(-a (x^2 + z^2)) with a = 5.  The acoustic system of Sec. 2 (dv/dt = -grad(sigma)/rho,
dsigma/dt = -rho c^2 div v) is solved in free space mode by mode.  The Hankel transform of exp(-a r^2) is
A(k) = exp(-k^2 / (4a)) / (2a), and each plane-wave mode of wavenumber k behaves as a harmonic oscillator of
frequency w = c k:

    sigma(r, t) = int_0^inf A(k) S(k, t) J0(k r) k dk,    v_r(r, t) = (1 / (rho c)) int_0^inf A(k) U(k, t) J1(k r) k dk,

with v3 = v_r z / r.

Two time laws are offered:

* continuous time, the exact solution of the PDE:  S = cos(w t),  U = sin(w t);
* the exact solution of the Strang-split time stepping of Sec. 3.3 with exact spatial derivatives.  Per mode,
  one step of length tau is a velocity half step, a full pressure step and a velocity half step, each exact with
  the other field frozen.  This is the Stormer-Verlet map of the oscillator, whose n-th iterate from (S, U) = (1, 0)
  is S_n = cos(n theta) and U_n = sin(n theta) sin(theta) / (w tau), where sin(theta / 2) = w tau / 2.
  Compared with this reference, a LOSS run at the same tau shows only its spatial error.  The paper's own
  reference, an FSM (Fourier spectral) solution, also shares the time step, so its errors behave the same way.

The k-integral is a Gauss-Legendre sum on [0, kmax]; A(k) is below 1e-34 at k = 40.
"""
from __future__ import annotations

import functools

import numpy as np
from scipy.special import j0, j1

PULSE_A = 5.0
PULSE_C = 50.0
PULSE_RHO = 1.0


def strang_mode_factors(w_tau: np.ndarray, steps: int):
    """(S_n, U_n) of the Strang map of one oscillator mode after ``steps`` steps from (1, 0); w_tau = w * tau < 2."""
    w_tau = np.asarray(w_tau, dtype=np.float64)
    theta = 2.0 * np.arcsin(0.5 * w_tau)
    with np.errstate(invalid="ignore", divide="ignore"):
        ratio = np.where(w_tau > 0, np.sin(theta) / np.where(w_tau > 0, w_tau, 1.0), 1.0)
    return np.cos(steps * theta), np.sin(steps * theta) * ratio


def _time_law(k, steps, dt, discrete, c):
    if discrete:
        return strang_mode_factors(c * k * dt, steps)
    t = steps * dt
    return np.cos(c * k * t), np.sin(c * k * t)


@functools.lru_cache(maxsize=8)
def _gauss_legendre(nodes: int):
    """Gauss-Legendre nodes and weights on [-1, 1] (computed once per node count; callers do not modify them)."""
    return np.polynomial.legendre.leggauss(nodes)


def pulse_radial(r, steps: int, dt: float, discrete: bool = True, a: float = PULSE_A, c: float = PULSE_C,
                 rho: float = PULSE_RHO, nodes: int = 600, kmax: float = 40.0):
    """(sigma, v_r) at radii r after ``steps`` steps of length dt (time t = steps * dt)."""
    k, wq = _gauss_legendre(nodes)
    k = 0.5 * kmax * (k + 1.0)
    wq = 0.5 * kmax * wq
    S, U = _time_law(k, steps, dt, discrete, c)
    base = wq * np.exp(-k**2 / (4.0 * a)) / (2.0 * a) * k
    r = np.asarray(r, dtype=np.float64)
    flat = r.reshape(-1)
    sig = np.empty_like(flat)
    vr = np.empty_like(flat)
    for i0 in range(0, flat.size, 4096):
        kr = np.outer(flat[i0:i0 + 4096], k)
        sig[i0:i0 + 4096] = j0(kr) @ (base * S)
        vr[i0:i0 + 4096] = j1(kr) @ (base * U) / (rho * c)
    return sig.reshape(r.shape), vr.reshape(r.shape)


def pulse_solution(x, z, steps: int, dt: float, discrete: bool = True, **kw):
    """(sigma, v3) at points (x, z) (broadcast together); v3 = v_r z / r and 0 at the centre."""
    x, z = np.broadcast_arrays(np.asarray(x, dtype=np.float64), np.asarray(z, dtype=np.float64))
    r = np.sqrt(x**2 + z**2)
    sig, vr = pulse_radial(r, steps, dt, discrete, **kw)
    with np.errstate(invalid="ignore", divide="ignore"):
        v3 = np.where(r > 0, vr * z / np.where(r > 0, r, 1.0), 0.0)
    return sig, v3


def pulse_on_grid(n: int, steps: int, dt: float, discrete: bool = True, half_width: float = 5.0, **kw):
    """(sigma, v3) on the centred grid of Sec. 4.1: n + 1 points per axis (n even) on [-5, 5]^2, array axis 0
    = z.  The field is radial, so the integral is evaluated once per distinct radius h sqrt(i^2 + j^2)."""
    if n % 2:
        raise ValueError("the centred grid needs an even number of intervals")
    h = 2.0 * half_width / n
    m = n // 2
    d = np.arange(m + 1)
    s2 = d[:, None] ** 2 + d[None, :] ** 2
    uniq, inv = np.unique(s2, return_inverse=True)
    sig_u, vr_u = pulse_radial(h * np.sqrt(uniq.astype(np.float64)), steps, dt, discrete, **kw)
    off = np.abs(np.arange(n + 1) - m)
    sig = sig_u[inv].reshape(s2.shape)[off[:, None], off[None, :]]
    vr = vr_u[inv].reshape(s2.shape)[off[:, None], off[None, :]]
    zc = h * (np.arange(n + 1) - m)
    r = h * np.sqrt(off[:, None] ** 2 + off[None, :] ** 2).astype(np.float64)
    v3 = np.where(r > 0, vr * zc[:, None] / np.where(r > 0, r, 1.0), 0.0)
    return sig, v3
