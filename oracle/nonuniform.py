"""Oracle, part 6: the 1-D LOSS derivative on a non-uniform grid (FP64).  TEST INFRASTRUCTURE ONLY.

The paper develops LOSS on a uniform grid and states that the construction carries over to non-uniform grids
through the scaling of the spline basis (Sec. 3, and the conclusion's future work).  This module takes the steps
of Sec. 3.1 and 3.2 with the uniform B-spline values replaced by those of cubic B-splines on the actual knots:

1. ``basis``: cubic B-splines B_k, k = -1..N+1, on the knots x_0 < ... < x_N extended by three mirrored knots at
   each end; B_k is supported on [x_{k-2}, x_{k+2}] (scipy's BSpline.basis_element evaluates them).  On a uniform
   grid B_k(x_k) = 2/3 and B_{k +- 1}(x_k) = 1/6, the (1, 4, 1)/6 rows of the paper.
2. ``global_matrix``: the (N+3) x (N+3) collocation matrix of Eq. (spline_cofficient_eq) with rows
   s''(x_0) = 0, s(x_i) = f_i, s''(x_N) = 0, where s = sum_k c_k B_k.
3. ``pmbc_weights``: phi_j = s'(x_{jM}) of the global spline as a weighted sum of the samples,
   W[j][m] = sum_k B_k'(x_{jM}) b_{k, jM+m} with b = A^{-1} (the data columns), truncated to |m| <= n_nb, one-sided
   at the two ends (Eqs. PMBC, PMBC_coeffcients and the end closures, with B_k' at the junction in place of
   +-1/(2h)).
4. ``local_coefficients``: per patch, the (M+3) x (M+3) system of Eq. (spline_cofficient_eq_piece) on the
   patch's knots, with Hermite rows s'(x_{lM}) = phi_l, s'(x_{(l+1)M}) = phi_{l+1}, solved with LAPACK gbsv.
5. ``derivative_1d``: s'(x_i) and s''(x_i) at every grid point from the local coefficients; at a junction the two
   patches' second derivatives are averaged (the first derivatives both equal phi).

With n_nb >= N every sum is complete and the result is the natural cubic spline through the samples (pinned
against scipy's CubicSpline in the tests); on a uniform grid it equals ``spline.derivative_1d``.

6. ``layer_profiles``: the absorbing layer of Sec. 3.3 on such an axis, its profiles taken on the physical distance
   into the layer (the paper defines them on a uniform grid, where distance and point count agree); used by
   ``simulation`` for the 2-D acoustic step with layers.
7. ``KnotSource``: the Gaussian source amplitude of Sec. 4.2 on such a grid, taken on the physical distance from
   the source knot with the width of the uniform grid (w = 2 h), on the same block of 25 knots per axis, and
   normalised with the knots' cell volumes (products of dual cell widths) so that it injects the same total as on
   the uniform grid.
"""
from __future__ import annotations

import functools
import math

import numpy as np
from scipy.interpolate import BSpline
from scipy.linalg import solve_banded


def extended_knots(x: np.ndarray) -> np.ndarray:
    """x_{-3}..x_{N+3}: the grid plus three knots mirrored about each end."""
    x = np.asarray(x, dtype=np.float64)
    left = x[0] - (x[1:4][::-1] - x[0])
    right = x[-1] + (x[-1] - x[-4:-1][::-1])
    return np.concatenate([left, x, right])


@functools.lru_cache(maxsize=256)
def _basis_cached(xt: tuple, at: tuple):
    xe = extended_knots(np.asarray(xt))
    pts = np.asarray(at)
    N = len(xt) - 1
    vals = np.zeros((3, len(pts), N + 3))  # [derivative order][point][k + 1]
    for k in range(-1, N + 2):
        b = BSpline.basis_element(xe[k + 1:k + 6], extrapolate=False)  # knots x_{k-2}..x_{k+2}
        for nu in range(3):
            f = b if nu == 0 else b.derivative(nu)
            v = f(pts)
            vals[nu, :, k + 1] = np.nan_to_num(v, nan=0.0)
    return vals


def basis(x: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """B_k^{(nu)}(pts) for nu = 0, 1, 2 and k = -1..N+1: array [3][len(pts)][N + 3]."""
    return _basis_cached(tuple(np.asarray(x, np.float64)), tuple(np.asarray(pts, np.float64)))


def global_matrix(x: np.ndarray) -> np.ndarray:
    """Dense A: row 0 s''(x_0) = 0, row i + 1 s(x_i) = f_i, row N + 2 s''(x_N) = 0 (unknown c_k in column k + 1)."""
    N = len(x) - 1
    B = basis(x, x)
    A = np.zeros((N + 3, N + 3))
    A[0] = B[2, 0]
    A[1:N + 2] = B[0]
    A[N + 2] = B[2, N]
    return A


@functools.lru_cache(maxsize=64)
def _weights_cached(xt: tuple, p: int, n_nb: int) -> np.ndarray:
    x = np.asarray(xt)
    N = len(x) - 1
    M = N // p
    A = global_matrix(x)
    Ainv = np.linalg.inv(A)
    b = Ainv[:, 1:N + 2]  # c = b f (the two natural-condition rows have zero right-hand side)
    B = basis(x, x)
    W = np.zeros((p + 1, 2 * n_nb + 1))
    for j in range(p + 1):
        c = j * M
        full = B[1, c] @ b  # s'(x_c) = sum_i full[i] f_i
        lo = 0 if j == 0 else -n_nb
        hi = 0 if j == p else n_nb
        for m in range(lo, hi + 1):
            if 0 <= c + m <= N:
                W[j, m + n_nb] = full[c + m]
    return W


def pmbc_weights(x: np.ndarray, p: int, n_nb: int) -> np.ndarray:
    """W[j, m + n_nb], j = 0..p, m = -n_nb..n_nb: phi_j = sum_m W[j, m + n_nb] f[jM + m]."""
    x = np.asarray(x, np.float64)
    if (len(x) - 1) % p:
        raise ValueError("N must be a multiple of p")
    return _weights_cached(tuple(x), int(p), int(n_nb))


def pmbc_phi(f: np.ndarray, x: np.ndarray, p: int, n_nb: int) -> np.ndarray:
    """phi for every junction of every line: f has shape (L, N + 1); returns (L, p + 1)."""
    W = pmbc_weights(x, p, n_nb)
    N = len(x) - 1
    M = N // p
    phi = np.zeros((f.shape[0], p + 1))
    for j in range(p + 1):
        for m in range(-n_nb, n_nb + 1):
            col = j * M + m
            if 0 <= col <= N and W[j, m + n_nb] != 0.0:
                phi[:, j] += W[j, m + n_nb] * f[:, col]
    return phi


def _local_band(xl: np.ndarray):
    """A_M^(l) of the patch with knots xl (M + 1 points) in LAPACK band storage (2 sub-, 2 super-diagonals), and
    the basis values at the patch's knots."""
    M = len(xl) - 1
    B = basis(xl, xl)
    A = np.zeros((M + 3, M + 3))
    A[0] = B[1, 0]
    A[1:M + 2] = B[0]
    A[M + 2] = B[1, M]
    ab = np.zeros((5, M + 3))
    for i in range(M + 3):
        for j in range(max(0, i - 2), min(M + 3, i + 3)):
            ab[2 + i - j, j] = A[i, j]
    return ab, B


def local_coefficients(f: np.ndarray, phi: np.ndarray, x: np.ndarray, p: int):
    """Local coefficients c^(l)_{-1..M+1} of every patch of every line: (L, p, M + 3), and the basis values of each
    patch (a list of [3][M + 1][M + 3] arrays)."""
    N = len(x) - 1
    M = N // p
    L = f.shape[0]
    c = np.empty((L, p, M + 3))
    bases = []
    for l in range(p):
        xl = x[l * M:l * M + M + 1]
        ab, B = _local_band(xl)
        rhs = np.empty((M + 3, L))
        rhs[0] = phi[:, l]
        rhs[1:M + 2] = f[:, l * M:l * M + M + 1].T
        rhs[M + 2] = phi[:, l + 1]
        c[:, l, :] = solve_banded((2, 2), ab, rhs).T
        bases.append(B)
    return c, bases


def derivative_1d(f: np.ndarray, x: np.ndarray, p: int, n_nb: int, second: bool = False):
    """LOSS derivative(s) on the non-uniform grid x of every line of f (shape (L, N + 1))."""
    f = np.asarray(f, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    N = len(x) - 1
    M = N // p
    phi = pmbc_phi(f, x, p, n_nb)
    c, bases = local_coefficients(f, phi, x, p)
    d1 = np.zeros((f.shape[0], N + 1))
    d2 = np.zeros((f.shape[0], N + 1))
    cnt = np.zeros(N + 1)
    for l in range(p):
        B = bases[l]
        d1[:, l * M:l * M + M + 1] += c[:, l, :] @ B[1].T
        d2[:, l * M:l * M + M + 1] += c[:, l, :] @ B[2].T
        cnt[l * M:l * M + M + 1] += 1.0
    d1 /= cnt
    d2 /= cnt
    return (d1, d2) if second else d1


def derivative(f: np.ndarray, axis: int, x: np.ndarray, p: int, n_nb: int, second: bool = False):
    """LOSS derivative of a multi-dimensional field along ``axis`` with knots x on that axis."""
    f = np.asarray(f, dtype=np.float64)
    fm = np.moveaxis(f, axis, -1)
    shp = fm.shape
    out = derivative_1d(fm.reshape(-1, shp[-1]), x, p, n_nb, second)
    if second:
        return tuple(np.moveaxis(o.reshape(shp), -1, axis) for o in out)
    return np.moveaxis(out.reshape(shp), -1, axis)


class Operator:
    """Per-axis LOSS first derivative on a tensor grid whose axes may carry their own knots (the interface of
    ``wave.Operator``): axis a uses the knots ``knots[a]`` when given, else the uniform spacing h[a]."""

    def __init__(self, n, p, h, n_nb, knots):
        from . import spline

        self._spline = spline
        self.n, self.p, self.h, self.n_nb = tuple(n), tuple(p), tuple(h), int(n_nb)
        self.dim = len(self.n)
        self.knots = {int(a): np.asarray(x, dtype=np.float64) for a, x in knots.items()}

    def D(self, f: np.ndarray, axis: int) -> np.ndarray:
        if axis in self.knots:
            return derivative(f, axis, self.knots[axis], self.p[axis], self.n_nb)
        return self._spline.derivative(f, axis, self.n[axis], self.p[axis], self.h[axis], self.n_nb)

    def Dc(self, f: np.ndarray, comp: int) -> np.ndarray:
        from .wave import component_axis

        return self.D(f, component_axis(comp, self.dim))


def layer_profiles(x: np.ndarray, width: int, R: float, k_max: float, f0: float, c_max: float):
    """The absorbing-layer profiles (d, k, alpha) of ``wave.PML`` along an axis with knots x, taken on the physical
    distance into each layer: the layer is the outer ``width`` intervals at each end, of thickness L = x_W - x_0
    (low end) or x_N - x_{N-W} (high end); a knot at distance s inside it has the normalised depth r = s / L, and
    d = d0 r^2 with d0 = -3 c_max log(R) / (2 L), k = 1 + (k_max - 1) r, alpha = pi f0 (1 - r).  On equally
    spaced knots these are the profiles of ``wave.PML``."""
    x = np.asarray(x, dtype=np.float64)
    N = len(x) - 1
    d = np.zeros(N + 1)
    r = np.zeros(N + 1)
    for lo, hi, inner in ((0, width, x[width]), (N - width, N, x[N - width])):
        L = abs(inner - (x[0] if lo == 0 else x[N]))
        d0 = -3.0 * c_max * math.log(R) / (2.0 * L)
        idx = np.arange(lo, hi + 1)
        rr = np.abs(x[idx] - inner) / L
        r[idx] = np.maximum(r[idx], rr)
        d[idx] = np.maximum(d[idx], d0 * rr**2)
    return d, 1.0 + (k_max - 1.0) * r, math.pi * f0 * (1.0 - r)


def cell_widths(c: np.ndarray) -> np.ndarray:
    """Dual cell width of every knot: half the distance between its neighbours (one-sided at the two ends)."""
    c = np.asarray(c, dtype=np.float64)
    v = np.empty_like(c)
    v[1:-1] = 0.5 * (c[2:] - c[:-2])
    v[0] = 0.5 * (c[1] - c[0])
    v[-1] = 0.5 * (c[-1] - c[-2])
    return v


class KnotSource:
    """Point source on a grid whose axes may carry knots: A(x) ~ exp(-|x - x0|^2 / (2 w^2)) with w = 2 h_a on axis a
    (h the nominal spacing) in physical distance from the source knot, on the knots within 12 of it per axis
    (clipped to the grid), normalised so that sum_i A_i V_i = amp with V_i the product of the knots' dual cell widths.
    On equally spaced knots away from the grid ends this is ``wave.Source``."""

    def __init__(self, index, kinds, f0, t0, amp, h, shape, knots):
        from .wave import SOURCE_RADIUS, SOURCE_WIDTH

        self.index = tuple(int(i) for i in index)
        self.kinds = tuple(kinds)
        self.f0, self.t0, self.amp = f0, t0, amp
        d = len(shape)
        lo = [max(0, self.index[a] - SOURCE_RADIUS) for a in range(d)]
        hi = [min(shape[a] - 1, self.index[a] + SOURCE_RADIUS) for a in range(d)]
        self.block = tuple(slice(lo[a], hi[a] + 1) for a in range(d))
        g, v = [], []
        for a in range(d):
            c = np.asarray(knots[a], dtype=np.float64) if a in knots else h[a] * np.arange(shape[a], dtype=np.float64)
            w = SOURCE_WIDTH * h[a]
            g.append(np.exp(-((c[lo[a]:hi[a] + 1] - c[self.index[a]]) ** 2) / (2.0 * w * w)))
            v.append(cell_widths(c)[lo[a]:hi[a] + 1])
        G = functools.reduce(np.multiply.outer, g)
        V = functools.reduce(np.multiply.outer, v)
        self.profile = amp * G / float(np.sum(G * V))

    def add(self, field: np.ndarray, scale: float, t: float):
        """field += scale * f_r(t) * A(x) on the profile block."""
        from .wave import ricker

        field[self.block] += scale * ricker(t, self.f0, self.t0) * self.profile


def simulation(w, knots, state=None):
    """A ``wave.Simulation`` of workload w whose derivatives use the given knots (dict axis -> coordinates).  The
    time stepping is the literal Strang sequence of ``wave``; an absorbing layer takes its profiles on the
    physical distance into the layer (``layer_profiles``) and a pressure source its amplitude on the physical
    distance from the source knot (``KnotSource``).  Other source kinds are not supported on such grids."""
    from .wave import Simulation

    if w.src_kinds and (w.dim != 2 or tuple(w.src_kinds) != ("pressure",)):
        raise ValueError("non-uniform grids: only a pressure source in 2-D")
    sim = Simulation(w, state=state)
    sim.op = Operator(w.n, w.p, w.h, w.n_nb, knots)
    if w.src_kinds:
        sim.src = KnotSource(w.src_index, w.src_kinds, w.f0, w.t0, w.amp, w.h, w.shape, knots)
    if sim.pml is not None:
        vp = w.model()[0]
        for a, x in knots.items():
            sim.pml.prof[int(a)] = layer_profiles(x, w.pml_width, w.pml_R, w.pml_kmax, w.f0, float(np.max(vp)))
    return sim
