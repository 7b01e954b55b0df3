"""Oracle, part 2: velocity-stress time stepping with the LOSS derivative (FP64).  TEST INFRASTRUCTURE ONLY.

Physics (Sec. 2):

* Acoustic (Eq. acoustic_wave): dv_k/dt = -b d_k sigma,  dsigma/dt = -kappa sum_k d_k v_k,
  with b = 1/rho and kappa = rho c_P^2; sigma is the pressure.
* Elastic (Eqs. conservation_momentum, defintion_strain, stress_strain_relation and the 6x6 matrix):
  rho dv_i/dt = sum_j d_j sigma_ij + f_i,  dsigma_ij/dt = lambda (div v) delta_ij + mu (d_j v_i + d_i v_j),
  with lambda = rho (c_P^2 - 2 c_S^2) and mu = rho c_S^2.

Time integration (Sec. 3.3, the Strang splitting at the end of the section, without PML): subsystem A
advances the velocities with the stresses frozen, subsystem B advances the stresses with the velocities
frozen; one step is half a step of A, a full step of B, half a step of A.  Without PML each sub-flow is
exact as a forward Euler step because its right-hand side does not depend on the advanced fields.

Sources (reading of the garbled Ricker formula in Sec. 4.2): f_r(t) = (1 - 2 (pi f0 (t - t0))^2)
exp(-(pi f0 (t - t0))^2), with the Gaussian spatial amplitude of Sec. 4.2 (class Source).  Stress sources
("pressure", "explosive", "shear_xz") act in B and are evaluated at t_n + dt/2; body forces ("force_x",
"force_y", "force_z": f_1, f_2, f_3 of Eq. conservation_momentum, each A(x) f_r(t)) act in each half of A, at
t_n and at t_{n+1}.

Absorbing layer (Sec. 3.3): an ADE-PML in the outer points of every axis with the exponential Strang
splitting of the paper (class PML).  Without it the natural-spline ends impose no physical boundary condition
and zero-frequency polynomial modes (uniform pressure fed by linear velocity fields) grow like a power of t
from any rounding perturbation.

Axes: array axis 0 is z, then y (3-D), then x.  v1 is along x, v2 along y, v3 along z.
"""
from __future__ import annotations

import math
from typing import Dict, Optional

import numpy as np

from . import spline

ACOUSTIC_FIELDS_2D = ("sigma", "v1", "v3")
ACOUSTIC_FIELDS_3D = ("sigma", "v1", "v2", "v3")
ELASTIC_FIELDS = ("v1", "v2", "v3", "s11", "s22", "s33", "s12", "s13", "s23")


def component_axis(comp: int, dim: int) -> int:
    """Array axis of the paper's coordinate x_comp (1 = x, 2 = y, 3 = z)."""
    if comp == 1:
        return dim - 1
    if comp == 3:
        return 0
    if comp == 2 and dim == 3:
        return 1
    raise ValueError("no such component")


class Operator:
    """Per-axis LOSS first derivative on a tensor grid (axis a has n[a] intervals in p[a] patches)."""

    def __init__(self, n, p, h, n_nb):
        self.n, self.p, self.h, self.n_nb = tuple(n), tuple(p), tuple(h), int(n_nb)
        self.dim = len(self.n)

    def D(self, f: np.ndarray, axis: int) -> np.ndarray:
        return spline.derivative(f, axis, self.n[axis], self.p[axis], self.h[axis], self.n_nb)

    def Dc(self, f: np.ndarray, comp: int) -> np.ndarray:
        """Derivative with respect to the paper's coordinate x_comp."""
        return self.D(f, component_axis(comp, self.dim))

    def DT(self, g: np.ndarray, axis: int) -> np.ndarray:
        """Transpose of D along ``axis`` through the explicit 1-D matrix (adjoint use only)."""
        Dm = spline.derivative_matrix(self.n[axis], self.p[axis], self.h[axis], self.n_nb)
        gm = np.moveaxis(g, axis, -1)
        return np.moveaxis(gm @ Dm, -1, axis)  # (D^T y)_j = sum_i D_ij y_i

    def DcT(self, g: np.ndarray, comp: int) -> np.ndarray:
        return self.DT(g, component_axis(comp, self.dim))


def ricker(t: float, f0: float, t0: float) -> float:
    a = (math.pi * f0 * (t - t0)) ** 2
    return (1.0 - 2.0 * a) * math.exp(-a)


def acoustic_moduli(vp, rho):
    """kappa = rho c_P^2 and b = 1 / rho (Sec. 2)."""
    return rho * vp**2, 1.0 / rho


def elastic_moduli(vp, vs, rho):
    """lambda = rho (c_P^2 - 2 c_S^2), mu = rho c_S^2, b = 1 / rho (Eq. stress_strain_relation)."""
    return rho * (vp**2 - 2.0 * vs**2), rho * vs**2, 1.0 / rho


SOURCE_RADIUS = 12  # cells per axis kept in the truncated Gaussian profile
SOURCE_WIDTH = 2.0  # standard deviation of the profile in cells


class Source:
    """Point-like source with the Gaussian spatial amplitude of Sec. 4.2, A(x) ~ exp(-|x - x0|^2 / (2 w^2)),
    w = 2 h per axis, truncated to |offset| <= 12 cells and clipped to the grid, normalised so that
    sum_i A_i h^d = 1 on the grid.  A smooth profile keeps grid-scale (non-propagating) modes out of the
    wavefield; a single-node injection excites them and they grow at the natural-spline ends."""

    def __init__(self, index, kinds, f0, t0, amp, h, shape):
        self.index = tuple(int(i) for i in index)
        self.kinds = tuple(kinds)
        self.f0, self.t0, self.amp = f0, t0, amp
        d = len(shape)
        lo = [max(0, self.index[a] - SOURCE_RADIUS) for a in range(d)]
        hi = [min(shape[a] - 1, self.index[a] + SOURCE_RADIUS) for a in range(d)]
        self.block = tuple(slice(lo[a], hi[a] + 1) for a in range(d))
        offs = np.meshgrid(*[np.arange(lo[a], hi[a] + 1) - self.index[a] for a in range(d)], indexing="ij")
        r2 = sum(o.astype(np.float64) ** 2 for o in offs)
        g = np.exp(-r2 / (2.0 * SOURCE_WIDTH**2))
        self.profile = amp * g / (g.sum() * float(np.prod(h)))

    def add(self, field: np.ndarray, scale: float, t: float):
        """field += scale * f_r(t) * A(x) on the profile block."""
        field[self.block] += scale * ricker(t, self.f0, self.t0) * self.profile


class PML:
    """ADE-PML of Sec. 3.3 in the outer ``width`` points of every axis.

    Profiles (Sec. 3.3 with m = p = 1): at normalised depth r in (0, 1] into a layer,
        d = d0 r^2,  k = 1 + (k_max - 1) r,  alpha = alpha_max (1 - r),
        d0 = -3 c_max log(R) / (2 L),  alpha_max = pi f0,  L = width * h.
    Memory variables Psi_a (one per velocity derivative axis) and Phi_a (one per stress derivative axis) obey
    dPsi/dt = -(d/k + alpha) Psi - (d/k^2) d_a(field) (Eq. ADE_PML_1).  With the other subsystem frozen each
    sub-flow is integrated exactly (Eq. Euler_approximation and the exponential splitting that follows):
        Psi(t + tau) = E Psi(t) - (d/k^2) (1 - E) / beta * g,         E = exp(-beta tau), beta = d/k + alpha,
        field += sign * (coefficient) * [ (1/beta) (Psi(t+tau) - Psi(t)) - tau alpha / (d + alpha k) g ],
    which reduces to field += sign * (coefficient) * (-tau g) outside the layers (d = 0, k = 1)."""

    def __init__(self, n, h, width, R, k_max, f0, c_max):
        self.width = int(width)
        self.prof = []
        for a in range(len(n)):
            i = np.arange(n[a] + 1, dtype=np.float64)
            if self.width > 0:
                r = np.maximum(np.maximum(self.width - i, i - (n[a] - self.width)), 0.0) / self.width
                L = self.width * h[a]
                d0 = -3.0 * c_max * math.log(R) / (2.0 * L)
            else:
                r = np.zeros(n[a] + 1)
                d0 = 0.0
            d = d0 * r**2
            k = 1.0 + (k_max - 1.0) * r
            alpha = math.pi * f0 * (1.0 - r)
            self.prof.append((d, k, alpha))

    def _bc(self, a, dim):
        shape = [1] * dim
        shape[a] = -1
        d, k, alpha = self.prof[a]
        return d.reshape(shape), k.reshape(shape), alpha.reshape(shape)

    def advance(self, mem: np.ndarray, g: np.ndarray, a: int, tau: float):
        """Advance memory variable ``mem`` along axis ``a`` over ``tau`` with frozen derivative ``g``; return the
        effective increment factor X such that field += sign * coefficient * X."""
        d, k, alpha = self._bc(a, g.ndim)
        in_layer = np.broadcast_to(d > 0, g.shape)
        beta = d / k + alpha
        with np.errstate(divide="ignore", invalid="ignore"):
            E = np.exp(-beta * tau)
            new = np.where(in_layer, E * mem - (d / k**2) * (1.0 - E) / beta * g, 0.0)
            X = np.where(in_layer, (new - mem) / beta - tau * alpha / (d + alpha * k) * g, -tau * g)
        mem[...] = new
        return X


def zero_state(physics: str, shape) -> Dict[str, np.ndarray]:
    names = ELASTIC_FIELDS if physics == "elastic" else (ACOUSTIC_FIELDS_2D if len(shape) == 2 else ACOUSTIC_FIELDS_3D)
    return {k: np.zeros(shape) for k in names}


def _velocity_names(dim):
    return (("v1", 1), ("v3", 3)) if dim == 2 else (("v1", 1), ("v2", 2), ("v3", 3))


def acoustic_half_A(st, op, b, tau, pml: Optional[PML] = None, mem=None):
    """Subsystem A for a time ``tau``: v_k <- v_k - tau * b * d_k sigma (Eq. acoustic_wave); with a PML the
    exact exponential flow of Eq. ADE_PML_A."""
    for name, comp in _velocity_names(op.dim):
        g = op.Dc(st["sigma"], comp)
        if pml is None:
            st[name] = st[name] - tau * b * g
        else:
            a = component_axis(comp, op.dim)
            st[name] = st[name] + b * pml.advance(mem[f"psi{comp}"], g, a, tau)


def acoustic_B(st, op, kappa, dt, src: Optional[Source], t_half, pml: Optional[PML] = None, mem=None):
    """Subsystem B for a time ``dt``: sigma <- sigma - dt * kappa * div v, plus the pressure source; with a PML
    the exact exponential flow of Eq. ADE_PML_B."""
    if pml is None:
        div = sum(op.Dc(st[name], comp) for name, comp in _velocity_names(op.dim))
        st["sigma"] = st["sigma"] - dt * kappa * div
    else:
        inc = 0.0
        for name, comp in _velocity_names(op.dim):
            a = component_axis(comp, op.dim)
            inc = inc + pml.advance(mem[f"phi{comp}"], op.Dc(st[name], comp), a, dt)
        st["sigma"] = st["sigma"] + kappa * inc
    if src is not None and "pressure" in src.kinds:
        src.add(st["sigma"], dt, t_half)


def acoustic_step(st, op, kappa, b, dt, t_n, src=None, pml=None, mem=None):
    acoustic_half_A(st, op, b, 0.5 * dt, pml, mem)
    acoustic_B(st, op, kappa, dt, src, t_n + 0.5 * dt, pml, mem)
    acoustic_half_A(st, op, b, 0.5 * dt, pml, mem)


_SIG = {(1, 1): "s11", (2, 2): "s22", (3, 3): "s33", (1, 2): "s12", (2, 1): "s12", (1, 3): "s13",
        (3, 1): "s13", (2, 3): "s23", (3, 2): "s23"}


def _tau_deriv(op, f, comp, tau, pml: Optional[PML], mem, key):
    """tau times the (PML-stretched) derivative of f along x_comp, integrated exactly over tau: tau d f outside
    the layers, and -PML.advance(...) (the exact integral of (1/k) d f + Psi) inside."""
    g = op.Dc(f, comp)
    if pml is None:
        return tau * g
    return -pml.advance(mem[key], g, component_axis(comp, op.dim), tau)


def elastic_half_A(st, op, b, tau, src: Optional[Source], t, pml: Optional[PML] = None, mem=None):
    """Subsystem A: v_i <- v_i + tau * b * (sum_j d_j sigma_ij + f_i)."""
    for i in (1, 2, 3):
        acc = sum(_tau_deriv(op, st[_SIG[(i, j)]], j, tau, pml, mem, f"psi_{i}{j}") for j in (1, 2, 3))
        st[f"v{i}"] = st[f"v{i}"] + b * acc
    if src is not None:
        for i, kind in ((1, "force_x"), (2, "force_y"), (3, "force_z")):
            if kind in src.kinds:
                st[f"v{i}"][src.block] += tau * b[src.block] * ricker(t, src.f0, src.t0) * src.profile


def elastic_B(st, op, lam, mu, dt, src: Optional[Source], t_half, pml: Optional[PML] = None, mem=None):
    """Subsystem B: sigma_ij <- sigma_ij + dt * (lambda tr(e) delta_ij + 2 mu e_ij), e_ij = (d_j v_i + d_i v_j)/2."""
    # x[i, j] = dt * d_j v_i (PML-stretched in the layers)
    x = {(i, j): _tau_deriv(op, st[f"v{i}"], j, dt, pml, mem, f"phi_{i}{j}") for i in (1, 2, 3) for j in (1, 2, 3)}
    tr = x[1, 1] + x[2, 2] + x[3, 3]
    for i in (1, 2, 3):
        st[f"s{i}{i}"] = st[f"s{i}{i}"] + (lam * tr + 2.0 * mu * x[i, i])
    for (i, j) in ((1, 2), (1, 3), (2, 3)):
        st[f"s{i}{j}"] = st[f"s{i}{j}"] + mu * (x[i, j] + x[j, i])
    if src is not None:
        if "explosive" in src.kinds:
            for k in ("s11", "s22", "s33"):
                src.add(st[k], dt, t_half)
        if "shear_xz" in src.kinds:
            src.add(st["s13"], dt, t_half)


def elastic_step(st, op, lam, mu, b, dt, t_n, src=None, pml=None, mem=None):
    elastic_half_A(st, op, b, 0.5 * dt, src, t_n, pml, mem)
    elastic_B(st, op, lam, mu, dt, src, t_n + 0.5 * dt, pml, mem)
    elastic_half_A(st, op, b, 0.5 * dt, src, t_n + dt, pml, mem)


def energy(st, physics, rho, moduli, h) -> float:
    """Discrete energy 1/2 sum (rho |v|^2 + sigma : C^{-1} : sigma) h^d."""
    cell = float(np.prod(h))
    ke = sum(rho * st[k] ** 2 for k in st if k.startswith("v"))
    if physics == "acoustic":
        kappa = moduli[0]
        pe = st["sigma"] ** 2 / kappa
    else:
        lam, mu = moduli
        s11, s22, s33 = st["s11"], st["s22"], st["s33"]
        tr = s11 + s22 + s33
        # C^{-1}: e = (sigma - lam/(3 lam + 2 mu) tr(sigma) I) / (2 mu)
        dev = s11**2 + s22**2 + s33**2 + 2.0 * (st["s12"] ** 2 + st["s13"] ** 2 + st["s23"] ** 2)
        pe = (dev - lam / (3.0 * lam + 2.0 * mu) * tr**2) / (2.0 * mu)
    return 0.5 * float(np.sum(ke + pe)) * cell


class Simulation:
    """A workload (synth.Workload) advanced by the oracle."""

    def __init__(self, w, state: Optional[Dict[str, np.ndarray]] = None, model=None):
        self.w = w
        self.op = Operator(w.n, w.p, w.h, w.n_nb)
        vp, vs, rho = w.model() if model is None else model
        self.rho = rho
        if w.physics == "acoustic":
            self.kappa, self.b = acoustic_moduli(vp, rho)
            self.moduli = (self.kappa,)
        else:
            self.lam, self.mu, self.b = elastic_moduli(vp, vs, rho)
            self.moduli = (self.lam, self.mu)
        self.src = Source(w.src_index, w.src_kinds, w.f0, w.t0, w.amp, w.h, w.shape) if w.src_kinds else None
        self.pml, self.mem = None, None
        if getattr(w, "pml_width", 0) > 0:
            self.pml = PML(w.n, w.h, w.pml_width, w.pml_R, w.pml_kmax, w.f0, float(np.max(vp)))
            if w.physics == "acoustic":
                comps = (1, 3) if w.dim == 2 else (1, 2, 3)
                self.mem = {f"{k}{c}": np.zeros(w.shape) for k in ("psi", "phi") for c in comps}
            else:
                self.mem = {f"{k}_{i}{j}": np.zeros(w.shape) for k in ("psi", "phi") for i in (1, 2, 3)
                            for j in (1, 2, 3)}
        self.state = zero_state(w.physics, w.shape) if state is None else {k: np.array(v, dtype=np.float64) for k, v in state.items()}
        self.step_index = 0
        self.traces = {k: [] for k in w.receivers}

    def step(self, count: int = 1, record: bool = True):
        w = self.w
        for _ in range(count):
            t_n = self.step_index * w.dt
            if w.physics == "acoustic":
                acoustic_step(self.state, self.op, self.kappa, self.b, w.dt, t_n, self.src, self.pml, self.mem)
            else:
                elastic_step(self.state, self.op, self.lam, self.mu, self.b, w.dt, t_n, self.src, self.pml, self.mem)
            self.step_index += 1
            if record:
                for k, idx in w.receivers.items():
                    self.traces[k].append(self.state[k].reshape(-1)[idx].copy())
        return self

    def trace_array(self, field: str) -> np.ndarray:
        return np.asarray(self.traces[field])

    def energy(self) -> float:
        return energy(self.state, self.w.physics, self.rho, self.moduli, self.w.h)
