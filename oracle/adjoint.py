"""Oracle, part 3: discrete adjoint of the LOSS time step and the gradient of a seismogram misfit (FP64).
TEST INFRASTRUCTURE ONLY.

The paper has no adjoint; this module differentiates the oracle's own time step (``wave.py``: the literal
Strang sequence "half A, full B, half A" of Sec. 3.3 with the ADE-PML exponential sub-flows) exactly.

With the model fixed, every sub-step is linear in the state u = (fields, PML memory variables), so the adjoint
of a sub-step is its transpose, written out term by term below:

* The PML sub-flow of one derivative term (``wave.PML.advance``) maps the memory value m and the derivative g
  to (m', X) with m' = E m + P g and X = Q m + R g, where, with beta = d/k + alpha and E = exp(-beta tau),
  P = -(d/k^2)(1 - E)/beta, Q = (E - 1)/beta and R = P/beta - tau alpha/(d + alpha k) inside the layers, and
  E = P = Q = 0, R = -tau outside (no memory, X = -tau g).  Its transpose maps (m', X) adjoints to
  m_adj = E m'_adj + Q X_adj and g_adj = P m'_adj + R X_adj.
* A derivative g = D f along one axis has the transpose f_adj += D^T g_adj (``wave.Operator.DT``).
* Products with the model (b, kappa, lambda, mu) are diagonal; the gradient with respect to a model
  coefficient c of a term "field += c * Z" is the sum over steps of Z (forward) times the field's adjoint.

Misfit: J = 1/2 sum_n sum_r (d_n,r - obs_n,r)^2 over the traces the oracle records after every step
(integer time levels).  The adjoint run goes backwards through the steps, injects the trace residuals, and
applies the transposed sub-steps in reverse order, re-running the forward sub-steps of each step from the
stored state to get the forward increments the gradient needs.  Gradients with respect to vp, vs, rho follow
from the chain rule through kappa = rho vp^2, lambda = rho (vp^2 - 2 vs^2), mu = rho vs^2, b = 1/rho.
The absorbing profile (its damping d0 uses the largest vp) and the time step are fixed numbers of the
discretisation, not functions of the model.
"""
from __future__ import annotations

from typing import Dict, Optional, Tuple

import numpy as np

from .wave import _SIG, PML, Simulation, component_axis, ricker

# ---------------------------------------------------------------------------------------------------------------
# PML sub-flow of one term as a linear map and its transpose.


def pml_coefficients(pml: Optional[PML], axis: int, tau: float, dim: int):
    """(E, P, Q, R) of the sub-flow over tau along array axis ``axis``, broadcastable to the grid."""
    if pml is None:
        return 0.0, 0.0, 0.0, -tau
    shape = [1] * dim
    shape[axis] = -1
    d, k, alpha = (x.reshape(shape) for x in pml.prof[axis])
    lay = d > 0
    beta = np.where(lay, d / k + alpha, 1.0)
    E = np.where(lay, np.exp(-beta * tau), 0.0)
    P = np.where(lay, -(d / k**2) * (1.0 - E) / beta, 0.0)
    Q = np.where(lay, (E - 1.0) / beta, 0.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        c3 = np.where(lay, tau * alpha / (d + alpha * k), 0.0)
    R = np.where(lay, P / beta - c3, -tau)
    return E, P, Q, R


def pml_transpose(coef, mem_adj: np.ndarray, x_adj: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Adjoint of (m', X) = (E m + P g, Q m + R g): returns (m_adj, g_adj)."""
    E, P, Q, R = coef
    return E * mem_adj + Q * x_adj, P * mem_adj + R * x_adj


# ---------------------------------------------------------------------------------------------------------------
# Forward sub-steps that also return their increments, and their transposes.  Acoustic.


def _acoustic_comps(dim):
    return (("v1", 1), ("v3", 3)) if dim == 2 else (("v1", 1), ("v2", 2), ("v3", 3))


def acoustic_A(st, mem, op, b, tau, pml):
    """v_k += b X_k with X_k the (PML) integral of -d_k sigma over tau; returns {k: X_k}."""
    X = {}
    for name, comp in _acoustic_comps(op.dim):
        g = op.Dc(st["sigma"], comp)
        X[name] = pml.advance(mem[f"psi{comp}"], g, component_axis(comp, op.dim), tau) if pml else -tau * g
        st[name] = st[name] + b * X[name]
    return X


def acoustic_A_T(lam, lmem, op, b, tau, pml):
    for name, comp in _acoustic_comps(op.dim):
        a = component_axis(comp, op.dim)
        x_adj = b * lam[name]
        key = f"psi{comp}"
        m_adj = lmem[key] if pml else np.zeros_like(x_adj)
        m_new, g_adj = pml_transpose(pml_coefficients(pml, a, tau, op.dim), m_adj, x_adj)
        if pml:
            lmem[key] = m_new
        lam["sigma"] = lam["sigma"] + op.DcT(g_adj, comp)


def acoustic_B(st, mem, op, kappa, dt, pml, src, t_half):
    """sigma += kappa sum_k X_k (X_k the integral of -d_k v_k over dt) + source; returns sum_k X_k."""
    inc = 0.0
    for name, comp in _acoustic_comps(op.dim):
        g = op.Dc(st[name], comp)
        inc = inc + (pml.advance(mem[f"phi{comp}"], g, component_axis(comp, op.dim), dt) if pml else -dt * g)
    st["sigma"] = st["sigma"] + kappa * inc
    if src is not None and "pressure" in src.kinds:
        src.add(st["sigma"], dt, t_half)
    return inc


def acoustic_B_T(lam, lmem, op, kappa, dt, pml):
    x_adj = kappa * lam["sigma"]
    for name, comp in _acoustic_comps(op.dim):
        a = component_axis(comp, op.dim)
        key = f"phi{comp}"
        m_adj = lmem[key] if pml else np.zeros_like(x_adj)
        m_new, g_adj = pml_transpose(pml_coefficients(pml, a, dt, op.dim), m_adj, x_adj)
        if pml:
            lmem[key] = m_new
        lam[name] = lam[name] + op.DcT(g_adj, comp)


# ---------------------------------------------------------------------------------------------------------------
# Elastic.  Y_ij = -X_ij is tau times the (stretched) derivative d_j of sigma_ij (sub-step A) or of v_i (B).


def _Y(op, f, comp, tau, pml, mem, key):
    g = op.Dc(f, comp)
    return -pml.advance(mem[key], g, component_axis(comp, op.dim), tau) if pml else tau * g


def elastic_A(st, mem, op, b, tau, pml, src, t):
    """v_i += b (sum_j Y_ij + tau f_i); returns {i: sum_j Y_ij} and the body-force increments {i: tau f_i} on the
    source block (empty without a body force)."""
    acc = {}
    for i in (1, 2, 3):
        acc[i] = sum(_Y(op, st[_SIG[(i, j)]], j, tau, pml, mem, f"psi_{i}{j}") for j in (1, 2, 3))
        st[f"v{i}"] = st[f"v{i}"] + b * acc[i]
    force = {}
    if src is not None:
        for i, kind in ((1, "force_x"), (2, "force_y"), (3, "force_z")):
            if kind in src.kinds:
                force[i] = tau * ricker(t, src.f0, src.t0) * src.profile
                st[f"v{i}"][src.block] += b[src.block] * force[i]
    return acc, force


def elastic_A_T(lam, lmem, op, b, tau, pml):
    for i in (1, 2, 3):
        y_adj = b * lam[f"v{i}"]
        for j in (1, 2, 3):
            a = component_axis(j, op.dim)
            key = f"psi_{i}{j}"
            m_adj = lmem[key] if pml else np.zeros_like(y_adj)
            m_new, g_adj = pml_transpose(pml_coefficients(pml, a, tau, op.dim), m_adj, -y_adj)
            if pml:
                lmem[key] = m_new
            s = _SIG[(i, j)]
            lam[s] = lam[s] + op.DcT(g_adj, j)


def elastic_B(st, mem, op, lam_, mu, dt, pml, src, t_half):
    """sigma += lambda tr(x) I + mu (x + x^T) with x_ij = Y_ij of v_i along x_j; returns x."""
    x = {(i, j): _Y(op, st[f"v{i}"], j, dt, pml, mem, f"phi_{i}{j}") for i in (1, 2, 3) for j in (1, 2, 3)}
    tr = x[1, 1] + x[2, 2] + x[3, 3]
    for i in (1, 2, 3):
        st[f"s{i}{i}"] = st[f"s{i}{i}"] + (lam_ * tr + 2.0 * mu * x[i, i])
    for (i, j) in ((1, 2), (1, 3), (2, 3)):
        st[f"s{i}{j}"] = st[f"s{i}{j}"] + mu * (x[i, j] + x[j, i])
    if src is not None:
        if "explosive" in src.kinds:
            for k in ("s11", "s22", "s33"):
                src.add(st[k], dt, t_half)
        if "shear_xz" in src.kinds:
            src.add(st["s13"], dt, t_half)
    return x


def elastic_B_T(lam, lmem, op, lam_, mu, dt, pml):
    sdiag = lam["s11"] + lam["s22"] + lam["s33"]
    for i in (1, 2, 3):
        for j in (1, 2, 3):
            if i == j:
                x_adj = lam_ * sdiag + 2.0 * mu * lam[f"s{i}{i}"]
            else:
                x_adj = mu * lam[_SIG[(i, j)]]
            a = component_axis(j, op.dim)
            key = f"phi_{i}{j}"
            m_adj = lmem[key] if pml else np.zeros_like(x_adj)
            m_new, g_adj = pml_transpose(pml_coefficients(pml, a, dt, op.dim), m_adj, -x_adj)
            if pml:
                lmem[key] = m_new
            lam[f"v{i}"] = lam[f"v{i}"] + op.DcT(g_adj, j)


# ---------------------------------------------------------------------------------------------------------------
# Misfit and gradient.


def _copy(d):
    return {k: np.array(v, copy=True) for k, v in d.items()}


def _inject(lam, resid_row, receivers):
    for f, idx in receivers.items():
        flat = lam[f].reshape(-1)
        np.add.at(flat, np.asarray(idx, dtype=np.int64), resid_row[f])


def misfit_gradient(w, d_obs: Dict[str, np.ndarray], steps: int, model=None):
    """Misfit J = 1/2 sum (traces - d_obs)^2 over ``steps`` steps of workload ``w`` from rest, and its gradient
    with respect to the model grids.  Returns (J, {"vp": g, "vs": g or None, "rho": g}, traces)."""
    sim = Simulation(w, model=model)
    vp, vs, rho = w.model() if model is None else model
    op, pml, src, dt = sim.op, sim.pml, sim.src, w.dt
    elastic = w.physics == "elastic"
    mem0 = sim.mem if sim.mem is not None else {}
    states = [(_copy(sim.state), _copy(mem0))]
    for _ in range(steps):
        sim.step(1)
        states.append((_copy(sim.state), _copy(sim.mem if sim.mem is not None else {})))
    traces = {f: sim.trace_array(f) for f in w.receivers}
    resid = {f: traces[f] - np.asarray(d_obs[f], dtype=np.float64)[:steps] for f in w.receivers}
    J = 0.5 * float(sum(np.sum(r**2) for r in resid.values()))

    lam = {k: np.zeros_like(v) for k, v in sim.state.items()}
    lmem = {k: np.zeros_like(v) for k, v in mem0.items()}
    shape = sim.state["v1"].shape
    if elastic:
        g_lam, g_mu, g_b = np.zeros(shape), np.zeros(shape), np.zeros(shape)
    else:
        g_kap, g_b = np.zeros(shape), np.zeros(shape)

    for n in reversed(range(steps)):
        _inject(lam, {f: resid[f][n] for f in w.receivers}, w.receivers)
        st, mem = _copy(states[n][0]), _copy(states[n][1])
        t_n = n * dt
        # forward sub-steps of step n from u_n, keeping the increments
        if elastic:
            acc1, f1 = elastic_A(st, mem, op, sim.b, 0.5 * dt, pml, src, t_n)
            x = elastic_B(st, mem, op, sim.lam, sim.mu, dt, pml, src, t_n + 0.5 * dt)
            acc2, f2 = elastic_A(st, mem, op, sim.b, 0.5 * dt, pml, src, t_n + dt)
            # transposes in reverse order, with the gradient terms
            g_b += sum(acc2[i] * lam[f"v{i}"] for i in (1, 2, 3))
            for i, fi in f2.items():
                g_b[src.block] += fi * lam[f"v{i}"][src.block]
            elastic_A_T(lam, lmem, op, sim.b, 0.5 * dt, pml)
            sdiag = lam["s11"] + lam["s22"] + lam["s33"]
            g_lam += (x[1, 1] + x[2, 2] + x[3, 3]) * sdiag
            g_mu += sum(2.0 * x[i, i] * lam[f"s{i}{i}"] for i in (1, 2, 3))
            g_mu += sum((x[i, j] + x[j, i]) * lam[f"s{i}{j}"] for (i, j) in ((1, 2), (1, 3), (2, 3)))
            elastic_B_T(lam, lmem, op, sim.lam, sim.mu, dt, pml)
            g_b += sum(acc1[i] * lam[f"v{i}"] for i in (1, 2, 3))
            for i, fi in f1.items():
                g_b[src.block] += fi * lam[f"v{i}"][src.block]
            elastic_A_T(lam, lmem, op, sim.b, 0.5 * dt, pml)
        else:
            X1 = acoustic_A(st, mem, op, sim.b, 0.5 * dt, pml)
            inc = acoustic_B(st, mem, op, sim.kappa, dt, pml, src, t_n + 0.5 * dt)
            X2 = acoustic_A(st, mem, op, sim.b, 0.5 * dt, pml)
            g_b += sum(X2[k] * lam[k] for k in X2)
            acoustic_A_T(lam, lmem, op, sim.b, 0.5 * dt, pml)
            g_kap += inc * lam["sigma"]
            acoustic_B_T(lam, lmem, op, sim.kappa, dt, pml)
            g_b += sum(X1[k] * lam[k] for k in X1)
            acoustic_A_T(lam, lmem, op, sim.b, 0.5 * dt, pml)

    if elastic:
        grads = {"vp": g_lam * 2.0 * rho * vp,
                 "vs": g_lam * (-4.0 * rho * vs) + g_mu * 2.0 * rho * vs,
                 "rho": g_lam * (vp**2 - 2.0 * vs**2) + g_mu * vs**2 - g_b / rho**2}
    else:
        grads = {"vp": g_kap * 2.0 * rho * vp, "vs": None, "rho": g_kap * vp**2 - g_b / rho**2}
    return J, grads, traces


def misfit(w, d_obs: Dict[str, np.ndarray], steps: int, model=None, c_max: Optional[float] = None) -> float:
    """J alone, from a forward oracle run (used for finite-difference checks)."""
    sim = Simulation(w, model=model)
    if c_max is not None and sim.pml is not None:
        sim.pml = PML(w.n, w.h, w.pml_width, w.pml_R, w.pml_kmax, w.f0, c_max)
    sim.step(steps)
    return 0.5 * float(sum(np.sum((sim.trace_array(f) - np.asarray(d_obs[f])[:steps]) ** 2) for f in w.receivers))


__all__ = ["pml_coefficients", "pml_transpose", "acoustic_A", "acoustic_A_T", "acoustic_B", "acoustic_B_T",
           "elastic_A", "elastic_A_T", "elastic_B", "elastic_B_T", "misfit_gradient", "misfit"]
