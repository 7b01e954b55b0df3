"""Pins of the oracle's discrete adjoint (CPU): the PML sub-flow coefficients against the forward sub-flow,
dot-product tests of every transposed sub-step (<lam, L u> = <L^T lam, u> for random u, lam), and the misfit
gradient against central finite differences of the forward oracle for vp, vs and rho."""

import numpy as np
import pytest

from oracle import adjoint as adj
from oracle.wave import ELASTIC_FIELDS, PML, Operator
from synth import acoustic2d_gradient_case, elastic3d_gradient_case, mean_model, random_field


def _pml(n, h, width, c_max=3000.0, f0=30.0):
    return PML(n, h, width, 1e-6, 1.0, f0, c_max)


def test_pml_coefficients_reproduce_the_forward_flow():
    rng = np.random.default_rng(1)
    n, h = (20, 24), (10.0, 10.0)
    pml = _pml(n, h, 5)
    for axis in (0, 1):
        m = rng.standard_normal((21, 25))
        g = rng.standard_normal((21, 25))
        in_layer = np.broadcast_to(pml._bc(axis, 2)[0] > 0, m.shape)
        m = np.where(in_layer, m, 0.0)  # memory variables vanish outside the layers
        E, P, Q, R = adj.pml_coefficients(pml, axis, 0.003, 2)
        mem = m.copy()
        X = pml.advance(mem, g, axis, 0.003)
        np.testing.assert_allclose(mem, E * m + P * g, rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(X, Q * m + R * g, rtol=1e-13, atol=1e-15)


def _dot(a, b):
    return sum(float(np.sum(a[k] * b[k])) for k in a)


def _rand(keys, shape, rng, mask=None):
    out = {}
    for k in keys:
        v = rng.standard_normal(shape)
        out[k] = np.where(mask, v, 0.0) if mask is not None else v
    return out


def _layer_mask(pml, shape):
    m = np.zeros(shape, dtype=bool)
    for a in range(len(shape)):
        d = pml._bc(a, len(shape))[0]
        m |= np.broadcast_to(d > 0, shape)
    return m


@pytest.mark.parametrize("with_pml", [False, True])
def test_acoustic_substeps_dot_product(with_pml):
    rng = np.random.default_rng(2)
    n, p, h = (24, 20), (2, 2), (10.0, 8.0)
    op = Operator(n, p, h, 6)
    shape = (25, 21)
    pml = _pml(n, h, 5) if with_pml else None
    kappa = 2e9 * (1 + 0.1 * rng.random(shape))
    b = 1e-3 * (1 + 0.1 * rng.random(shape))
    mkeys = ("psi1", "psi3", "phi1", "phi3") if with_pml else ()
    mask = _layer_mask(pml, shape) if with_pml else None
    for which in ("A", "B"):
        u = _rand(("sigma", "v1", "v3"), shape, rng)
        um = _rand(mkeys, shape, rng, mask)
        lam = _rand(("sigma", "v1", "v3"), shape, rng)
        lm = _rand(mkeys, shape, rng, mask)
        st, mem = {k: v.copy() for k, v in u.items()}, {k: v.copy() for k, v in um.items()}
        if which == "A":
            adj.acoustic_A(st, mem, op, b, 0.0011, pml)
        else:
            adj.acoustic_B(st, mem, op, kappa, 0.0022, pml, None, 0.0)
        lhs = _dot(lam, st) + _dot(lm, mem)
        la, lma = {k: v.copy() for k, v in lam.items()}, {k: v.copy() for k, v in lm.items()}
        if which == "A":
            adj.acoustic_A_T(la, lma, op, b, 0.0011, pml)
        else:
            adj.acoustic_B_T(la, lma, op, kappa, 0.0022, pml)
        rhs = _dot(la, u) + _dot(lma, um)
        assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs)), (which, lhs, rhs)


@pytest.mark.parametrize("with_pml", [False, True])
def test_elastic_substeps_dot_product(with_pml):
    rng = np.random.default_rng(3)
    n, p, h = (10, 12, 8), (2, 2, 2), (10.0, 9.0, 11.0)
    op = Operator(n, p, h, 4)
    shape = (11, 13, 9)
    pml = _pml(n, h, 3) if with_pml else None
    lam_ = 2e9 * (1 + 0.1 * rng.random(shape))
    mu = 1e9 * (1 + 0.1 * rng.random(shape))
    b = 1e-3 * (1 + 0.1 * rng.random(shape))
    mkeys = tuple(f"{k}_{i}{j}" for k in ("psi", "phi") for i in (1, 2, 3) for j in (1, 2, 3)) if with_pml else ()
    mask = _layer_mask(pml, shape) if with_pml else None
    for which in ("A", "B"):
        u = _rand(ELASTIC_FIELDS, shape, rng)
        um = _rand(mkeys, shape, rng, mask)
        lam = _rand(ELASTIC_FIELDS, shape, rng)
        lm = _rand(mkeys, shape, rng, mask)
        st, mem = {k: v.copy() for k, v in u.items()}, {k: v.copy() for k, v in um.items()}
        if which == "A":
            adj.elastic_A(st, mem, op, b, 0.0011, pml, None, 0.0)
        else:
            adj.elastic_B(st, mem, op, lam_, mu, 0.0022, pml, None, 0.0)
        lhs = _dot(lam, st) + _dot(lm, mem)
        la, lma = {k: v.copy() for k, v in lam.items()}, {k: v.copy() for k, v in lm.items()}
        if which == "A":
            adj.elastic_A_T(la, lma, op, b, 0.0011, pml)
        else:
            adj.elastic_B_T(la, lma, op, lam_, mu, 0.0022, pml)
        rhs = _dot(la, u) + _dot(lma, um)
        assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs)), (which, lhs, rhs)


def _acoustic_case():
    return acoustic2d_gradient_case()


def _elastic_case():
    """Explosive source plus a body force, so that the force term of the b gradient is checked too."""
    return elastic3d_gradient_case(src_kinds=("explosive", "force_z"))


def _direction(shape, seed, ref):
    """Smooth random perturbation direction that vanishes where ref is largest (the absorbing profile uses the
    largest vp and is held fixed)."""
    d = random_field(shape, seed, 2.0)
    d.reshape(-1)[np.argmax(ref)] = 0.0
    return d


@pytest.mark.parametrize("case", ["acoustic", "elastic"])
def test_gradient_matches_finite_differences(case):
    w, (vp, vs, rho) = _acoustic_case() if case == "acoustic" else _elastic_case()
    steps = w.steps
    # observed data: the traces of a homogeneous model
    base = mean_model((vp, vs, rho))
    _, _, d_obs = adj.misfit_gradient(w, {f: np.zeros((steps, len(i))) for f, i in w.receivers.items()}, steps,
                                      model=base)
    J, grads, _ = adj.misfit_gradient(w, d_obs, steps, model=(vp, vs, rho))
    assert J > 0
    c_max = float(vp.max())
    params = ["vp", "rho"] + (["vs"] if vs is not None else [])
    for k, name in enumerate(params):
        ref = {"vp": vp, "vs": vs, "rho": rho}[name]
        d = _direction(w.shape, 100 + k, vp) * ref
        eps = 1e-4

        def model_at(s):
            m = {"vp": vp, "vs": vs, "rho": rho}
            m = dict(m)
            m[name] = ref + s * eps * d
            return (m["vp"], m["vs"], m["rho"])

        fd = (adj.misfit(w, d_obs, steps, model=model_at(1.0), c_max=c_max)
              - adj.misfit(w, d_obs, steps, model=model_at(-1.0), c_max=c_max)) / (2 * eps)
        an = float(np.sum(grads[name] * d))
        assert abs(fd - an) <= 2e-6 * abs(an), (name, fd, an)


def test_zero_residual_gives_zero_gradient():
    w, model = _acoustic_case()
    _, _, d_obs = adj.misfit_gradient(w, {f: np.zeros((10, len(i))) for f, i in w.receivers.items()}, 10, model=model)
    J, grads, _ = adj.misfit_gradient(w, d_obs, 10, model=model)
    assert J == 0.0
    assert not grads["vp"].any() and not grads["rho"].any()
