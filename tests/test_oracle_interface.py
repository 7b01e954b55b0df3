"""Pin of the oracle in layered media (CPU only): a plane P or S packet crossing the interface of the paper's
double-layer model (Sec. 4.3) at normal incidence splits as continuity of velocity and traction demands.  For a
packet in the upper layer (impedance Z1 = rho c) reaching the deeper one (Z2), the particle velocity reflects
with R = (Z1 - Z2) / (Z1 + Z2) and transmits with T = 2 Z1 / (Z1 + Z2); with the paper's layers both wave types
give R = -0.389 and T = 0.611.

The grid is a column of the double-layer workload: 257 points along z with the interface at the middle, 5 points
along x and y with every field uniform across them, and absorbing layers at both ends of the column.  This pins
how the model enters the stepper across a sharp contrast (rho and the moduli at each point, Eqs.
conservation_momentum and stress_strain_relation), which homogeneous tests cannot see.
"""
import dataclasses

import numpy as np
import pytest

from oracle.wave import Simulation, zero_state
from synth import DOUBLE_LAYER_DEEPER, DOUBLE_LAYER_UPPER, elastic3d_double_layer


@pytest.mark.parametrize("wave", ["P", "S"])
def test_normal_incidence_reflection_and_transmission(wave):
    nz, start, back, width = 256, 40, 30, 6.0
    w = elastic3d_double_layer(n=4, nz=nz, p=1, pz=1, precision="fp64")
    hz = w.h[0]
    w = dataclasses.replace(w, dt=0.4 * hz / DOUBLE_LAYER_DEEPER[0], src_kinds=(), receivers={})
    zi = nz // 2  # first point of the upper layer
    vp1, vs1, rho1 = DOUBLE_LAYER_UPPER
    vp2, vs2, rho2 = DOUBLE_LAYER_DEEPER
    c1, c2 = (vp1, vp2) if wave == "P" else (vs1, vs2)
    Z1, Z2 = rho1 * c1, rho2 * c2
    # a packet in the upper layer travelling towards -z (the deeper layer): sigma = +Z v for a wave moving to -z
    z = np.arange(nz + 1)
    g = np.exp(-(((z - (zi + start)) / width) ** 2))[:, None, None] * np.ones(w.shape)
    st = zero_state("elastic", w.shape)
    if wave == "P":  # plane strain: sigma11 = sigma22 = lambda / (lambda + 2 mu) sigma33
        lam1 = rho1 * (vp1**2 - 2 * vs1**2)
        st.update(v3=g.copy(), s33=Z1 * g, s11=(lam1 / c1) * g, s22=(lam1 / c1) * g)
        comp = "v3"
    else:
        st.update(v1=g.copy(), s13=Z1 * g)
        comp = "v1"
    sim = Simulation(w, state=st)
    # until the reflected packet is `back` cells above the interface
    sim.step(int(round((start + back) * hz / c1 / w.dt)), record=False)
    v = sim.state[comp][:, 2, 2]
    up, down = v[zi:], v[:zi]
    R = up[np.argmax(np.abs(up))]
    T = down[np.argmax(np.abs(down))]
    assert abs(R - (Z1 - Z2) / (Z1 + Z2)) < 2e-3, (R, (Z1 - Z2) / (Z1 + Z2))
    assert abs(T - 2 * Z1 / (Z1 + Z2)) < 6e-3, (T, 2 * Z1 / (Z1 + Z2))
    # the reflected packet travels back at c1 and the transmitted one at c2 (2 c1 here)
    assert abs(zi + np.argmax(np.abs(up)) - (zi + back)) <= 2
    assert abs(np.argmax(np.abs(down)) - (zi - back * c2 / c1)) <= 2
