"""Checks of the seeded input generators (synth/), which both the oracle and the CUDA path consume (CPU only).

Every workload must describe a grid the library accepts (n divisible by p, patch length at least the halo width,
layer at most half an axis), carry a model of the grid's shape with physical values (vp / vs >= 1.5 where there
is shear), keep its source and receivers on the grid, and step within the stability bound of the
leapfrog-type splitting.  The same seed must give the same arrays.
"""
import numpy as np
import pytest

from synth import (acoustic2d_layered, acoustic2d_small, batched_shots, elastic3d_double_layer,
                   elastic3d_heterogeneous, elastic3d_homogeneous, gaussian_pulse_2d, scaled)
from synth.workloads import DOUBLE_LAYER_DEEPER, DOUBLE_LAYER_UPPER


def _small_workloads():
    ws = [acoustic2d_small(n=64, p=2, n_nb=12),
          scaled(acoustic2d_layered(), n=128, p=2, steps=10),
          elastic3d_homogeneous(n=24, p=2, n_nb=8, pml_width=6),
          scaled(elastic3d_heterogeneous(), n=24, p=2, steps=10, n_nb=8, pml_width=6),
          elastic3d_double_layer(n=16, nz=32, p=2, pz=2, n_nb=8, pml_width=4),
          gaussian_pulse_2d(64, p=2, n_nb=20)[0],
          gaussian_pulse_2d(64, p=2, n_nb=20, pad=10)[0]]
    ws += batched_shots(n_shots=3, sizes=(256, 384), M=128, steps=10)
    return ws


@pytest.mark.parametrize("w", _small_workloads(), ids=lambda w: w.name)
def test_workload_is_a_valid_grid(w):
    assert len(w.n) == len(w.p) == len(w.h) == w.dim
    for n, p in zip(w.n, w.p):
        assert n % p == 0 and n // p >= w.n_nb, (n, p, w.n_nb)
        assert 2 * w.pml_width <= n
    vp, vs, rho = w.model()
    for a in (vp, rho) + ((vs,) if vs is not None else ()):
        assert a.shape == w.shape and np.isfinite(a).all() and (a > 0).all()
    if w.physics == "elastic":
        assert vs is not None and (vp / vs >= 1.5 - 1e-12).all()
    else:
        assert vs is None
    assert all(0 <= i <= n for i, n in zip(w.src_index, w.n))
    for idx in w.receivers.values():
        assert idx.dtype == np.int64 and (idx >= 0).all() and (idx < w.points).all()
    # dt within the stability bound 2 / (sqrt(3) sqrt(d)) of the LOSS operator
    cfl = w.dt * vp.max() / min(w.h)
    assert 0 < cfl <= 2.0 / (np.sqrt(3.0) * np.sqrt(w.dim)), cfl


def test_seeded_models_are_reproducible():
    a = scaled(acoustic2d_layered(), n=128, p=2, steps=10).model()[0]
    b = scaled(acoustic2d_layered(), n=128, p=2, steps=10).model()[0]
    assert np.array_equal(a, b)
    a = [w.model()[0] for w in batched_shots(n_shots=3, sizes=(256, 384), M=128, steps=10)]
    b = [w.model()[0] for w in batched_shots(n_shots=3, sizes=(256, 384), M=128, steps=10)]
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    d = scaled(acoustic2d_layered(seed=2003), n=128, p=2, steps=10).model()[0]
    e = scaled(acoustic2d_layered(), n=128, p=2, steps=10).model()[0]
    assert not np.array_equal(d, e)  # another seed, another perturbation


def test_double_layer_geometry():
    """Sec. 4.3: [-40 km, 40 km]^3, upper layer z >= 0, source at (0, 0, 10 km), v3 receivers on x = y = 0."""
    w = elastic3d_double_layer(n=16, nz=32, p=2, pz=2, n_nb=8, pml_width=4)
    vp, vs, rho = w.model()
    assert w.h == (2500.0, 5000.0, 5000.0)
    iz = np.arange(33)
    upper = iz >= 16  # z = -40 km + 2.5 km * iz >= 0
    for arr, (u, d) in zip((vp, vs, rho), zip(DOUBLE_LAYER_UPPER, DOUBLE_LAYER_DEEPER)):
        assert (arr[upper] == u).all() and (arr[~upper] == d).all()
    assert w.src_index == (20, 8, 8)  # 10 km above the centre
    line = w.receivers["v3"]
    zz, yy, xx = np.unravel_index(line, w.shape)
    assert (yy == 8).all() and (xx == 8).all() and np.array_equal(zz, iz)


def test_padded_pulse_is_the_pulse_on_a_larger_grid():
    w0, s0 = gaussian_pulse_2d(64, p=2)
    w1, s1 = gaussian_pulse_2d(64, p=2, pad=10)
    assert w1.n == (84, 84) and w1.h == w0.h
    assert np.array_equal(s1[10:75, 10:75], s0)
