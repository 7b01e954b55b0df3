"""Workload descriptions with seeded synthetic models (input generation only).

Index conventions used everywhere in this repository:

* A grid axis has ``n`` intervals and ``n + 1`` points; axis 0 is z (slowest), then y (3-D only), then x
  (fastest, contiguous).
* Each axis is cut into ``p`` patches of ``M = n / p`` intervals (the paper's Sec. 3.2); junction points
  are stored once.
* Velocity components: ``v1`` is along x, ``v2`` along y, ``v3`` along z (the paper's x_1, x_2, x_3).

The five standard workloads follow the paper's experiments in shape (2-D acoustic and 3-D elastic
velocity-stress propagation with a Ricker point source, Sec. 4) at the sizes of the benchmark table:
a small 2-D parity case, a 2-D layered model with a Gaussian-correlated perturbation, a 3-D homogeneous
elastic model, a 3-D smooth heterogeneous elastic model for the adjoint, and a batch of 2-D shots with
uneven grid sizes.  Every random draw is seeded.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Dict, Optional, Tuple

import numpy as np
from scipy.ndimage import gaussian_filter


@dataclasses.dataclass
class Workload:
    name: str
    dim: int
    physics: str  # "acoustic" or "elastic"
    n: Tuple[int, ...]  # intervals per axis, axis 0 = z
    p: Tuple[int, ...]  # patches per axis
    h: Tuple[float, ...]  # spacing per axis [m]
    n_nb: int  # PMBC halo width
    dt: float  # time step [s]
    steps: int
    model_fn: Callable[[], Tuple[np.ndarray, Optional[np.ndarray], np.ndarray]]
    src_index: Tuple[int, ...]
    src_kinds: Tuple[str, ...]  # subset of "pressure", "explosive", "shear_xz", "force_x", "force_y", "force_z"
    f0: float  # Ricker peak frequency [Hz]
    t0: float  # Ricker delay [s]
    amp: float = 1.0
    receivers: Dict[str, np.ndarray] = dataclasses.field(default_factory=dict)  # field -> flat indices
    precision: str = "fp64"
    checkpoint_every: int = 0
    seed: int = 0
    pml_width: int = 0  # points of the absorbing ADE-PML layer on each side of every axis (0 = none)
    pml_R: float = 1e-6  # theoretical reflection coefficient
    pml_kmax: float = 1.0

    @property
    def shape(self) -> Tuple[int, ...]:
        return tuple(int(k) + 1 for k in self.n)

    @property
    def points(self) -> int:
        return int(np.prod(self.shape))

    def model(self):
        """(vp, vs, rho) as float64 arrays of the grid shape; vs is None for acoustic workloads."""
        return self.model_fn()


def random_field(shape, seed: int, corr_cells: float) -> np.ndarray:
    """White noise (seeded) smoothed by a Gaussian of std ``corr_cells`` cells, renormalised to zero mean
    and unit standard deviation."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(shape)
    if corr_cells > 0:
        g = gaussian_filter(g, sigma=corr_cells, mode="reflect")
    g = g - g.mean()
    return g / g.std()


def _cfl_dt(h: float, vmax: float, cfl: float = 0.4) -> float:
    return cfl * h / vmax


def _top_row_receivers(shape) -> np.ndarray:
    """Flat indices of every point on the plane z = 0 (axis-0 index 0)."""
    return np.arange(int(np.prod(shape[1:])), dtype=np.int64)


def _row_receivers(shape, z: int) -> np.ndarray:
    """Flat indices of every point on the plane of axis-0 index z."""
    plane = int(np.prod(shape[1:]))
    return z * plane + np.arange(plane, dtype=np.int64)


def acoustic2d_small(n: int = 128, p: int = 2, steps: int = 300, n_nb: int = 12, pml_width: int = 20) -> Workload:
    """2-D acoustic, constant v = 2000 m/s, rho = 1000 kg/m^3, h = 10 m, Ricker 15 Hz at the centre, FP64, with
    an absorbing ADE-PML layer of ``pml_width`` points on every side."""
    shape = (n + 1, n + 1)
    h = 10.0

    def model():
        return np.full(shape, 2000.0), None, np.full(shape, 1000.0)

    f0 = 15.0
    return Workload(
        name=f"acoustic2d_{n}_p{p}", dim=2, physics="acoustic", n=(n, n), p=(p, p), h=(h, h), n_nb=n_nb,
        dt=_cfl_dt(h, 2000.0), steps=steps, model_fn=model, src_index=(n // 2, n // 2),
        src_kinds=("pressure",), f0=f0, t0=1.2 / f0,
        receivers={"sigma": _top_row_receivers(shape)}, precision="fp64", pml_width=pml_width)


def _layered_velocity_2d(n: int, seed: int) -> np.ndarray:
    """Three layers (1500 / 2500 / 3500 m/s by depth thirds) times (1 + 0.05 g), g Gaussian-correlated with
    a 50 m correlation length (5 cells at h = 10 m)."""
    shape = (n + 1, n + 1)
    z = np.arange(n + 1)[:, None] * np.ones((1, n + 1))
    v = np.where(z < n / 3, 1500.0, np.where(z < 2 * n / 3, 2500.0, 3500.0))
    g = random_field(shape, seed, corr_cells=5.0)
    return v * (1.0 + 0.05 * g)


def acoustic2d_layered(n: int = 2048, p: int = 8, steps: int = 2000, n_nb: int = 20,
                       precision: str = "fp32_kahan", seed: int = 2002, pml_width: int = 40) -> Workload:
    """2-D acoustic three-layer model with a 5 % Gaussian-correlated perturbation, Ricker 20 Hz at the centre."""
    shape = (n + 1, n + 1)
    h = 10.0
    vp = _layered_velocity_2d(n, seed)
    vmax = float(vp.max())

    def model():
        return vp.copy(), None, np.full(shape, 1000.0)

    f0 = 20.0
    return Workload(
        name=f"acoustic2d_layered_{n}_p{p}", dim=2, physics="acoustic", n=(n, n), p=(p, p), h=(h, h),
        n_nb=n_nb, dt=_cfl_dt(h, vmax), steps=steps, model_fn=model, src_index=(n // 2, n // 2),
        src_kinds=("pressure",), f0=f0, t0=1.2 / f0, receivers={"sigma": _top_row_receivers(shape)},
        precision=precision, seed=seed, pml_width=pml_width)


def elastic3d_homogeneous(n: int = 256, p: int = 4, steps: int = 1000, n_nb: int = 20,
                          precision: str = "fp32_kahan", pml_width: int = 20) -> Workload:
    """3-D isotropic elastic, vp = 3000, vs = 1730, rho = 2000, explosive plus shear source at the centre,
    15 Hz Ricker, receivers v1, v2, v3 on the top plane of the physical domain (z = pml_width; on the outermost
    plane of the absorbing layer the field is an attenuated remnant carrying undamped rounding modes)."""
    shape = (n + 1,) * 3
    h = 10.0

    def model():
        return np.full(shape, 3000.0), np.full(shape, 1730.0), np.full(shape, 2000.0)

    f0 = 15.0
    top = _row_receivers(shape, pml_width)
    return Workload(
        name=f"elastic3d_homog_{n}_p{p}", dim=3, physics="elastic", n=(n,) * 3, p=(p,) * 3, h=(h,) * 3,
        n_nb=n_nb, dt=_cfl_dt(h, 3000.0), steps=steps, model_fn=model, src_index=(n // 2,) * 3,
        src_kinds=("explosive", "shear_xz"), f0=f0, t0=1.2 / f0,
        receivers={"v1": top, "v2": top, "v3": top}, precision=precision, pml_width=pml_width)


def elastic3d_heterogeneous(n: int = 192, p: int = 4, steps: int = 1500, n_nb: int = 20,
                            precision: str = "fp32_kahan", seeds=(4001, 4002, 4003),
                            true_model: bool = True, pml_width: int = 20) -> Workload:
    """3-D elastic with smooth random vp/vs/rho (5 %, 100 m correlation length, clipped so vp/vs >= 1.5).
    ``true_model=False`` gives the homogeneous starting model of the inversion.  The v3 receivers cover the plane
    z = pml_width, the top of the physical domain: the adjoint run injects its sources there, and on the
    outermost plane of an absorbing layer (z = 0) rounding differences accumulate undamped."""
    shape = (n + 1,) * 3
    h = 10.0
    corr = 100.0 / h

    def model():
        if not true_model:
            return np.full(shape, 3000.0), np.full(shape, 1730.0), np.full(shape, 2000.0)
        vp = 3000.0 * (1.0 + 0.05 * random_field(shape, seeds[0], corr))
        vs = 1730.0 * (1.0 + 0.05 * random_field(shape, seeds[1], corr))
        rho = 2000.0 * (1.0 + 0.05 * random_field(shape, seeds[2], corr))
        vs = np.minimum(vs, vp / 1.5)
        return vp, vs, rho

    vmax = 3000.0 * 1.25  # 5-sigma bound of the perturbed vp; keeps one dt for the true and start models
    f0 = 15.0
    return Workload(
        name=f"elastic3d_hetero_{n}_p{p}", dim=3, physics="elastic", n=(n,) * 3, p=(p,) * 3, h=(h,) * 3,
        n_nb=n_nb, dt=_cfl_dt(h, vmax), steps=steps, model_fn=model, src_index=(n // 2,) * 3,
        src_kinds=("explosive", "shear_xz"), f0=f0, t0=1.2 / f0,
        receivers={"v3": _row_receivers(shape, pml_width)}, precision=precision,
        checkpoint_every=int(math.ceil(math.sqrt(steps))), seed=seeds[0], pml_width=pml_width)


def batched_shots(n_shots: int = 64, steps: int = 1500, n_nb: int = 20, seed: int = 5000,
                  sizes=tuple(range(512, 2049, 128)), M: int = 128, precision: str = "fp32"):
    """Shots of a 2-D acoustic survey with uneven square grids: n_s drawn uniformly from ``sizes`` (multiples
    of M), p_s = n_s / M patches per axis, 3-5 horizontal layers with v ~ U[1500, 4000] sorted by depth,
    rho = 1000, absorbing layers of 40 points on every side.  Source and receivers lie at the top of the physical
    domain, just below the upper layer: a Ricker 20 Hz at (z = 45, x = n_s / 2), receivers on the row z = 40.
    (Inside an absorbing layer the fields are not physical, and its outermost row carries a slowly decaying
    residual whose update is a near-cancellation between the memory variable and the derivative it balances.)"""
    rng = np.random.default_rng(seed)
    ns = rng.choice(np.asarray(sizes), size=n_shots)
    out = []
    h = 10.0
    pml = 40
    for s, n in enumerate(ns):
        n = int(n)
        r = np.random.default_rng(seed + 1 + s)
        n_layers = int(r.integers(3, 6))
        v_layers = np.sort(r.uniform(1500.0, 4000.0, size=n_layers))
        bounds = np.sort(r.uniform(0.1, 0.9, size=n_layers - 1)) * n
        shape = (n + 1, n + 1)

        def model(n=n, v_layers=v_layers, bounds=bounds, shape=shape):
            z = np.arange(n + 1, dtype=np.float64)
            vz = v_layers[np.searchsorted(bounds, z, side="right")]
            return np.repeat(vz[:, None], n + 1, axis=1), None, np.full(shape, 1000.0)

        f0 = 20.0
        out.append(Workload(
            name=f"shot{s}_{n}", dim=2, physics="acoustic", n=(n, n), p=(n // M, n // M), h=(h, h),
            n_nb=n_nb, dt=_cfl_dt(h, float(v_layers.max())), steps=steps, model_fn=model,
            src_index=(pml + 5, n // 2), src_kinds=("pressure",), f0=f0, t0=1.2 / f0,
            receivers={"sigma": _row_receivers(shape, pml)}, precision=precision, seed=seed + 1 + s,
            pml_width=pml))
    return out


# The two layers of the paper's double-layer experiment (Sec. 4.3), read in SI units (km -> m, km/s -> m/s,
# the printed densities as g/cm^3): the upper layer z >= 0 and the deeper layer z < 0.
DOUBLE_LAYER_UPPER = (2614.0, 802.0, 2200.0)   # vp, vs, rho
DOUBLE_LAYER_DEEPER = (5228.0, 1604.0, 2500.0)


def elastic3d_double_layer(n: int = 128, nz: Optional[int] = None, p: int = 4, pz: Optional[int] = None,
                           steps: int = 2000, n_nb: int = 20, f0: float = 0.5, precision: str = "fp32_kahan",
                           pml_width: int = 20) -> Workload:
    """The double-layer model of Sec. 4.3 on [-40 km, 40 km]^3: n intervals along x and y, nz along z (nz = 2n
    gives the paper's z-refined grid), dt = 5 ms as printed.  The interface z = 0 lies on a grid point when nz is
    even and belongs to the upper layer.  The source sits at (0, 0, 10 km) with a Ricker history; the printed 100 Hz
    cannot be resolved at these spacings (a garbled unit), so f0 is a parameter, 0.5 Hz by default, with
    t0 = 1.2 / f0.  The source is the paper's body force along all three axes (f_1 = f_2 = f_3).  Receivers: v3
    on the vertical line x = y = 0, where the paper samples v3(0, 0, z)."""
    nz = n if nz is None else nz
    pz = p if pz is None else pz
    shape = (nz + 1, n + 1, n + 1)
    hz, hxy = 80000.0 / nz, 80000.0 / n

    def model():
        up = (-40000.0 + hz * np.arange(nz + 1) >= 0.0)[:, None, None]
        out = [np.where(up, u, d) * np.ones(shape) for u, d in zip(DOUBLE_LAYER_UPPER, DOUBLE_LAYER_DEEPER)]
        return out[0], out[1], out[2]

    src = (int(round(50000.0 / hz)), n // 2, n // 2)
    line = np.arange(nz + 1, dtype=np.int64) * (n + 1) * (n + 1) + (n // 2) * (n + 1) + n // 2
    return Workload(
        name=f"elastic3d_double_layer_{nz}x{n}x{n}", dim=3, physics="elastic", n=(nz, n, n), p=(pz, p, p),
        h=(hz, hxy, hxy), n_nb=n_nb, dt=0.005, steps=steps, model_fn=model, src_index=src,
        src_kinds=("force_x", "force_y", "force_z"),
        f0=f0, t0=1.2 / f0, receivers={"v3": line}, precision=precision, pml_width=pml_width)


def gaussian_pulse_2d(n: int, p: int, n_nb: int = 20, dt: float = 1e-4, steps: int = 200, pad: int = 0):
    """The paper's 2-D convergence setup (Sec. 4.1): [-5, 5]^2 with n intervals per axis, c = 50 m/s, rho = 1,
    zero velocity and the initial pressure exp(-5 (x^2 + z^2)); no source.  ``pad`` adds that many points of the
    same spacing beyond [-5, 5] on every side, room for an absorbing layer outside the domain (p patches then
    cut n + 2 pad intervals).  Returns (workload, initial sigma)."""
    nt = n + 2 * pad
    shape = (nt + 1, nt + 1)
    h = 10.0 / n
    x = -5.0 + h * (np.arange(nt + 1) - pad)
    sigma0 = np.exp(-5.0 * (x[:, None] ** 2 + x[None, :] ** 2))

    def model():
        return np.full(shape, 50.0), None, np.full(shape, 1.0)

    w = Workload(name=f"gauss2d_{n}_p{p}" + (f"_pad{pad}" if pad else ""), dim=2, physics="acoustic", n=(nt, nt),
                 p=(p, p), h=(h, h), n_nb=n_nb, dt=dt, steps=steps, model_fn=model, src_index=(nt // 2, nt // 2),
                 src_kinds=(), f0=1.0, t0=0.0, amp=0.0, precision="fp64")
    return w, sigma0


def scaled(w: Workload, n: int, p: int, steps: int, n_nb: Optional[int] = None,
           pml_width: Optional[int] = None) -> Workload:
    """A smaller copy of an acoustic/elastic workload on an n-interval grid (same physics, h, dt, source
    type), used for parity cases that the oracle finishes in seconds.  Models are rebuilt at the new size
    with the same recipe (constant or freshly seeded)."""
    d = w.dim
    shape = (n + 1,) * d
    vp0, vs0, rho0 = w.model()
    # Resample the model by nearest-point lookup so that layered structure is kept.
    idx = [np.minimum((np.arange(n + 1) * (w.n[a] / n)).round().astype(int), w.n[a]) for a in range(d)]
    sl = np.ix_(*idx)
    vp = vp0[sl]
    vs = None if vs0 is None else vs0[sl]
    rho = rho0[sl]

    def model():
        return vp.copy(), (None if vs is None else vs.copy()), rho.copy()

    rec = {k: np.arange(int(np.prod(shape[1:])), dtype=np.int64) for k in w.receivers}
    return dataclasses.replace(
        w, name=f"{w.name}_as{n}_p{p}", n=(n,) * d, p=(p,) * d, steps=steps, model_fn=model,
        n_nb=w.n_nb if n_nb is None else n_nb, src_index=tuple(n // 2 for _ in range(d)), receivers=rec,
        pml_width=w.pml_width if pml_width is None else pml_width)


def acoustic2d_gradient_case(n: int = 24, p: int = 2, n_nb: int = 6, steps: int = 40, pml_width: int = 5,
                              precision: str = "fp64"):
    """Small misfit-gradient case: (n+1)^2 points, smooth random vp (2000 m/s +- 5 %) and rho (1000 +- 5 %),
    seeds 11 and 12, a 60 Hz pressure source at the centre, pressure and velocity receivers on the rows z = 2
    (inside the absorbing layer) and z = n - 4.  Returns (workload, (vp, None, rho))."""
    w = acoustic2d_small(n=n, p=p, n_nb=n_nb, steps=steps, pml_width=pml_width)
    shape = w.shape
    vp = 2000.0 * (1 + 0.05 * random_field(shape, 11, 2.0))
    rho = 1000.0 * (1 + 0.05 * random_field(shape, 12, 2.0))
    rows = np.concatenate([2 * (n + 1) + np.arange(n + 1), (n - 4) * (n + 1) + np.arange(n + 1)]).astype(np.int64)
    w = dataclasses.replace(w, f0=60.0, t0=1.2 / 60.0, dt=0.4 * 10.0 / vp.max(), precision=precision,
                            receivers={"sigma": rows, "v1": rows, "v3": rows}, model_fn=lambda: (vp, None, rho))
    return w, (vp, None, rho)


def elastic3d_gradient_case(n: int = 12, p: int = 2, n_nb: int = 4, steps: int = 24, pml_width: int = 3,
                            src_kinds=("explosive", "shear_xz"), precision: str = "fp64"):
    """Small misfit-gradient case: (n+1)^3 points, smooth random vp (3000 +- 5 %), vs (1730 +- 5 %), rho
    (2000 +- 5 %), seeds 21-23, an 80 Hz source at the centre, v1..v3 and s33 receivers on the plane z = 1.
    Returns (workload, (vp, vs, rho))."""
    w = elastic3d_homogeneous(n=n, p=p, n_nb=n_nb, steps=steps, pml_width=pml_width)
    shape = w.shape
    vp = 3000.0 * (1 + 0.05 * random_field(shape, 21, 2.0))
    vs = 1730.0 * (1 + 0.05 * random_field(shape, 22, 2.0))
    rho = 2000.0 * (1 + 0.05 * random_field(shape, 23, 2.0))
    plane = ((n + 1) ** 2 + np.arange((n + 1) ** 2)).astype(np.int64)
    w = dataclasses.replace(w, f0=80.0, t0=1.2 / 80.0, dt=0.4 * 10.0 / vp.max(), src_kinds=tuple(src_kinds),
                            precision=precision, receivers={"v1": plane, "v2": plane, "v3": plane, "s33": plane},
                            model_fn=lambda: (vp, vs, rho))
    return w, (vp, vs, rho)


def mean_model(model):
    """Homogeneous model with the means of ``model`` (the data of the gradient cases come from it)."""
    return tuple(None if a is None else np.full(a.shape, float(a.mean())) for a in model)


WORKLOADS = {
    "acoustic2d_small": acoustic2d_small,
    "acoustic2d_layered": acoustic2d_layered,
    "elastic3d_homogeneous": elastic3d_homogeneous,
    "elastic3d_heterogeneous": elastic3d_heterogeneous,
    "elastic3d_double_layer": elastic3d_double_layer,
}
