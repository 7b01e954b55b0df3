"""GPU parity of the LOSS derivative rows (PMBC closure, local solve, first and second derivatives) against the
FP64 oracle, element by element, through the C ABI (loss_derivative / loss_pmbc_phi)."""
import numpy as np
import pytest

from oracle import spline

pytestmark = pytest.mark.gpu

# (dim, n per axis, p per axis, n_nb, h per axis): several tiles, ragged line bundles (n + 1 not a multiple of
# the bundle width), chunk tails (M - 1 not a multiple of the chunk length), n_nb = M, p = 1.
CASES = [
    (2, (32, 48), (2, 3), 8, (1.0, 0.5)),
    (2, (64, 64), (4, 2), 12, (10.0, 10.0)),
    (2, (128, 96), (2, 4), 20, (1.0, 2.0)),
    (2, (300, 256), (3, 8), 20, (10.0, 10.0)),
    (2, (40, 36), (1, 2), 18, (0.3, 0.7)),
    (3, (24, 32, 40), (2, 2, 4), 10, (1.0, 1.5, 0.5)),
    (3, (48, 20, 66), (4, 1, 3), 12, (2.0, 1.0, 1.0)),
]
TOL = {"fp64": (1e-12, 1e-11), "fp32": (2e-5, 2e-4)}


def _grid(pkg, dim, n, p, n_nb, h, prec):
    d = pkg.make_desc(dim, pkg.LOSS_ACOUSTIC, pkg.PRECISIONS[prec], n_nb, n, p, h, 1e-3)
    return pkg.Grid([d])


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as ge

    ge.build()
    import paper_2301_05127_gb300 as p

    return p


def _field(shape, seed):
    rng = np.random.default_rng(seed)
    f = rng.standard_normal(shape)
    # add smooth content so that derivatives are not dominated by grid-scale noise
    grids = np.meshgrid(*[np.linspace(0, 1, s) for s in shape], indexing="ij")
    return f + 5.0 * np.sin(3.0 * sum(grids))


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_derivative_matches_oracle(pkg, case, prec):
    dim, n, p, n_nb, h = CASES[case]
    g = _grid(pkg, dim, n, p, n_nb, h, prec)
    f = _field(g.shape(), seed=100 + case)
    fw = f.astype(g.dtype)
    t1, t2 = TOL[prec]
    for axis in range(dim):
        d1, d2 = g.derivative(0, axis, fw, second=True)
        r1, r2 = spline.derivative(fw.astype(np.float64), axis, n[axis], p[axis], h[axis], n_nb, second=True)
        e1 = np.abs(d1 - r1).max() / np.abs(r1).max()
        e2 = np.abs(d2 - r2).max() / np.abs(r2).max()
        assert e1 < t1, (axis, e1)
        assert e2 < t2, (axis, e2)
    g.close()


@pytest.mark.parametrize("case", [0, 3, 5])
def test_pmbc_phi_matches_oracle(pkg, case):
    dim, n, p, n_nb, h = CASES[case]
    g = _grid(pkg, dim, n, p, n_nb, h, "fp32")
    f = _field(g.shape(), seed=7).astype(np.float32)
    for axis in range(dim):
        phi = g.pmbc_phi(0, axis, f)
        lines = np.moveaxis(f.astype(np.float64), axis, -1).reshape(-1, n[axis] + 1)
        ref = spline.pmbc_phi(lines, n[axis], p[axis], h[axis], n_nb)
        assert np.abs(phi - ref).max() <= 1e-13 * np.abs(ref).max(), axis
    g.close()


def test_derivative_device_buffers(pkg):
    import torch

    g = _grid(pkg, 2, (64, 64), (2, 2), 12, (1.0, 1.0), "fp32")
    f = torch.from_numpy(_field(g.shape(), 3).astype(np.float32)).cuda()
    d1 = g.derivative(0, 1, f)
    ref = spline.derivative(f.cpu().double().numpy(), 1, 64, 2, 1.0, 12)
    assert torch.is_tensor(d1) and d1.is_cuda
    assert np.abs(d1.cpu().numpy() - ref).max() < 2e-5 * np.abs(ref).max()
    g.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_full_size_layered_grid_derivative(pkg, prec):
    """2049^2 points in 8 x 8 patches (the layered 2-D benchmark geometry), both axes, element-wise."""
    g = _grid(pkg, 2, (2048, 2048), (8, 8), 20, (10.0, 10.0), prec)
    f = _field(g.shape(), 11).astype(g.dtype)
    t1, _ = TOL[prec]
    for axis in (0, 1):
        d1 = g.derivative(0, axis, f)
        r1 = spline.derivative(f.astype(np.float64), axis, 2048, 8, 10.0, 20)
        assert np.abs(d1 - r1).max() / np.abs(r1).max() < t1
    g.close()


def test_full_size_elastic_grid_derivative(pkg):
    """257^3 points in 4 x 4 x 4 patches (the homogeneous 3-D benchmark geometry), all three axes, FP32."""
    g = _grid(pkg, 3, (256, 256, 256), (4, 4, 4), 20, (10.0, 10.0, 10.0), "fp32")
    rng = np.random.default_rng(5)
    f = rng.standard_normal(g.shape()).astype(np.float32)
    for axis in (0, 1, 2):
        d1 = g.derivative(0, axis, f)
        r1 = spline.derivative(f.astype(np.float64), axis, 256, 4, 10.0, 20)
        assert np.abs(d1 - r1).max() / np.abs(r1).max() < 2e-5
    g.close()
