"""Pins of the 1-D oracle derivative against facts fixed by the paper and by mathematics (CPU only).

Each test checks the oracle against something other than itself:
* an independent natural cubic spline (scipy.interpolate.CubicSpline), which the global collocation system of
  Sec. 3.1 defines, for the complete-sum limit of the PMBC (Sec. 3.2);
* the exponential decay of the truncation error with n_nb (Fig. element_decay, Eq. truncated_solution);
* closed forms of the inverse Toeplitz entries and of the PMBC weights (derived from Eq. PMBC_coeffcients);
* algebraic identities implied by the collocation rows (compact scheme, junction consistency);
* the Fourier symbol of the spline derivative and exact reproduction of low-degree polynomials.
"""
import numpy as np
import pytest
from scipy.interpolate import CubicSpline

from oracle import spline

R = np.sqrt(3.0) - 2.0  # root of z^2 + 4 z + 1 with |z| < 1


def _data(n, h, seed=0):
    x = np.arange(n + 1) * h
    rng = np.random.default_rng(seed)
    f = np.sin(2.0 * np.pi * x / (n * h) * 3.3) + 0.2 * rng.standard_normal(n + 1)
    return x, f


@pytest.mark.parametrize("n,p,h", [(16, 1, 1.0), (32, 2, 0.5), (48, 3, 2.0), (64, 4, 1.0), (60, 5, 0.1)])
def test_complete_sums_equal_natural_cubic_spline(n, p, h):
    """P1: with n_nb >= N every PMBC sum is complete and the patched local splines reproduce the global
    natural cubic spline exactly (Sec. 3.2, Eq. relation); first and second derivatives at the knots."""
    x, f = _data(n, h)
    cs = CubicSpline(x, f, bc_type="natural")
    d1, d2 = spline.derivative_1d(f[None], n, p, h, n_nb=n, second=True)
    scale1 = np.abs(cs(x, 1)).max()
    scale2 = np.abs(cs(x, 2)).max()
    assert np.abs(d1[0] - cs(x, 1)).max() <= 1e-13 * scale1
    assert np.abs(d2[0] - cs(x, 2)).max() <= 1e-12 * scale2


def test_truncation_error_decays_like_r_power_nnb():
    """P1b: truncating the PMBC sums at n_nb leaves an error bounded by C |r|^n_nb, r = sqrt(3) - 2, and the
    error shrinks by about |r|^4 for every 4 extra halo points (Fig. element_decay)."""
    n, p, h = 96, 4, 1.0
    x, f = _data(n, h, seed=3)
    exact = CubicSpline(x, f, bc_type="natural")(x, 1)
    errs = {}
    for n_nb in (6, 10, 14, 18):
        d1 = spline.derivative_1d(f[None], n, p, h, n_nb)[0]
        errs[n_nb] = np.abs(d1 - exact).max()
        # Bound: each of the two halves of a junction sum drops a geometric tail of the weights
        # w_k = sqrt(3)(1 - r^2) r^(k-1)/(2h); the tail beyond n_nb sums to sqrt(3)(1+|r|)|r|^n_nb/(2h).
        tail = 2.0 * np.sqrt(3.0) * (1.0 + abs(R)) * abs(R) ** n_nb / (2.0 * h)
        assert errs[n_nb] <= tail * np.abs(f).max() * 4.0
    for a, b in ((6, 10), (10, 14), (14, 18)):
        ratio = errs[b] / errs[a]
        assert 0.1 * abs(R) ** 4 < ratio < 10.0 * abs(R) ** 4


def test_inverse_toeplitz_interior_closed_form():
    """P2: far from both ends the inverse of the collocation matrix is Toeplitz, b_{i,i+k} = sqrt(3) r^|k|
    (the bi-infinite inverse of tridiag(1, 4, 1)/6)."""
    n, h = 200, 1.0
    i = 100
    b = spline.inverse_rows(n, h, [i])[0]
    k = np.arange(-30, 31)
    assert np.allclose(b[i + k], np.sqrt(3.0) * R ** np.abs(k), rtol=0, atol=1e-14)


def test_pmbc_weights_closed_form_and_linear_exactness():
    """P2: interior PMBC weights (Eq. PMBC_coeffcients) are antisymmetric, W[0] = c_0 = 0 and
    W[+-k] = +-sqrt(3)(1 - r^2) r^(k-1)/(2h); the complete sums reproduce the derivative of a linear
    function: sum_k 2 k h w_k = 1."""
    n, p, h, n_nb = 256, 4, 10.0, 20
    W = spline.pmbc_weights(n, p, h, n_nb)
    k = np.arange(1, n_nb + 1)
    wk = np.sqrt(3.0) * (1.0 - R**2) * R ** (k - 1) / (2.0 * h)
    for j in (1, 2, 3):
        assert abs(W[j, n_nb]) < 1e-16
        assert np.allclose(W[j, n_nb + k], wk, rtol=1e-12, atol=0)
        assert np.allclose(W[j, n_nb - k], -wk, rtol=1e-12, atol=0)
    kk = np.arange(1, 200)
    full = np.sqrt(3.0) * (1.0 - R**2) * R ** (kk - 1) / (2.0 * h)
    assert abs(np.sum(2.0 * kk * h * full) - 1.0) < 1e-13


def test_end_closure_is_natural_spline_end_derivative():
    """The one-sided end sums with n_nb >= N give the global natural spline's slope at both ends."""
    n, p, h = 40, 2, 0.25
    x, f = _data(n, h, seed=7)
    phi = spline.pmbc_phi(f[None], n, p, h, n_nb=n)[0]
    cs = CubicSpline(x, f, bc_type="natural")
    assert abs(phi[0] - cs(x[0], 1)) < 1e-12 * np.abs(cs(x, 1)).max()
    assert abs(phi[-1] - cs(x[-1], 1)) < 1e-12 * np.abs(cs(x, 1)).max()
    assert abs(phi[1] - cs(x[n // p], 1)) < 1e-12 * np.abs(cs(x, 1)).max()


@pytest.mark.parametrize("n_nb", [4, 12, 20])
def test_compact_scheme_identity_inside_patches(n_nb):
    """P3: the collocation rows imply (d_{i-1} + 4 d_i + d_{i+1})/6 = (f_{i+1} - f_{i-1})/(2h) at every
    point strictly inside a patch, whatever phi and n_nb are (Eqs. spline_cofficient_eq_piece and
    derivative_approximation)."""
    n, p, h = 120, 3, 0.7
    M = n // p
    _, f = _data(n, h, seed=11)
    d = spline.derivative_1d(f[None], n, p, h, n_nb)[0]
    for l in range(p):
        i = np.arange(l * M + 1, (l + 1) * M)
        lhs = (d[i - 1] + 4.0 * d[i] + d[i + 1]) / 6.0
        rhs = (f[i + 1] - f[i - 1]) / (2.0 * h)
        assert np.abs(lhs - rhs).max() <= 1e-13 * np.abs(rhs).max()


def test_junction_derivative_equals_phi_from_both_patches():
    """P4: at a shared junction the Hermite rows force the first derivative of the left patch and of the
    right patch to equal phi (Sec. 3.2, effective Hermite boundary conditions)."""
    n, p, h, n_nb = 64, 4, 1.0, 10
    M = n // p
    _, f = _data(n, h, seed=5)
    phi = spline.pmbc_phi(f[None], n, p, h, n_nb)
    c = spline.local_coefficients(f[None], phi, n, p, h)[0]
    for l in range(1, p):
        left = (c[l - 1, M + 2] - c[l - 1, M]) / (2.0 * h)
        right = (c[l, 2] - c[l, 0]) / (2.0 * h)
        assert abs(left - phi[0, l]) < 1e-13
        assert abs(right - phi[0, l]) < 1e-13


def test_fourier_symbol_of_spline_derivative():
    """P5: for f = cos(k x) the interior derivative is -3 sin(kh) / (h (2 + cos kh)) sin(k x), the symbol of
    the compact relation (d_{i-1} + 4 d_i + d_{i+1})/6 = (f_{i+1} - f_{i-1})/(2h), up to boundary
    influence that decays like |r|^distance."""
    n, p, h, n_nb = 400, 4, 1.0, 24
    x = np.arange(n + 1) * h
    for kh in (0.1, 0.5, 1.0, 2.0):
        f = np.cos(kh * x)
        d = spline.derivative_1d(f[None], n, p, h, n_nb)[0]
        sym = -3.0 * np.sin(kh) / (h * (2.0 + np.cos(kh)))
        mid = slice(60, n - 60)
        assert np.abs(d[mid] - sym * np.sin(kh * x[mid])).max() < 1e-11


def test_polynomial_reproduction():
    """P6: linear data are differentiated exactly everywhere and cubic data exactly away from the ends (the
    natural end conditions perturb the spline by a term decaying like |r|^distance); complete sums."""
    n, p, h = 120, 4, 0.5
    x = np.arange(n + 1) * h
    lin = 3.0 - 2.5 * x
    d = spline.derivative_1d(lin[None], n, p, h, n_nb=n)[0]
    assert np.abs(d + 2.5).max() < 1e-12
    cub = 0.01 * (x - 20.0) ** 3 - 0.3 * x**2 + x
    d = spline.derivative_1d(cub[None], n, p, h, n_nb=n)[0]
    exact = 0.03 * (x - 20.0) ** 2 - 0.6 * x + 1.0
    mid = slice(30, n - 30)
    assert np.abs(d[mid] - exact[mid]).max() < 1e-12 * np.abs(exact).max()


def test_multidim_derivative_acts_along_one_axis():
    """Tensor-product derivatives (Sec. 3): d/dx of f(z) g(x) equals f(z) g'(x) line by line."""
    n, p, h, n_nb = 32, 2, 1.0, 16
    z = np.arange(n + 1) * h
    fz = np.cos(0.2 * z)
    gx = np.sin(0.3 * z)
    F = fz[:, None] * gx[None, :]
    dx = spline.derivative(F, 1, n, p, h, n_nb)
    dg = spline.derivative_1d(gx[None], n, p, h, n_nb)[0]
    assert np.allclose(dx, fz[:, None] * dg[None, :], rtol=0, atol=1e-14)
