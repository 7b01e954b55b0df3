"""Oracle, part 1: the 1-D LOSS derivative along one grid axis (FP64).  TEST INFRASTRUCTURE ONLY.

Follows Sec. 3.1 and 3.2 of the paper step by step:

1. ``global_matrix``: the (N+3)x(N+3) collocation matrix A of Eq. (spline_cofficient_eq), rows
   (1, -2, 1)/h^2 for the natural end conditions (Eq. natural_boundary) and (1, 4, 1)/6 for the
   collocation rows (Eq. spline_coefficient_relation).
2. ``inverse_rows``: rows of b = A^{-1} (Eq. exact_solution), obtained by solving A^T x = e_i with a dense
   pivoted LU (LAPACK gesv).
3. ``pmbc_weights``: the PMBC weights of Eqs. (PMBC) and (PMBC_coeffcients) for every inner junction lM,
   summed over m = -n_nb..n_nb after the four-term completion, with the junction term c_0 counted once; and
   the one-sided end closures phi_L^(1), phi_R^(p) (the equations that close Sec. 3.2).
4. ``pmbc_phi``: the truncated sums phi_j = sum_m W[j, m] f[jM + m].
5. ``local_coefficients``: for each patch, the (M+3)x(M+3) system A_M^(l) of Eq.
   (spline_cofficient_eq_piece) with Hermite rows (-1/(2h), 0, 1/(2h)) = phi, solved by a generic pivoted
   banded solver (LAPACK gbsv).  The paper's explicit LU (Eqs. explicit_L / explicit_U) is not used.
6. ``derivative_1d``: first derivative (c_{i+1} - c_{i-1})/(2h) (Eq. derivative_approximation) and second
   derivative (c_{i-1} - 2 c_i + c_{i+1})/h^2 (the operator of Eq. natural_boundary) at every grid point;
   at a junction shared by two patches both patches' values are averaged.

Truncation: a stencil column outside [0, N] does not exist and is dropped.  With n_nb >= N every sum is
complete and the patched derivative equals the global spline derivative (pinned against an independent
natural cubic spline in the tests).
"""
from __future__ import annotations

import functools

import numpy as np
from scipy.linalg import solve_banded


def global_matrix(n: int, h: float) -> np.ndarray:
    """Dense A of Eq. (spline_cofficient_eq).  Unknown c_k (k = -1..n+1) sits in column k + 1; row 0 and
    row n + 2 are the natural end conditions, row i + 1 is the collocation at x_i."""
    A = np.zeros((n + 3, n + 3))
    A[0, 0:3] = (1.0 / h**2, -2.0 / h**2, 1.0 / h**2)
    for i in range(n + 1):
        A[i + 1, i:i + 3] = (1.0 / 6.0, 4.0 / 6.0, 1.0 / 6.0)
    A[n + 2, n:n + 3] = (1.0 / h**2, -2.0 / h**2, 1.0 / h**2)
    return A


def inverse_rows(n: int, h: float, rows) -> np.ndarray:
    """b_{i,j} for the coefficient indices ``rows`` (each in -1..n+1) and every data index j = 0..n.

    Returns an array of shape (len(rows), n + 1); column j multiplies the sample f_j (the right-hand side
    entries of the two end-condition rows are zero, so their columns never contribute)."""
    A = global_matrix(n, h)
    E = np.zeros((n + 3, len(rows)))
    for k, i in enumerate(rows):
        E[i + 1, k] = 1.0
    # Row i of A^{-1} is the solution x of A^T x = e_i.
    X = np.linalg.solve(A.T, E)
    return X[1:n + 2, :].T.copy()


@functools.lru_cache(maxsize=64)
def pmbc_weights(n: int, p: int, h: float, n_nb: int) -> np.ndarray:
    """W[j, m + n_nb] for junction j = 0..p (0 and p are the two ends) and offset m = -n_nb..n_nb, such that
    phi_j = sum_m W[j, m + n_nb] * f[j*M + m] (Eqs. PMBC, PMBC_coeffcients and the end closures).

    Interior junction lM:  W[l, m] = (-b_{lM-1, lM+m} + b_{lM+1, lM+m}) / (2h), m = -n_nb..n_nb.
    Left end:              W[0, m] = (-b_{-1, m} + b_{1, m}) / (2h),           m = 0..n_nb.
    Right end:             W[p, -k] = (-b_{N-1, N-k} + b_{N+1, N-k}) / (2h),   k = 0..n_nb.
    Offsets whose column falls outside 0..N are zero."""
    if n % p:
        raise ValueError("n must be a multiple of p")
    M = n // p
    rows = sorted({r for l in range(p + 1) for r in (l * M - 1, l * M + 1)})
    B = inverse_rows(n, h, rows)
    row = {r: B[k] for k, r in enumerate(rows)}
    W = np.zeros((p + 1, 2 * n_nb + 1))
    for l in range(p + 1):
        c = l * M
        if l == 0:
            ms = range(0, n_nb + 1)
        elif l == p:
            ms = range(-n_nb, 1)
        else:
            ms = range(-n_nb, n_nb + 1)
        for m in ms:
            col = c + m
            if 0 <= col <= n:
                W[l, m + n_nb] = (-row[c - 1][col] + row[c + 1][col]) / (2.0 * h)
    return W


def pmbc_phi(f: np.ndarray, n: int, p: int, h: float, n_nb: int) -> np.ndarray:
    """phi for every junction of every line.  ``f`` has shape (L, n + 1); returns (L, p + 1)."""
    W = pmbc_weights(n, p, h, n_nb)
    M = n // p
    L = f.shape[0]
    phi = np.zeros((L, p + 1))
    for j in range(p + 1):
        for m in range(-n_nb, n_nb + 1):
            col = j * M + m
            w = W[j, m + n_nb]
            if w != 0.0 and 0 <= col <= n:
                phi[:, j] += w * f[:, col]
    return phi


@functools.lru_cache(maxsize=64)
def local_matrix_banded(M: int, h: float) -> np.ndarray:
    """A_M^(l) of Eq. (spline_cofficient_eq_piece) in LAPACK band storage with 2 sub- and 2
    super-diagonals (row 0: -1/(2h), 0, 1/(2h); rows 1..M+1: (1, 4, 1)/6; row M+2: -1/(2h), 0, 1/(2h))."""
    size = M + 3
    A = np.zeros((size, size))
    A[0, 0], A[0, 2] = -1.0 / (2.0 * h), 1.0 / (2.0 * h)
    for i in range(M + 1):
        A[i + 1, i:i + 3] = (1.0 / 6.0, 4.0 / 6.0, 1.0 / 6.0)
    A[M + 2, M], A[M + 2, M + 2] = -1.0 / (2.0 * h), 1.0 / (2.0 * h)
    lo, up = 2, 2
    ab = np.zeros((lo + up + 1, size))
    for i in range(size):
        for j in range(max(0, i - lo), min(size, i + up + 1)):
            ab[up + i - j, j] = A[i, j]
    return ab


def local_coefficients(f: np.ndarray, phi: np.ndarray, n: int, p: int, h: float) -> np.ndarray:
    """Local spline coefficients c^(l)_{-1..M+1} of every patch of every line: shape (L, p, M + 3)."""
    M = n // p
    ab = local_matrix_banded(M, h)
    L = f.shape[0]
    c = np.empty((L, p, M + 3))
    for l in range(p):
        rhs = np.empty((M + 3, L))
        rhs[0] = phi[:, l]
        rhs[1:M + 2] = f[:, l * M:l * M + M + 1].T
        rhs[M + 2] = phi[:, l + 1]
        c[:, l, :] = solve_banded((2, 2), ab, rhs).T
    return c


def derivative_1d(f: np.ndarray, n: int, p: int, h: float, n_nb: int, second: bool = False):
    """LOSS derivative(s) of every line of ``f`` (shape (L, n + 1)).  Returns d1, or (d1, d2) if
    ``second``."""
    f = np.asarray(f, dtype=np.float64)
    M = n // p
    phi = pmbc_phi(f, n, p, h, n_nb)
    c = local_coefficients(f, phi, n, p, h)
    L = f.shape[0]
    d1 = np.zeros((L, n + 1))
    d2 = np.zeros((L, n + 1))
    cnt = np.zeros(n + 1)
    for l in range(p):
        cl = c[:, l, :]
        d1[:, l * M:l * M + M + 1] += (cl[:, 2:] - cl[:, :-2]) / (2.0 * h)
        d2[:, l * M:l * M + M + 1] += (cl[:, :-2] - 2.0 * cl[:, 1:-1] + cl[:, 2:]) / h**2
        cnt[l * M:l * M + M + 1] += 1.0
    d1 /= cnt
    d2 /= cnt
    return (d1, d2) if second else d1


def derivative(f: np.ndarray, axis: int, n: int, p: int, h: float, n_nb: int, second: bool = False):
    """LOSS derivative of a multi-dimensional field along ``axis`` (tensor-product splines, Sec. 3: each
    axis uses only the 1-D splines along that axis)."""
    f = np.asarray(f, dtype=np.float64)
    fm = np.moveaxis(f, axis, -1)
    shp = fm.shape
    out = derivative_1d(fm.reshape(-1, shp[-1]), n, p, h, n_nb, second)
    if second:
        return tuple(np.moveaxis(o.reshape(shp), -1, axis) for o in out)
    return np.moveaxis(out.reshape(shp), -1, axis)


@functools.lru_cache(maxsize=32)
def derivative_matrix(n: int, p: int, h: float, n_nb: int) -> np.ndarray:
    """The (n+1)x(n+1) matrix of the linear map f -> d1 along one line, built column by column by applying
    ``derivative_1d`` to unit vectors.  Used by the adjoint and by dot-product tests."""
    return derivative_1d(np.eye(n + 1), n, p, h, n_nb).T
