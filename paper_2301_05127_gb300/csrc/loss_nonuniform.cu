// LOSS derivative on an axis with non-uniform grid spacing.
//
// The paper develops LOSS on a uniform grid and notes that the construction carries over to non-uniform grids
// (Sec. 3, and the future work of its conclusion).  On knots x_0 < ... < x_N the cubic spline through the samples
// is described here by its knot slopes d_i = s'(x_i), which is equivalent to the B-spline coefficients of the paper
// (the spline restricted to a patch is fixed by its samples and its two end slopes):
//
//   - C^2 continuity at an interior knot i gives the slope equation
//       h_i d_{i-1} + 2 (h_{i-1} + h_i) d_i + h_{i-1} d_{i+1} = a_i (f_i - f_{i-1}) + b_i (f_{i+1} - f_i),
//     with h_i = x_{i+1} - x_i, a_i = 3 h_i / h_{i-1}, b_i = 3 h_{i-1} / h_i (uniform grid: d_{i-1} + 4 d_i + d_{i+1}
//     = 3 (f_{i+1} - f_{i-1}) / h);
//   - the natural end conditions s''(x_0) = s''(x_N) = 0 give 2 d_0 + d_1 = 3 (f_1 - f_0) / h_0 and
//     d_{N-1} + 2 d_N = 3 (f_N - f_{N-1}) / h_{N-1}.
//
// PMBC weights (Eqs. PMBC, PMBC_coeffcients): the junction slope of the global spline is row jM of T^{-1} R (T the
// slope matrix, R the right-hand-side operator), computed in FP64 on the host by one tridiagonal solve with T^T per
// junction and truncated to |m| <= n_nb (one-sided at the ends).  The local solve of each patch is the slope system
// of its interior knots with the junction values phi as Dirichlet ends, by Thomas elimination with per-position
// factors (the patch matrices differ, so there is no shared factor table).  Samples of the PMBC sums are
// accumulated in FP64.
//
// One thread per (grid line, patch): it forms both junction sums, sweeps forward writing the eliminated right-hand
// side into the output line, and sweeps back.  Consecutive threads take consecutive lines of the same patch, so
// lines along y and z (consecutive x) load and store coalesced; lines along x are walked by each thread alone.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "loss_host.h"
#include "loss_line.cuh"

namespace lossk {

#define NU_TRY(expr)                \
  do {                              \
    loss_status_t st_ = (expr);     \
    if (st_ != LOSS_OK) return st_; \
  } while (0)

static loss_status_t fail_msg(loss_ctx* h, loss_status_t st, const std::string& msg) {
  h->err = msg;
  return st;
}

// Host: FP64 tables of one non-uniform axis.  W: [(p + 1)][2 n_nb + 1] PMBC weights.  Per knot i: A = h_i,
// G = h_{i-1} (the off-diagonal coefficients), L = the forward-elimination multiplier (0 at a patch's first
// interior knot), IU = 1 / pivot, a_i, b_i (right-hand side); entries at junctions are unused.
struct NuHost {
  std::vector<double> W, A, G, L, IU, ra, rb;
};

static bool nu_tables(const std::vector<double>& x, int p, int n_nb, NuHost* t, std::string* why) {
  const int N = (int)x.size() - 1;
  if (N < 2 || N % p) return *why = "bad knot count", false;
  std::vector<double> h(N);
  for (int i = 0; i < N; ++i) {
    h[i] = x[i + 1] - x[i];
    if (!(h[i] > 0.0) || !std::isfinite(h[i])) return *why = "knots must be finite and strictly increasing", false;
  }
  const int M = N / p;
  // Global slope system T d = R f: sub (lo), diagonal (di), super (up) of T; R row i has entries at i - 1, i, i + 1.
  std::vector<double> lo(N + 1, 0.0), di(N + 1), up(N + 1, 0.0), rm(N + 1, 0.0), r0(N + 1, 0.0), rp(N + 1, 0.0);
  di[0] = 2.0, up[0] = 1.0, r0[0] = -3.0 / h[0], rp[0] = 3.0 / h[0];
  di[N] = 2.0, lo[N] = 1.0, rm[N] = -3.0 / h[N - 1], r0[N] = 3.0 / h[N - 1];
  for (int i = 1; i < N; ++i) {
    lo[i] = h[i];
    di[i] = 2.0 * (h[i - 1] + h[i]);
    up[i] = h[i - 1];
    const double a = 3.0 * h[i] / h[i - 1], b = 3.0 * h[i - 1] / h[i];
    rm[i] = -a, r0[i] = a - b, rp[i] = b;
  }
  // Row c of T^{-1} R: solve T^T y = e_c (T^T has sub-diagonal up[i - 1] and super-diagonal lo[i + 1]), then
  // w_j = sum_i y_i R_{i, j}.
  const int wl = 2 * n_nb + 1;
  t->W.assign((size_t)(p + 1) * wl, 0.0);
  std::vector<double> cp(N + 1), y(N + 1);
  for (int j = 0; j <= p; ++j) {
    const int c = j * M;
    // Thomas on T^T: row i reads y_{i-1} up[i-1] + y_i di[i] + y_{i+1} lo[i+1] = delta_{ic}
    double den = di[0];
    cp[0] = (N > 0 ? lo[1] : 0.0) / den;
    y[0] = (c == 0 ? 1.0 : 0.0) / den;
    for (int i = 1; i <= N; ++i) {
      const double sub = up[i - 1];
      den = di[i] - sub * cp[i - 1];
      cp[i] = (i < N ? lo[i + 1] : 0.0) / den;
      y[i] = ((i == c ? 1.0 : 0.0) - sub * y[i - 1]) / den;
    }
    for (int i = N - 1; i >= 0; --i) y[i] -= cp[i] * y[i + 1];
    const int mlo = (j == 0) ? 0 : -n_nb, mhi = (j == p) ? 0 : n_nb;
    for (int m = mlo; m <= mhi; ++m) {
      const int col = c + m;
      if (col < 0 || col > N) continue;
      double w = 0.0;  // (R^T y)_col = y_{col+1} R_{col+1,col} + y_col R_{col,col} + y_{col-1} R_{col-1,col}
      if (col + 1 <= N) w += y[col + 1] * rm[col + 1];
      w += y[col] * r0[col];
      if (col - 1 >= 0) w += y[col - 1] * rp[col - 1];
      t->W[(size_t)j * wl + (m + n_nb)] = w;
    }
  }
  // Local elimination tables of the patch systems (interior knots lM + 1 .. (l + 1)M - 1).
  t->A.assign(N + 1, 0.0), t->G.assign(N + 1, 0.0), t->L.assign(N + 1, 0.0), t->IU.assign(N + 1, 0.0);
  t->ra.assign(N + 1, 0.0), t->rb.assign(N + 1, 0.0);
  for (int l = 0; l < p; ++l) {
    double u_prev = 0.0;
    for (int i = l * M + 1; i < (l + 1) * M; ++i) {
      t->A[i] = h[i];
      t->G[i] = h[i - 1];
      t->ra[i] = 3.0 * h[i] / h[i - 1];
      t->rb[i] = 3.0 * h[i - 1] / h[i];
      const double d = 2.0 * (h[i - 1] + h[i]);
      if (i == l * M + 1) {
        t->L[i] = 0.0;
        u_prev = d;
      } else {
        t->L[i] = h[i] / u_prev;
        u_prev = d - t->L[i] * h[i - 2];  // the previous knot's super-diagonal is G_{i-1} = h_{i-2}
      }
      t->IU[i] = 1.0 / u_prev;
    }
  }
  return true;
}

template <typename T>
struct NuArgs {
  const T* f;
  T* d1;
  double* phi;       // [lines][p + 1] or null
  const double* W;   // [(p + 1)][2 n_nb + 1]
  const T* tab;      // A, G, L, IU, ra, rb, H (knot spacings h_i = x_{i+1} - x_i): 7 x (n + 1)
  int64_t lines, stride;
  int64_t outer_stride;  // base of line q: (q / inner) * outer_stride + (q % inner) * inner_mul
  int64_t inner, inner_mul;
  int n, p, M, n_nb;
};

template <typename T>
__global__ void __launch_bounds__(128) k_nu_deriv(NuArgs<T> a) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= a.lines * a.p) return;
  const int l = (int)(tid / a.lines);
  const int64_t q = tid - (int64_t)l * a.lines;
  const int64_t base = (q / a.inner) * a.outer_stride + (q % a.inner) * a.inner_mul;
  const T* f = a.f + base;
  const int64_t s = a.stride;
  const int wl = 2 * a.n_nb + 1;
  auto phi_sum = [&](int j) {
    const int c = j * a.M;
    const int mlo = max(-a.n_nb, -c), mhi = min(a.n_nb, a.n - c);
    const double* w = a.W + (size_t)j * wl + a.n_nb;
    double acc = 0.0;
    for (int m = mlo; m <= mhi; ++m) acc = fma(w[m], (double)f[(c + m) * s], acc);
    return acc;
  };
  const double phL = phi_sum(l), phR = phi_sum(l + 1);
  if (a.phi) {
    a.phi[q * (a.p + 1) + l] = phL;
    if (l == a.p - 1) a.phi[q * (a.p + 1) + a.p] = phR;
  }
  if (!a.d1) return;
  T* d = a.d1 + base;
  const int np = a.n + 1;
  const T* A = a.tab;
  const T* G = A + np;
  const T* L = G + np;
  const T* IU = L + np;
  const T* RA = IU + np;
  const T* RB = RA + np;
  const int c0 = l * a.M, c1 = c0 + a.M;
  T fm = f[c0 * s], f0 = f[(c0 + 1) * s];
  T y = T(0);
  for (int i = c0 + 1; i < c1; ++i) {
    const T fp = f[(i + 1) * s];
    T r = RA[i] * (f0 - fm) + RB[i] * (fp - f0);
    if (i == c0 + 1) r -= A[i] * (T)phL;
    if (i == c1 - 1) r -= G[i] * (T)phR;
    y = r - L[i] * y;
    d[i * s] = y;
    fm = f0;
    f0 = fp;
  }
  T dn = T(0);
  for (int i = c1 - 1; i > c0; --i) {
    const T v = (d[i * s] - (i < c1 - 1 ? G[i] * dn : T(0))) * IU[i];
    d[i * s] = v;
    dn = v;
  }
  d[c0 * s] = (T)phL;
  if (l == a.p - 1) d[c1 * s] = (T)phR;
}

// Second derivative of the patched spline from the samples f and the slopes d1 (k_nu_deriv's output): on each
// interval the spline is the cubic with values f_i, f_{i+1} and slopes d_i, d_{i+1}, whose second derivative is
// 6 (f_{i+1} - f_i) / h^2 - (4 d_i + 2 d_{i+1}) / h at x_i and -6 (f_{i+1} - f_i) / h^2 + (2 d_i + 4 d_{i+1}) / h at
// x_{i+1}.  Inside a patch the slope equations make the spline C^2, so one side serves; at a junction the two
// patches' values are averaged, as for the uniform grid.  One thread per (line, patch), as k_nu_deriv.
template <typename T>
__global__ void __launch_bounds__(128) k_nu_d2(NuArgs<T> a, T* __restrict__ d2) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= a.lines * a.p) return;
  const int l = (int)(tid / a.lines);
  const int64_t q = tid - (int64_t)l * a.lines;
  const int64_t base = (q / a.inner) * a.outer_stride + (q % a.inner) * a.inner_mul;
  const T* f = a.f + base;
  const T* d = a.d1 + base;
  T* o = d2 + base;
  const int64_t s = a.stride;
  const T* H = a.tab + 6 * (int64_t)(a.n + 1);
  auto right = [&](int i) {  // s''(x_i) on [x_i, x_{i+1}]
    const T h = H[i];
    return T(6) * (f[(i + 1) * s] - f[i * s]) / (h * h) - (T(4) * d[i * s] + T(2) * d[(i + 1) * s]) / h;
  };
  auto left = [&](int i) {  // s''(x_i) on [x_{i-1}, x_i]
    const T h = H[i - 1];
    return T(-6) * (f[i * s] - f[(i - 1) * s]) / (h * h) + (T(2) * d[(i - 1) * s] + T(4) * d[i * s]) / h;
  };
  const int c0 = l * a.M, c1 = c0 + a.M;
  for (int i = c0 + 1; i < c1; ++i) o[i * s] = right(i);
  o[c0 * s] = l == 0 ? right(c0) : T(0.5) * (left(c0) + right(c0));
  if (l == a.p - 1) o[c1 * s] = left(c1);
}

// Transpose of the derivative on knots, out = D^T g, in two passes.  The forward operator per (line, patch) is
// d_int = T^{-1} r with r_i = -RA_i f_{i-1} + (RA_i - RB_i) f_i + RB_i f_{i+1} - A_{c0+1} phi_L [i = c0 + 1]
// - G_{c1-1} phi_R [i = c1 - 1], d at the patch's first knot = phi_L (and at the line's last knot = phi_R), and
// phi_j = sum_m W[j][m] f_{jM+m}.  Pass 1, per (line, patch): y = T^{-T} g_int by the transposed Thomas factors
// (T = L U: U^T z = g forward, L^T y = z backward), the interior f-bar = R^T y at the patch's interior knots, and
// into scratch the patch's contributions at its two end knots (from R^T) and to its two junction sums (from the
// phi terms and the junction outputs).  Pass 2, per sample: the end-knot contributions of both patches at a
// junction and W^T applied to the junction adjoints, in FP64 as the forward junction sums.
template <typename T>
__global__ void __launch_bounds__(128) k_nu_adj1(NuArgs<T> a, const T* __restrict__ gin, T* __restrict__ out,
                                                 double* __restrict__ scr) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nt = a.lines * a.p;
  if (tid >= nt) return;
  const int l = (int)(tid / a.lines);
  const int64_t q = tid - (int64_t)l * a.lines;
  const int64_t base = (q / a.inner) * a.outer_stride + (q % a.inner) * a.inner_mul;
  const T* g = gin + base;
  T* o = out + base;
  const int64_t s = a.stride;
  const int np = a.n + 1;
  const T* A = a.tab;
  const T* G = A + np;
  const T* L = G + np;
  const T* IU = L + np;
  const T* RA = IU + np;
  const T* RB = RA + np;
  const int c0 = l * a.M, c1 = c0 + a.M;
  T zp = T(0);
  for (int i = c0 + 1; i < c1; ++i) {  // U^T z = g
    const T z = (g[i * s] - (i > c0 + 1 ? G[i - 1] * zp : T(0))) * IU[i];
    o[i * s] = z;
    zp = z;
  }
  T yn = T(0);
  for (int i = c1 - 1; i > c0; --i) {  // L^T y = z
    const T y = o[i * s] - (i < c1 - 1 ? L[i + 1] * yn : T(0));
    o[i * s] = y;
    yn = y;
  }
  const T y0 = o[(c0 + 1) * s], y1 = o[(c1 - 1) * s];
  T yprev = T(0);
  for (int i = c0 + 1; i < c1; ++i) {  // f-bar = R^T y at the interior knots
    const T yi = o[i * s];
    T fb = (RA[i] - RB[i]) * yi;
    if (i + 1 < c1) fb -= RA[i + 1] * o[(i + 1) * s];
    if (i - 1 > c0) fb += RB[i - 1] * yprev;
    o[i * s] = fb;
    yprev = yi;
  }
  scr[tid] = -(double)RA[c0 + 1] * (double)y0;                       // f-bar at the first knot
  scr[nt + tid] = (double)RB[c1 - 1] * (double)y1;                   // f-bar at the last knot
  scr[2 * nt + tid] = (double)g[c0 * s] - (double)A[c0 + 1] * (double)y0;  // adjoint of phi_L
  scr[3 * nt + tid] = -(double)G[c1 - 1] * (double)y1 + (l == a.p - 1 ? (double)g[c1 * s] : 0.0);  // of phi_R
}

template <typename T>
__global__ void __launch_bounds__(256) k_nu_adj2(NuArgs<T> a, T* __restrict__ out, const double* __restrict__ scr) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int np = a.n + 1;
  if (tid >= a.lines * np) return;
  const int64_t q = tid / np;
  const int i = (int)(tid - q * np);
  const int64_t nt = a.lines * a.p;
  const int64_t base = (q / a.inner) * a.outer_stride + (q % a.inner) * a.inner_mul;
  T* o = out + base + (int64_t)i * a.stride;
  auto at = [&](int part, int l) { return scr[part * nt + (int64_t)l * a.lines + q]; };
  double acc = 0.0;
  const bool junction = i % a.M == 0;
  if (junction) {
    const int j = i / a.M;
    if (j >= 1) acc += at(1, j - 1);
    if (j < a.p) acc += at(0, j);
  }
  const int wl = 2 * a.n_nb + 1;
  const int jlo = max(0, (i - a.n_nb + a.M - 1) / a.M), jhi = min(a.p, (i + a.n_nb) / a.M);
  for (int j = jlo; j <= jhi; ++j) {
    const int m = i - j * a.M;
    if (m < -a.n_nb || m > a.n_nb) continue;
    const double pb = (j >= 1 ? at(3, j - 1) : 0.0) + (j < a.p ? at(2, j) : 0.0);
    acc = fma(a.W[(size_t)j * wl + (m + a.n_nb)], pb, acc);
  }
  *o = junction ? (T)acc : (T)((double)*o + acc);
}

// Uploads the tables of axis slot k of shot s (built from the knots x, n[k] + 1 of them).
static loss_status_t nu_upload(loss_ctx* h, Shot& s, int k, const std::vector<double>& x) {
  NuHost t;
  std::string why;
  if (!nu_tables(x, s.p[k], s.d.n_nb, &t, &why)) return fail_msg(h, LOSS_E_ARG, why);
  const size_t np = (size_t)s.n[k] + 1;
  const size_t wbytes = t.W.size() * sizeof(double);
  const size_t tbytes = 7 * np * s.esize;
  std::vector<unsigned char> blob(wbytes + tbytes);
  std::memcpy(blob.data(), t.W.data(), wbytes);
  std::vector<double> hs(np, 0.0);
  for (size_t i = 0; i + 1 < np; ++i) hs[i] = x[i + 1] - x[i];
  const std::vector<double>* cols[7] = {&t.A, &t.G, &t.L, &t.IU, &t.ra, &t.rb, &hs};
  for (int c = 0; c < 7; ++c)
    for (size_t i = 0; i < np; ++i) {
      unsigned char* dst = blob.data() + wbytes + (c * np + i) * s.esize;
      if (s.esize == 8) {
        const double v = (*cols[c])[i];
        std::memcpy(dst, &v, 8);
      } else {
        const float v = (float)(*cols[c])[i];
        std::memcpy(dst, &v, 4);
      }
    }
  if (s.nu_tab[k]) dev_free(h, s.nu_tab[k]);
  s.nu_tab[k] = nullptr;
  NU_TRY(dev_alloc(h, blob.size(), &s.nu_tab[k]));
  NU_TRY(cuda_check(h, cudaMemcpyAsync(s.nu_tab[k], blob.data(), blob.size(), cudaMemcpyHostToDevice, h->stream),
                      "upload knot tables"));
  return cuda_check(h, cudaStreamSynchronize(h->stream), "sync");
}

// Derivative along axis slot k of a field stored with row pitch py (elements between consecutive y, or z in 2-D,
// rows) and plane pitch pz: dense arrays have py = nx, pz = nx * ny; the handle's fields have py = s.sy, pz = s.sz.
template <typename T>
static void nu_args(const Shot& s, int k, int64_t py, int64_t pz, NuArgs<T>* pa) {
  NuArgs<T>& a = *pa;
  a.W = (const double*)s.nu_tab[k];
  const size_t wl = 2 * (size_t)s.d.n_nb + 1;
  a.tab = (const T*)((const unsigned char*)s.nu_tab[k] + (s.p[k] + 1) * wl * sizeof(double));
  a.n = (int)s.n[k];
  a.p = s.p[k];
  a.M = a.n / a.p;
  a.n_nb = s.d.n_nb;
  const int64_t nx = s.len[2], ny = s.len[1];
  a.lines = s.dense / s.len[k];
  if (k == 2) {  // x lines: q = z * ny + y
    a.stride = 1, a.inner = ny, a.inner_mul = py, a.outer_stride = pz;
  } else if (k == 1) {  // y lines: q = z * nx + x
    a.stride = py, a.inner = nx, a.inner_mul = 1, a.outer_stride = pz;
  } else {  // z lines: q = y * nx + x
    a.stride = pz, a.inner = nx, a.inner_mul = 1, a.outer_stride = py;
  }
}

template <typename T>
static loss_status_t nu_launch(loss_ctx* h, Shot& s, int k, const T* f, T* d1, double* phi, int64_t py, int64_t pz,
                               int kernel, T* d2 = nullptr) {
  NuArgs<T> a{};
  nu_args(s, k, py, pz, &a);
  a.f = f;
  a.d1 = d1;
  a.phi = phi;
  const int64_t threads = a.lines * a.p;
  LaunchScope ls(h, kernel);
  k_nu_deriv<T><<<(unsigned)((threads + 127) / 128), 128, 0, h->stream>>>(a);
  if (d2 && d1) {
    NU_TRY(cuda_check(h, cudaGetLastError(), "non-uniform derivative kernel"));
    k_nu_d2<T><<<(unsigned)((threads + 127) / 128), 128, 0, h->stream>>>(a, d2);
  }
  return cuda_check(h, cudaGetLastError(), "non-uniform derivative kernel");
}

template <typename T>
loss_status_t run_nu_derivative(loss_ctx* h, Shot& s, int k, const T* f, T* d1, double* phi, T* d2) {
  return nu_launch<T>(h, s, k, f, d1, phi, s.len[2], s.len[2] * s.len[1], LOSS_KERNEL_DERIVATIVE, d2);
}

// --- time step on grids with non-uniform axes (2-D acoustic) ------------------------------------------------
// The literal Strang sequence of Sec. 3.3 (half A, B, half A) with every derivative taken on the axis's knots; the
// velocities are kept at the integer time level (no staggering), so a step is six derivatives and three pointwise
// updates.  Axes without knots of their own get equally spaced ones, so that every derivative uses one kernel.

// u += coef * scale * (g0 + g1) (g1 may be null; coef an array or the scalar coef0), compensated when K.
template <typename T, bool K>
__global__ void __launch_bounds__(256) k_nu_update(T* __restrict__ u, T* __restrict__ c, const T* __restrict__ g0,
                                                   const T* __restrict__ g1, const T* __restrict__ coef, T coef0,
                                                   T scale, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const T g = g1 ? g0[i] + g1[i] : g0[i];
    const T delta = (scale * (coef ? coef[i] : coef0)) * g;
    if constexpr (K) {
      float v = u[i], cc = c[i];
      kahan_add(v, cc, delta);
      u[i] = v;
      c[i] = cc;
    } else {
      u[i] += delta;
    }
  }
}

// With absorbing layers.  Velocity v along axis slot k: v += b X, X the exact sub-flow of the layer over tau
// (PmlAxis::step, which also advances the memory variable) at positions inside the layer, -tau g elsewhere.
template <typename T, bool K>
__global__ void __launch_bounds__(256) k_nu_vel_pml(T* __restrict__ u, T* __restrict__ c, const T* __restrict__ g,
                                                    const T* __restrict__ b, T b0, T tau, PmlAxis<T> pa, T* mem,
                                                    int64_t px, int nx, int along_x, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int64_t row = i / px;
    const int col = (int)(i - row * px);
    if (col > nx) continue;  // row padding
    const int pos = along_x ? col : (int)row;
    const T gv = g[i];
    const T X = pa.in(pos) ? pa.step(mem, i, pos, gv) : -tau * gv;
    const T delta = (b ? b[i] : b0) * X;
    if constexpr (K) {
      float v = u[i], cc = c[i];
      kahan_add(v, cc, delta);
      u[i] = v;
      c[i] = cc;
    } else {
      u[i] += delta;
    }
  }
}
// sigma += kappa (X_x + X_z) over tau, with the memory variables of both axes.
template <typename T, bool K>
__global__ void __launch_bounds__(256) k_nu_sig_pml(T* __restrict__ u, T* __restrict__ c, const T* __restrict__ gx,
                                                    const T* __restrict__ gz, const T* __restrict__ kappa, T tau,
                                                    PmlAxis<T> pxa, T* memx, PmlAxis<T> pza, T* memz, int64_t px,
                                                    int nx, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int64_t row = i / px;
    const int col = (int)(i - row * px);
    if (col > nx) continue;
    const T ax = gx[i], az = gz[i];
    const T Xx = pxa.in(col) ? pxa.step(memx, i, col, ax) : -tau * ax;
    const T Xz = pza.in((int)row) ? pza.step(memz, i, (int)row, az) : -tau * az;
    const T delta = kappa[i] * (Xx + Xz);
    if constexpr (K) {
      float v = u[i], cc = c[i];
      kahan_add(v, cc, delta);
      u[i] = v;
      c[i] = cc;
    } else {
      u[i] += delta;
    }
  }
}

// Pressure source on knots: sigma += amp gz[oz] gx[ox] over the 25 x 25 knots around the source knot (zs, xs); gz,
// gx: the Gaussian of width 2 h on the physical distance from the source knot (0 off the grid); amp: dt f_r(t)
// times the amplitude over the cell-volume weighted sum of the profile.
struct NuSrc {
  int zs, xs;
  double amp;
  double gz[25], gx[25];
};
template <typename T, bool K>
__global__ void __launch_bounds__(640) k_nu_source(T* __restrict__ u, T* __restrict__ c, NuSrc q, int64_t px) {
  const int i = threadIdx.x;
  if (i >= 625) return;
  const int oz = i / 25, ox = i - 25 * oz;
  const double gz = q.gz[oz], gx = q.gx[ox];
  if (gz == 0.0 || gx == 0.0) return;  // off the grid
  const int64_t gi = (int64_t)(q.zs + oz - 12) * px + (q.xs + ox - 12);
  const T delta = (T)(q.amp * gz * gx);
  if constexpr (K) {
    float v = u[gi], cc = c[gi];
    kahan_add(v, cc, delta);
    u[gi] = v;
    c[gi] = cc;
  } else {
    u[gi] += delta;
  }
}

// The source of step n on knots (slots 0 = z, 2 = x), as above.
static NuSrc nu_source(const Shot& s, int64_t n) {
  NuSrc q{};
  q.zs = (int)s.src_idx[0];
  q.xs = (int)s.src_idx[2];
  double sum[2] = {0.0, 0.0};
  for (int a = 0; a < 2; ++a) {
    const int k = a == 0 ? 0 : 2;
    const int N = (int)s.n[k];
    auto coord = [&](int i) { return s.coords[k].empty() ? s.h[k] * i : s.coords[k][i]; };
    const int i0 = (int)s.src_idx[k];
    const double w = 2.0 * s.h[k];
    double* g = a == 0 ? q.gz : q.gx;
    for (int o = -12; o <= 12; ++o) {
      const int i = i0 + o;
      g[o + 12] = 0.0;
      if (i < 0 || i > N) continue;
      const double d = coord(i) - coord(i0);
      g[o + 12] = std::exp(-d * d / (2.0 * w * w));
      const double v = 0.5 * (coord(std::min(i + 1, N)) - coord(std::max(i - 1, 0)));  // dual cell width
      sum[a] += g[o + 12] * v;
    }
  }
  const double t = (double)n * s.d.dt + 0.5 * s.d.dt;
  const double ar = M_PI * s.src_f0 * (t - s.src_t0);
  const double rk = (1.0 - 2.0 * ar * ar) * std::exp(-ar * ar);
  q.amp = s.d.dt * rk * s.src_amp / (sum[0] * sum[1]);
  return q;
}

loss_status_t nu_ensure_axes(loss_ctx* h, Shot& s) {
  for (int k = 0; k < 3; ++k) {
    if (s.dim == 2 && k == 1) continue;
    if (s.nu_tab[k]) continue;
    std::vector<double> x((size_t)s.n[k] + 1);
    for (size_t i = 0; i < x.size(); ++i) x[i] = s.h[k] * (double)i;
    NU_TRY(nu_upload(h, s, k, x));
  }
  if (!s.tmp[1]) {
    NU_TRY(dev_alloc(h, (size_t)s.total * s.esize, &s.tmp[1]));
    NU_TRY(cuda_check(h, cudaMemsetAsync(s.tmp[1], 0, (size_t)s.total * s.esize, h->stream), "memset"));
  }
  return LOSS_OK;
}

template <typename T, bool K>
static loss_status_t nu_update(loss_ctx* h, Shot& s, int field, const void* g0, const void* g1, const void* coef,
                               double coef0, double scale) {
  const int grid = (int)std::min<int64_t>((s.total + 255) / 256, 8LL * h->num_sms);
  LaunchScope ls(h, LOSS_KERNEL_ACOUSTIC_X2);
  k_nu_update<T, K><<<grid, 256, 0, h->stream>>>((T*)s.field[field], K ? (T*)s.comp[field] : nullptr,
                                                  (const T*)g0, (const T*)g1, (const T*)coef, (T)coef0, (T)scale,
                                                  s.total);
  return cuda_check(h, cudaGetLastError(), "non-uniform update kernel");
}

// Layer coefficients of axis slot k for the sub-step length tau (tables for dt and dt / 2).
template <typename T>
static PmlAxis<T> nu_pml_axis(const Shot& s, int k, double tau) {
  return PmlAxis<T>{(const T*)s.pml_tab[k][tau == s.d.dt ? 0 : 1], s.pml_width, (int)s.n[k], nullptr};
}

template <typename T, bool K>
static loss_status_t nu_step_t(loss_ctx* h, Shot& s) {
  const double dt = s.d.dt;
  T* t0 = (T*)s.tmp[0];
  T* t1 = (T*)s.tmp[1];
  const void* b = s.b_const ? nullptr : s.model[1];
  const int grid = (int)std::min<int64_t>((s.total + 255) / 256, 8LL * h->num_sms);
  const int nx = (int)s.n[2];
  // velocity along slot k over dt / 2 with the layer's sub-flow (memory psi)
  auto vel_pml = [&](int field, const T* g, int k) -> loss_status_t {
    LaunchScope ls(h, LOSS_KERNEL_ACOUSTIC_X2);
    k_nu_vel_pml<T, K><<<grid, 256, 0, h->stream>>>((T*)s.field[field], K ? (T*)s.comp[field] : nullptr, g,
                                                     (const T*)b, (T)s.b0, (T)(0.5 * dt), nu_pml_axis<T>(s, k, 0.5 * dt),
                                                     (T*)s.psi[k], s.px, nx, k == 2 ? 1 : 0, s.total);
    return cuda_check(h, cudaGetLastError(), "non-uniform layer update kernel");
  };
  auto half_A = [&]() -> loss_status_t {
    NU_TRY(nu_launch<T>(h, s, 2, (const T*)s.field[LOSS_FIELD_SIGMA], t0, nullptr, s.sy, s.sz,
                        LOSS_KERNEL_ACOUSTIC_X));
    NU_TRY(nu_launch<T>(h, s, 0, (const T*)s.field[LOSS_FIELD_SIGMA], t1, nullptr, s.sy, s.sz,
                        LOSS_KERNEL_ACOUSTIC_Z));
    if (s.pml_on) {
      NU_TRY(vel_pml(LOSS_FIELD_V1, t0, 2));
      return vel_pml(LOSS_FIELD_V3, t1, 0);
    }
    NU_TRY((nu_update<T, K>(h, s, LOSS_FIELD_V1, t0, nullptr, b, s.b0, -0.5 * dt)));
    return nu_update<T, K>(h, s, LOSS_FIELD_V3, t1, nullptr, b, s.b0, -0.5 * dt);
  };
  NU_TRY(half_A());
  NU_TRY(nu_launch<T>(h, s, 2, (const T*)s.field[LOSS_FIELD_V1], t0, nullptr, s.sy, s.sz, LOSS_KERNEL_ACOUSTIC_X));
  NU_TRY(nu_launch<T>(h, s, 0, (const T*)s.field[LOSS_FIELD_V3], t1, nullptr, s.sy, s.sz, LOSS_KERNEL_ACOUSTIC_Z));
  if (s.pml_on) {
    LaunchScope ls(h, LOSS_KERNEL_ACOUSTIC_X2);
    k_nu_sig_pml<T, K><<<grid, 256, 0, h->stream>>>(
        (T*)s.field[LOSS_FIELD_SIGMA], K ? (T*)s.comp[LOSS_FIELD_SIGMA] : nullptr, t0, t1, (const T*)s.model[0],
        (T)dt, nu_pml_axis<T>(s, 2, dt), (T*)s.phi[2], nu_pml_axis<T>(s, 0, dt), (T*)s.phi[0], s.px, nx, s.total);
    NU_TRY(cuda_check(h, cudaGetLastError(), "non-uniform layer update kernel"));
  } else {
    NU_TRY((nu_update<T, K>(h, s, LOSS_FIELD_SIGMA, t0, t1, s.model[0], 0.0, -dt)));
  }
  if (s.src_on && (s.src_kinds & LOSS_SRC_PRESSURE)) {
    LaunchScope ls(h, LOSS_KERNEL_ACOUSTIC_X2);
    k_nu_source<T, K><<<1, 640, 0, h->stream>>>((T*)s.field[LOSS_FIELD_SIGMA],
                                                 K ? (T*)s.comp[LOSS_FIELD_SIGMA] : nullptr, nu_source(s, s.step), s.px);
    NU_TRY(cuda_check(h, cudaGetLastError(), "non-uniform source kernel"));
  }
  return half_A();
}

loss_status_t nu_step(loss_ctx* h, Shot& s) {
  if (s.d.physics != LOSS_ACOUSTIC || s.dim != 2)
    return fail_msg(h, LOSS_E_UNSUPPORTED, "time steps on non-uniform grids are built for 2-D acoustic grids");
  if (s.src_on && (s.src_kinds & ~(uint32_t)LOSS_SRC_PRESSURE))
    return fail_msg(h, LOSS_E_UNSUPPORTED, "non-uniform grids: pressure sources only");
  NU_TRY(nu_ensure_axes(h, s));
  if (s.esize == 8) return nu_step_t<double, false>(h, s);
  if (s.kahan) return nu_step_t<float, true>(h, s);
  return nu_step_t<float, false>(h, s);
}

template <typename T>
loss_status_t run_nu_derivative_adjoint(loss_ctx* h, Shot& s, int k, const T* g, T* out) {
  NuArgs<T> a{};
  nu_args(s, k, s.len[2], s.len[2] * s.len[1], &a);
  const int64_t nt = a.lines * a.p;
  void* scr = nullptr;
  NU_TRY(dev_alloc(h, (size_t)4 * nt * sizeof(double), &scr));
  LaunchScope ls(h, LOSS_KERNEL_ADJOINT);
  k_nu_adj1<T><<<(unsigned)((nt + 127) / 128), 128, 0, h->stream>>>(a, g, out, (double*)scr);
  loss_status_t st = cuda_check(h, cudaGetLastError(), "non-uniform adjoint kernel");
  if (st == LOSS_OK) {
    const int64_t ne = a.lines * (a.n + 1);
    k_nu_adj2<T><<<(unsigned)((ne + 255) / 256), 256, 0, h->stream>>>(a, out, (const double*)scr);
    st = cuda_check(h, cudaGetLastError(), "non-uniform adjoint kernel");
  }
  dev_free(h, scr);
  return st;
}
template loss_status_t run_nu_derivative_adjoint<float>(loss_ctx*, Shot&, int, const float*, float*);
template loss_status_t run_nu_derivative_adjoint<double>(loss_ctx*, Shot&, int, const double*, double*);

template loss_status_t run_nu_derivative<float>(loss_ctx*, Shot&, int, const float*, float*, double*, float*);
template loss_status_t run_nu_derivative<double>(loss_ctx*, Shot&, int, const double*, double*, double*, double*);

loss_status_t set_coordinates(loss_ctx* h, Shot& s, int k, const double* x) {
  if (!x) {
    if (s.nu_tab[k]) dev_free(h, s.nu_tab[k]);
    s.nu_tab[k] = nullptr;
    s.coords[k].clear();
  } else {
    std::vector<double> xs(x, x + s.n[k] + 1);
    NU_TRY(nu_upload(h, s, k, xs));
    s.coords[k] = xs;
  }
  // the absorbing layer's profiles follow the knots
  return s.pml_on ? pml_upload_tables(h, s) : LOSS_OK;
}

}  // namespace lossk
