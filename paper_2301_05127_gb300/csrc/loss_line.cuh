// Device building blocks of the LOSS derivative along one grid axis, for a bundle of whole grid lines
// held in shared memory by one thread block.
//
// Per line the method (paper Sec. 3.2) needs
//   (1) the PMBC closure phi_j at every junction j = 0..p (ends included):
//         phi_j = sum_m W[j][m] f[jM + m],  m = -n_nb..n_nb  (Eqs. PMBC, PMBC_coeffcients, end closures);
//   (2) per patch the local spline coefficients of Eq. (spline_cofficient_eq_piece) and the derivative
//       d_i = (c_{i+1} - c_{i-1}) / (2h) (Eq. derivative_approximation).
//
// Step (2) is computed without forming c: subtracting collocation rows i-1 and i+1 of the local system gives
//         d_{i-1} + 4 d_i + d_{i+1} = (3/h) (f_{i+1} - f_{i-1}),   i = 1..M-1,
// with d_0 = phi_L and d_M = phi_R from the two Hermite rows.  In scaled form e = d h / 3 this is the
// constant tridiagonal system  e_{i-1} + 4 e_i + e_{i+1} = f_{i+1} - f_{i-1}  with Dirichlet values
// e_0 = phi_L h/3, e_M = phi_R h/3 (the host stores W already multiplied by h/3).  It is solved by the
// Thomas recurrences with the position-only factors m_0 = 1, m_j = 1/u_j, u_1 = 4, u_j = 4 - m_{j-1}:
//         forward   y_i = q_i - m_{i-1} y_{i-1},  y_0 = e_0
//         backward  e_i = m_i (y_i - e_{i+1}),    e_M given
// Each patch line is cut into chunks of C unknowns handled by different threads.  Both recurrences are
// first-order affine, so each chunk first computes its affine summary with a zero carry-in, the carries are
// composed across the chunks of the patch, and each chunk then reruns its recurrence from the true carry.
// This is exact (no truncation beyond the PMBC of the paper); only rounding differs from a serial sweep.
// Factors m_j converge to 2 - sqrt(3) geometrically (ratio ~0.072): from j = 16 on they equal the limit to
// double rounding, so only the first chunk of a patch (C >= 16) reads the table.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lossk {

constexpr int kMaxTable = 64;

// Shared-memory position index with one pad slot every 2^LOGC positions, so that the threads of
// neighbouring chunks (C = 2^LOGC apart) hit different banks.
template <int LOGC>
__device__ __forceinline__ int padpos(int pos) { return pos + (pos >> LOGC); }

// A bundle of whole lines staged in shared memory.
//   X flavour (lines along the contiguous axis): element (line, pos) at line * pitch + padpos(pos).
//   S flavour (lines along a strided axis, neighbouring lines are neighbouring x): at padpos(pos) * pitch + line.
template <int LOGC, bool SFLAV>
struct Bundle {
  int pitch;
  __device__ __forceinline__ int at(int line, int pos) const {
    return SFLAV ? padpos<LOGC>(pos) * pitch + line : line * pitch + padpos<LOGC>(pos);
  }
};

// Work item w <-> (line, patch, chunk).
//   X: w = (line * p + patch) * NC + chunk      (lanes walk consecutive chunks of one line)
//   S: w = (patch * NC + chunk) * L + line      (lanes walk consecutive lines)
template <bool SFLAV>
struct WorkMap {
  int L, p, NC;
  __device__ __forceinline__ void decode(int w, int& line, int& patch, int& chunk) const {
    if (SFLAV) {
      line = w % L;
      int r = w / L;
      chunk = r % NC;
      patch = r / NC;
    } else {
      chunk = w % NC;
      int r = w / NC;
      patch = r % p;
      line = r / p;
    }
  }
  // work item of chunk k of the same (line, patch) as item w with chunk c
  __device__ __forceinline__ int sibling(int w, int c, int k) const { return SFLAV ? w + (k - c) * L : w + (k - c); }
  __device__ __forceinline__ int count() const { return L * p * NC; }
};

template <typename T>
struct Tab;
template <>
struct Tab<float> {
  static __device__ __forceinline__ float m(const float* t32, const double*, int j) { return __ldg(t32 + j); }
};
template <>
struct Tab<double> {
  static __device__ __forceinline__ double m(const float*, const double* t64, int j) { return __ldg(t64 + j); }
};

// PMBC sums phi[line][j] for all lines and junctions of a bundle, accumulated in double.  G threads share
// one (line, junction) and combine partial sums with shuffles.  W is [(p+1)][2 n_nb + 1], already scaled.
template <typename T, int G, class BUN>
__device__ void pmbc_phi(const T* __restrict__ f, const BUN& bun, int L, int nvalid, int n, int p, int M, int n_nb,
                         const double* __restrict__ W, double* __restrict__ phi) {
  const int items = L * (p + 1);
  const int g = threadIdx.x % G;
  const int lane = threadIdx.x & 31;
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  const int wlen = 2 * n_nb + 1;
  for (int it = threadIdx.x / G; it < items; it += blockDim.x / G) {
    const int line = it / (p + 1);
    const int j = it - line * (p + 1);
    const int c = j * M;
    const int mlo = max(-n_nb, -c);
    const int mhi = min(n_nb, n - c);
    double s = 0.0;
    if (line < nvalid) {
      const double* wj = W + (size_t)j * wlen + n_nb;
      for (int m = mlo + g; m <= mhi; m += G) s = fma(__ldg(wj + m), (double)f[bun.at(line, c + m)], s);
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(gmask, s, o, G);
    if (g == 0) phi[it] = s;
  }
}

// First-derivative right-hand side q_i = f_{i+1} - f_{i-1}.
struct RhsD1 {
  template <typename T>
  __device__ __forceinline__ T operator()(T fm1, T f0, T fp1) const { return fp1 - fm1; }
};
// Second-derivative right-hand side q_i = f_{i+1} - 2 f_i + f_{i-1}.
struct RhsD2 {
  template <typename T>
  __device__ __forceinline__ T operator()(T fm1, T f0, T fp1) const { return (fp1 - f0) - (f0 - fm1); }
};

// Solve e_{i-1} + 4 e_i + e_{i+1} = q_i (i = 1..M-1) on every patch of every line of the bundle, with
// Dirichlet values from bnd.left(line, patch) / bnd.right(line, patch).  Writes e_i (i = 1..M-1) into `out`
// at the same (line, position) slots as f; junction slots of `out` are not written.  sA/sB hold two values
// per work item.  Must be called by all threads of the block (contains __syncthreads).
template <typename T, int C, bool SFLAV, class BUN, class RHS, class BND>
__device__ void solve_bundle(const T* __restrict__ f, T* __restrict__ out, T* __restrict__ sA, T* __restrict__ sB,
                             const BUN& bun, const WorkMap<SFLAV>& wm, int nvalid, int M, const float* t32,
                             const double* t64, T minf, RHS rhs, BND bnd) {
  const int nwork = wm.count();
  // Pass 1: forward summaries with zero carry-in.
  for (int w = threadIdx.x; w < nwork; w += blockDim.x) {
    int line, patch, chunk;
    wm.decode(w, line, patch, chunk);
    T P = T(1), y = T(0);
    if (line < nvalid) {
      const int a = 1 + chunk * C;
      const int len = min(C, M - a);
      const int base = patch * M;
      T fm1 = f[bun.at(line, base + a - 1)];
      T f0 = f[bun.at(line, base + a)];
#pragma unroll
      for (int j = 0; j < C; ++j) {
        if (j < len) {
          const T fp1 = f[bun.at(line, base + a + j + 1)];
          const T m = (chunk == 0) ? Tab<T>::m(t32, t64, j) : minf;  // m_{i-1}, i - 1 = chunk*C + j
          y = rhs(fm1, f0, fp1) - m * y;
          P = -m * P;
          fm1 = f0;
          f0 = fp1;
        }
      }
    }
    sA[w] = P;
    sB[w] = y;
  }
  __syncthreads();
  // Pass 2: forward recurrence from the composed carry; y into out.
  for (int w = threadIdx.x; w < nwork; w += blockDim.x) {
    int line, patch, chunk;
    wm.decode(w, line, patch, chunk);
    if (line >= nvalid) continue;
    T y = bnd.left(line, patch);
    for (int k = 0; k < chunk; ++k) {
      const int s = wm.sibling(w, chunk, k);
      y = sB[s] + sA[s] * y;
    }
    const int a = 1 + chunk * C;
    const int len = min(C, M - a);
    const int base = patch * M;
    T fm1 = f[bun.at(line, base + a - 1)];
    T f0 = f[bun.at(line, base + a)];
#pragma unroll
    for (int j = 0; j < C; ++j) {
      if (j < len) {
        const T fp1 = f[bun.at(line, base + a + j + 1)];
        const T m = (chunk == 0) ? Tab<T>::m(t32, t64, j) : minf;
        y = rhs(fm1, f0, fp1) - m * y;
        out[bun.at(line, base + a + j)] = y;
        fm1 = f0;
        f0 = fp1;
      }
    }
  }
  __syncthreads();
  // Pass 3: backward summaries with zero carry-in.
  for (int w = threadIdx.x; w < nwork; w += blockDim.x) {
    int line, patch, chunk;
    wm.decode(w, line, patch, chunk);
    T R = T(1), e = T(0);
    if (line < nvalid) {
      const int a = 1 + chunk * C;
      const int len = min(C, M - a);
      const int base = patch * M;
#pragma unroll
      for (int j = C - 1; j >= 0; --j) {
        if (j < len) {
          const T m = (chunk == 0) ? Tab<T>::m(t32, t64, j + 1) : minf;  // m_i, i = chunk*C + j + 1
          e = m * (out[bun.at(line, base + a + j)] - e);
          R = -m * R;
        }
      }
    }
    sA[w] = R;
    sB[w] = e;
  }
  __syncthreads();
  // Pass 4: backward recurrence from the composed carry; e into out (in place over y).
  for (int w = threadIdx.x; w < nwork; w += blockDim.x) {
    int line, patch, chunk;
    wm.decode(w, line, patch, chunk);
    if (line >= nvalid) continue;
    T e = bnd.right(line, patch);
    for (int k = wm.NC - 1; k > chunk; --k) {
      const int s = wm.sibling(w, chunk, k);
      e = sB[s] + sA[s] * e;
    }
    const int a = 1 + chunk * C;
    const int len = min(C, M - a);
    const int base = patch * M;
#pragma unroll
    for (int j = C - 1; j >= 0; --j) {
      if (j < len) {
        const T m = (chunk == 0) ? Tab<T>::m(t32, t64, j + 1) : minf;
        const int k = bun.at(line, base + a + j);
        e = m * (out[k] - e);
        out[k] = e;
      }
    }
  }
  __syncthreads();
}

// Boundary values e_0 = phi_l, e_M = phi_{l+1} (first derivative).
template <typename T>
struct BndPhi {
  const double* phi;
  int p1;  // p + 1
  __device__ __forceinline__ T left(int line, int patch) const { return (T)phi[line * p1 + patch]; }
  __device__ __forceinline__ T right(int line, int patch) const { return (T)phi[line * p1 + patch + 1]; }
};

// Boundary values of the scaled second derivative s = d2 h^2 / 6 of each patch, from the local collocation
// rows next to the patch ends and the scaled first derivative e (see loss_derivative):
//   s_0 = f_1 - f_0 - 2 e_0 - e_1,   s_M = f_{M-1} - f_M + 2 e_M + e_{M-1}.
template <typename T, class BUN>
struct BndD2 {
  const T* f;
  const T* e;  // e at interior slots
  const double* phi;
  int p1, M;
  BUN bun;
  __device__ __forceinline__ T left(int line, int patch) const {
    const int b = patch * M;
    const T e0 = (T)phi[line * p1 + patch];
    return (f[bun.at(line, b + 1)] - f[bun.at(line, b)]) - T(2) * e0 - e[bun.at(line, b + 1)];
  }
  __device__ __forceinline__ T right(int line, int patch) const {
    const int b = patch * M + M;
    const T eM = (T)phi[line * p1 + patch + 1];
    return (f[bun.at(line, b - 1)] - f[bun.at(line, b)]) + T(2) * eM + e[bun.at(line, b - 1)];
  }
};

// Kahan-compensated u += delta (c carries the negated lost low-order part).
__device__ __forceinline__ void kahan_add(float& u, float& c, float delta) {
  const float y = __fsub_rn(delta, c);
  const float t = __fadd_rn(u, y);
  c = __fsub_rn(__fsub_rn(t, u), y);
  u = t;
}

}  // namespace lossk
