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
  // Offset of position s0 + r from position s0 when s0 is a multiple of 2^LOGC and 0 <= r < 2^(LOGC+1):
  // compile-time for a compile-time r (X flavour) or one multiply (S flavour).
  __device__ __forceinline__ int rel(int r) const { return SFLAV ? (r + (r >> LOGC)) * pitch : r + (r >> LOGC); }
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

// x times a coefficient carried as an unevaluated sum c + c_lo (c: the coefficient rounded to T; c_lo: its rounding
// error, rounded to T; 0 in FP64), to within about one rounding of the product.  A coefficient rounded once to FP32
// (dt, 3 / h, 1 / rho) scales every product of every step by the same factor; over thousands of steps that bias
// becomes a phase drift of the wavefield (a relative error of about omega t times 5e-8), which the second term
// removes.
template <typename T>
__device__ __forceinline__ T mulc(T x, T c, T c_lo) {
  return fma(c_lo, x, c * x);
}

// FP32 -> FP64 widening on the integer units (IEEE 754: binary32 exponent bias 127, binary64 bias 1023, the 23
// fraction bits become the top of the 52).  Exact for normal numbers; zero and subnormals (|f| < 1.2e-38) give 0;
// the all-ones exponent (Inf, NaN) maps to the all-ones binary64 exponent, so a diverged field stays Inf / NaN in
// the FP64 sums.  Keeps the FP64 pipe, which is narrow on this GPU, free for the FMAs of the junction sums.
__device__ __forceinline__ double widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xffu;
  const unsigned ex64 = ex == 0xffu ? 0x7ffu : ex + 896u;
  const unsigned hi = (u & 0x80000000u) | (ex64 << 20) | ((u & 0x7fffffu) >> 3);
  return ex ? __hiloint2double((int)hi, (int)(u << 29)) : 0.0;
}

__device__ __forceinline__ double to_f64(float f) { return widen(f); }
__device__ __forceinline__ double to_f64(double f) { return f; }

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
    double s = 0.0, s2 = 0.0;  // two independent accumulators shorten the FP64 dependency chain
    if (line < nvalid) {
      const double* wj = W + (size_t)j * wlen + n_nb;
      int m = mlo + g;
      for (; m + G <= mhi; m += 2 * G) {
        s = fma(__ldg(wj + m), to_f64(f[bun.at(line, c + m)]), s);
        s2 = fma(__ldg(wj + m + G), to_f64(f[bun.at(line, c + m + G)]), s2);
      }
      if (m <= mhi) s = fma(__ldg(wj + m), to_f64(f[bun.at(line, c + m)]), s);
      s += s2;
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
// Right-hand side q_i = f_i (the symmetric tridiagonal solve of the transposed derivative).
struct RhsId {
  template <typename T>
  __device__ __forceinline__ T operator()(T fm1, T f0, T fp1) const { return f0; }
};
// Second-derivative right-hand side q_i = f_{i+1} - 2 f_i + f_{i-1}.
struct RhsD2 {
  template <typename T>
  __device__ __forceinline__ T operator()(T fm1, T f0, T fp1) const { return (fp1 - f0) - (f0 - fm1); }
};

// Per-block constants of the chunked solve, by chunk class (0: first chunk of a patch, which uses the exact
// leading Thomas factors; 1: a full middle chunk; 2: the last chunk).  For a chunk of length len with local
// forward sweep y_hat (zero carry-in) and local backward sweep e_hat (zero carry-out), the exact solution is
//     y_j = y_hat_j + P_j y_in,        e_j = e_hat_j + alpha_j y_in + beta_j e_out,
// where P_j = prod_{k<=j} (-m_fwd(k)), alpha is the backward sweep applied to P and beta_j = prod (-m_bwd(k)),
// all independent of the data.  Pend = P_{len-1}, A = alpha_0, B = beta_0 summarise a chunk for the carries.
template <typename T, int C>
struct ChunkClasses {
  T alpha[3][C + 1];  // stride C + 1: the three classes fall on different banks
  T beta[3][C + 1];
  T Pend[3], A[3], B[3];
  int len[3];
  T mt[kMaxTable];  // Thomas factors m_0..m_63 in the working precision
};

template <typename T, int C>
__device__ void chunk_classes_init(ChunkClasses<T, C>* cc, int M, int NC, const float* t32, const double* t64,
                                   T minf) {
  for (int j = threadIdx.x; j < kMaxTable; j += blockDim.x) cc->mt[j] = Tab<T>::m(t32, t64, j);
  const int cls = threadIdx.x;
  if (cls < 3) {
    int len;
    if (cls == 0) len = min(C, M - 1);
    else if (cls == 1) len = C;
    else len = (M - 1) - (NC - 1) * C;
    if (cls == 2 && NC == 1) len = min(C, M - 1);
    cc->len[cls] = len;
    T P[C];
    T p = T(1);
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const T m = (cls == 0) ? Tab<T>::m(t32, t64, j) : minf;
      p = -m * p;
      P[j] = p;
    }
    T al = T(0), be = T(1);
#pragma unroll
    for (int j = C - 1; j >= 0; --j) {
      if (j < len) {
        const T m = (cls == 0) ? Tab<T>::m(t32, t64, j + 1) : minf;
        al = m * (P[j] - al);
        be = -m * be;
      }
      cc->alpha[cls][j] = al;
      cc->beta[cls][j] = be;
    }
    T pend = T(1);
#pragma unroll
    for (int j = 0; j < C; ++j)
      if (j < len) pend = P[j];
    cc->Pend[cls] = pend;
    cc->A[cls] = al;
    cc->B[cls] = be;
  }
}

// Solve e_{i-1} + 4 e_i + e_{i+1} = q_i (i = 1..M-1) on every patch of every line of the bundle, with
// Dirichlet values e_0 = bnd.left(line, patch), e_M = bnd.right(line, patch).  Writes e_i for i = 1..M-1 into
// `out` at the (line, position) slots of f, plus the left value at each patch start and the right value at
// the last line end, so `out` holds e at every point of every line.  One work item (chunk) per thread
// (wm.count() <= blockDim.x); sum holds 2 values per work item; cc from chunk_classes_init.  Must be called by
// all threads of the block (contains __syncthreads).
//
// Carries: with y_in(0) = e_0 and y_in(k+1) = Y_k + Pend_k y_in(k) (forward), and
// e_out(NC-1) = e_M, e_out(k-1) = E_k + A_k y_in(k) + B_k e_out(k) (backward), every chunk needs its own y_in
// and e_out.  When the chunks of a (line, patch) are aligned groups of consecutive lanes (X flavour, NC a power
// of two) both recurrences are affine scans done with warp shuffles; otherwise each thread walks the chunk
// summaries in shared memory.
template <typename T, int C, bool SFLAV, class BUN, class RHS, class BND>
__device__ void solve_bundle(const T* __restrict__ f, T* __restrict__ out, T* __restrict__ sum,
                             const ChunkClasses<T, C>* __restrict__ cc, const BUN& bun, const WorkMap<SFLAV>& wm,
                             int nvalid, int M, const float* t32, const double* t64, T minf, RHS rhs, BND bnd) {
  constexpr int LOGC = (C == 32) ? 5 : ((C == 16) ? 4 : 3);
  static_assert((1 << LOGC) == C, "chunk length must be 8, 16 or 32");
  const int nwork = wm.count();
  const int w = threadIdx.x;
  int line = 0, patch = 0, chunk = 0;
  if (w < nwork) wm.decode(w, line, patch, chunk);
  const bool act = w < nwork && line < nvalid;
  const int NC = wm.NC;
  const int cls = (chunk == 0) ? 0 : (chunk == NC - 1 ? 2 : 1);
  const int len = act ? cc->len[cls] : 0;
  const int s0 = patch * M + chunk * C;  // position of the left neighbour of the chunk's first unknown
  const bool fast = (M & (C - 1)) == 0;  // chunk starts are multiples of C: compile-time offsets
  T v[C];
  T yend = T(0), ebeg = T(0);
  if (act) {
    const T* fp = f + bun.at(line, s0);
    T fm1 = fast ? fp[bun.rel(0)] : f[bun.at(line, s0)];
    T f0 = fast ? fp[bun.rel(1)] : f[bun.at(line, s0 + 1)];
    T y = T(0);
#pragma unroll
    for (int j = 0; j < C; ++j) {
      if (j < len) {
        const T fp1 = fast ? fp[bun.rel(j + 2)] : f[bun.at(line, s0 + j + 2)];
        T m = minf;
        if (chunk == 0) m = cc->mt[j];
        y = rhs(fm1, f0, fp1) - m * y;
        v[j] = y;
        fm1 = f0;
        f0 = fp1;
      }
    }
    yend = y;
    T e = T(0);
#pragma unroll
    for (int j = C - 1; j >= 0; --j) {
      if (j < len) {
        T m = minf;
        if (chunk == 0) m = cc->mt[j + 1];
        e = m * (v[j] - e);
        v[j] = e;
      }
    }
    ebeg = e;
  }
  T myin, eout;
  const T left = act ? bnd.left(line, patch) : T(0);
  const T right = act ? bnd.right(line, patch) : T(0);
  const bool shfl = !SFLAV && NC <= 32 && (NC & (NC - 1)) == 0;
  if (shfl) {
    // forward inclusive scan of x -> Y + P x over the NC lanes of the group
    const int g = w & (NC - 1);
    T P = cc->Pend[cls], Y = yend;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      if (d >= NC) break;
      const T Pp = __shfl_up_sync(0xffffffffu, P, d, NC);
      const T Yp = __shfl_up_sync(0xffffffffu, Y, d, NC);
      if (g >= d) {
        Y = Y + P * Yp;
        P = P * Pp;
      }
    }
    const T yout = Y + P * left;  // y at the end of this chunk
    const T yprev = __shfl_up_sync(0xffffffffu, yout, 1, NC);
    myin = (g == 0) ? left : yprev;
    // backward suffix scan of x -> K + B x, K = E + A y_in
    T Bm = cc->B[cls], K = ebeg + cc->A[cls] * myin;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      if (d >= NC) break;
      const T Bn = __shfl_down_sync(0xffffffffu, Bm, d, NC);
      const T Kn = __shfl_down_sync(0xffffffffu, K, d, NC);
      if (g + d < NC) {
        K = K + Bm * Kn;
        Bm = Bm * Bn;
      }
    }
    const T ea = K + Bm * right;  // e at the start of this chunk
    const T enext = __shfl_down_sync(0xffffffffu, ea, 1, NC);
    eout = (g == NC - 1) ? right : enext;
  } else {
    if (act) {
      sum[w] = yend;
      sum[nwork + w] = ebeg;
    }
    __syncthreads();
    T yin = left, acc = T(0), prod = T(1);
    myin = left;
    if (act) {
      for (int k = 0; k < NC; ++k) {
        const int ck = (k == 0) ? 0 : (k == NC - 1 ? 2 : 1);
        const int sk = wm.sibling(w, chunk, k);
        if (k == chunk) myin = yin;
        if (k > chunk) {
          acc += prod * (sum[nwork + sk] + cc->A[ck] * yin);
          prod *= cc->B[ck];
        }
        yin = sum[sk] + cc->Pend[ck] * yin;
      }
    }
    eout = acc + prod * right;
  }
  if (act) {
    T* op = out + bun.at(line, s0);
#pragma unroll
    for (int j = 0; j < C; ++j) {
      if (j < len) {
        const T e = v[j] + cc->alpha[cls][j] * myin + cc->beta[cls][j] * eout;
        if (fast)
          op[bun.rel(j + 1)] = e;
        else
          out[bun.at(line, s0 + j + 1)] = e;
      }
    }
    if (chunk == 0) out[bun.at(line, patch * M)] = left;
    if (chunk == NC - 1 && patch == wm.p - 1) out[bun.at(line, patch * M + M)] = right;
  }
  __syncthreads();
}

// Zero boundary values (transposed derivative: the junction unknowns are not solved for).
template <typename T>
struct BndZero {
  __device__ __forceinline__ T left(int, int) const { return T(0); }
  __device__ __forceinline__ T right(int, int) const { return T(0); }
};

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

// Asynchronous global -> shared copies of 4, 8 or 16 bytes (cp.async); no registers are used and the issuing
// thread does not wait.  cp_async_wait<N>() waits until at most N committed groups are still in flight.
template <int B>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (B == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(s), "l"(gmem), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// floor(pos / M) for 0 <= pos < 65536, 1 <= M < 32768, with magic = ceil(2^32 / M).
__device__ __forceinline__ int div_magic(int pos, unsigned magic) { return (int)__umulhi((unsigned)pos, magic); }

// Asynchronous bulk prefetch of [p, p + bytes) into L2 by the copy engine (bytes a multiple of 16, p 16-byte
// aligned).  Issued at block start for every array a block will touch, so that DRAM streams while the block
// solves; the later loads then hit L2.
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Kahan-compensated u += delta (c carries the negated lost low-order part).
__device__ __forceinline__ void kahan_add(float& u, float& c, float delta) {
  const float y = __fsub_rn(delta, c);
  const float t = __fadd_rn(u, y);
  c = __fsub_rn(__fsub_rn(t, u), y);
  u = t;
}

}  // namespace lossk
