// Truncated-convolution form of the LOSS first derivative (the local patch solve of Sec. 3.2 closed by the PMBC
// junction values), used by the FP32 time-step kernels.
//
// With r = sqrt(3) - 2 the inverse of the infinite tridiagonal operator (1, 4, 1) has entries r^|i-j| / (2 sqrt 3),
// so one particular solution of e_{i-1} + 4 e_i + e_{i+1} = f_{i+1} - f_{i-1} is
//   eF_i = a (R_i - L_i),  a = (1 - r^2) / (2 sqrt 3),  R_i = sum_{k>=1} r^{k-1} f_{i+k},  L_i = sum_{k>=1} r^{k-1} f_{i-k},
// with L_{i+1} = f_i + r L_i and R_{i-1} = f_i + r R_i.  A thread starts each recursion at its chunk edge from a
// sum truncated after K terms (|r|^K = 7e-10 for K = 16), so chunks need no carries from their neighbours.  The
// patch solution with the PMBC junction values e_{jL} = phi_L, e_{jR} = phi_R is then exact up to that
// truncation:  e_i = eF_i + A r^(i - jL) + B r^(jR - i),  where, with D_L = phi_L - eF_{jL}, D_R = phi_R - eF_{jR}
// and rho = r^M,  A = (D_L - rho D_R) / (1 - rho^2)  and  B = (D_R - rho D_L) / (1 - rho^2).  Beyond the two
// physical ends the line is continued by odd reflection (f_{-k} = 2 f_0 - f_k), which keeps eF close to the
// derivative there so that the corrections stay small.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "loss_line.cuh"

namespace lossk {

constexpr int kFirPow = 64;  // r^d table length; r^d is treated as 0 beyond

// Field value at line position pos (0..n inside), continued by odd reflection beyond the ends.
template <typename T, class BUN>
__device__ __forceinline__ T fir_at(const T* __restrict__ f, const BUN& bun, int l, int pos, int n) {
  if (pos >= 0 && pos <= n) return f[bun.at(l, pos)];
  if (pos < 0) {
    const int q = min(-pos, n);
    return T(2) * f[bun.at(l, 0)] - f[bun.at(l, q)];
  }
  const int q = max(n - (pos - n), 0);
  return T(2) * f[bun.at(l, n)] - f[bun.at(l, q)];
}

// Truncated sums  L = sum_{k=1..K} r^{k-1} f_{pos-k}  and  R = sum_{k=1..K} r^{k-1} f_{pos+k}  (Horner, innermost
// term first).
template <typename T, int K, class BUN>
__device__ __forceinline__ T fir_left(const T* __restrict__ f, const BUN& bun, int l, int pos, int n, T r) {
  T s = T(0);
  if (pos - K >= 0) {
#pragma unroll
    for (int k = K; k >= 1; --k) s = f[bun.at(l, pos - k)] + r * s;
  } else {
    for (int k = K; k >= 1; --k) s = fir_at(f, bun, l, pos - k, n) + r * s;
  }
  return s;
}
template <typename T, int K, class BUN>
__device__ __forceinline__ T fir_right(const T* __restrict__ f, const BUN& bun, int l, int pos, int n, T r) {
  T s = T(0);
  if (pos + K <= n) {
#pragma unroll
    for (int k = K; k >= 1; --k) s = f[bun.at(l, pos + k)] + r * s;
  } else {
    for (int k = K; k >= 1; --k) s = fir_at(f, bun, l, pos + k, n) + r * s;
  }
  return s;
}

// Truncation length: |r|^K below the working precision's rounding (7e-10 for FP32, 1e-16 for FP64).
template <typename T>
struct FirLen {
  static constexpr int K = sizeof(T) == 4 ? 16 : 28;
};

// Contiguous run of up to C + 1 floats starting at a 16-byte aligned address (16-byte accesses where possible).
template <int C>
__device__ __forceinline__ void load_run(const float* __restrict__ p, int len, float (&v)[C + 1]) {
  if ((C % 4) == 0 && len >= C) {
#pragma unroll
    for (int j = 0; j < C; j += 4) {
      const float4 q = *reinterpret_cast<const float4*>(p + j);
      v[j] = q.x, v[j + 1] = q.y, v[j + 2] = q.z, v[j + 3] = q.w;
    }
    if (len > C) v[C] = p[C];
  } else {
#pragma unroll
    for (int j = 0; j <= C; ++j)
      if (j < len) v[j] = p[j];
  }
}
template <int C>
__device__ __forceinline__ void store_run(float* __restrict__ p, int len, const float (&v)[C + 1]) {
  if ((C % 4) == 0 && len >= C) {
#pragma unroll
    for (int j = 0; j < C; j += 4) *reinterpret_cast<float4*>(p + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
    if (len > C) p[C] = v[C];
  } else {
#pragma unroll
    for (int j = 0; j <= C; ++j)
      if (j < len) p[j] = v[j];
  }
}

// Bulk (TMA) copies into shared memory completed on an mbarrier, and bounded waits on it.
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
// 16-byte aligned global source and shared destination, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d),
               "l"(src), "r"(bytes), "r"(b)
               : "memory");
}
// Orders this thread's earlier generic shared-memory accesses before later bulk copies into the same memory.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// Poll limit of the waits that drain a block's own copies in flight after another wait gave up.  The copies were
// issued by the block and complete without it, so this limit only bounds the exit path.
constexpr unsigned kDrainPolls = 1u << 24;
// Waits until the phase with parity `parity` of the barrier has completed; gives up after `limit` polls and then
// returns false (the caller records the failure and stops).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned limit) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  for (unsigned it = 0; it < limit; ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Host-side constants of the truncated-convolution form for patch length M.
struct FirConst {
  double r, a, rho, inv;
};
inline FirConst fir_const(int M) {
  const double r = 1.7320508075688772 - 2.0;  // sqrt(3) - 2
  double rho = 1.0;
  for (int i = 0; i < M; ++i) rho *= r;
  return FirConst{r, (1.0 - r * r) / (2.0 * 1.7320508075688772), rho, 1.0 / (1.0 - rho * rho)};
}

}  // namespace lossk
