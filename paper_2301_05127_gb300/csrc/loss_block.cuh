// Block-level helpers shared by the line kernels: shared-memory carve-up, bundle geometry, cp.async staging of
// whole lines, coalesced point iteration and 16-byte vector access.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "loss_line.cuh"
#include "loss_types.h"

namespace lossk {

namespace {

template <typename T>
__device__ __forceinline__ T* align_ptr(void* p) {
  uintptr_t u = reinterpret_cast<uintptr_t>(p);
  u = (u + 15) & ~uintptr_t(15);
  return reinterpret_cast<T*>(u);
}

// Shared-memory carve-up: nbuf padded line buffers, nstage dense staging buffers, two summary arrays, phi,
// line bases.  Must match smem_bytes().
template <typename T>
struct Carve {
  T* buf[6];
  T* stg[4];
  T* sA;
  T* sB;
  double* phi;
  int64_t* lb;
  __device__ Carve(unsigned char* sm, const LineGeom& g, int nbuf, int nstage) {
    T* p = reinterpret_cast<T*>(sm);
    for (int i = 0; i < 6; ++i) {
      buf[i] = p;
      if (i < nbuf) p += g.buf;
    }
    p = align_ptr<T>(p);
    for (int i = 0; i < 4; ++i) {
      stg[i] = p;
      if (i < nstage) p += g.stage;
    }
    const int nw = g.L * g.p * g.NC;
    sA = align_ptr<T>(p);
    sB = sA + nw;
    phi = align_ptr<double>(sB + nw);
    lb = align_ptr<int64_t>(phi + g.L * (g.p + 1));
  }
};

// Line bases of this block's bundle; returns the number of existing lines.
template <bool SFLAV>
__device__ __forceinline__ int bundle_bases(const LineGeom& g, int bundle, int64_t* lb) {
  int nvalid;
  if (SFLAV) {
    const int outer = bundle / g.nxb;
    const int x0 = (bundle - outer * g.nxb) * g.L;
    nvalid = min(g.L, g.nx1 - x0);
    for (int l = threadIdx.x; l < g.L; l += blockDim.x) lb[l] = (int64_t)outer * g.so + x0 + l;
  } else {
    const int64_t r0 = (int64_t)bundle * g.L;
    nvalid = (int)min((int64_t)g.L, g.nrows - r0);
    for (int l = threadIdx.x; l < g.L; l += blockDim.x) {
      const int64_t r = r0 + l;
      lb[l] = (r / g.ny1) * g.sz + (r % g.ny1) * g.sy;
    }
  }
  return nvalid;
}

// Issue cp.async copies of whole lines of a global field into a padded line buffer (no wait).
template <typename T, bool SFLAV, class BUN>
__device__ __forceinline__ void stage_padded(const T* __restrict__ src, T* dst, const BUN& bun, const LineGeom& g,
                                             const int64_t* lb, int nvalid, int logL) {
  const int np = g.n + 1;
  if (SFLAV) {
    const int tot = np << logL;
    for (int i = threadIdx.x; i < tot; i += blockDim.x) {
      const int pos = i >> logL;
      const int l = i & (g.L - 1);
      if (l < nvalid) cp_async<sizeof(T)>(&dst[bun.at(l, pos)], src + lb[l] + (int64_t)pos * g.pstride);
    }
  } else {
    for (int l = 0; l < nvalid; ++l)
      for (int pos = threadIdx.x; pos < np; pos += blockDim.x)
        cp_async<sizeof(T)>(&dst[bun.at(l, pos)], src + lb[l] + pos);
  }
}

// Issue 16-byte cp.async copies of whole rows (X flavour) into a dense staging buffer of pitch g.spitch.
template <typename T>
__device__ __forceinline__ void stage_rows(const T* __restrict__ src, T* dst, const LineGeom& g, const int64_t* lb,
                                           int nvalid) {
  constexpr int V = 16 / sizeof(T);
  const int nchunks = g.spitch / V;
  for (int l = 0; l < nvalid; ++l)
    for (int c = threadIdx.x; c < nchunks; c += blockDim.x) cp_async<16>(dst + l * g.spitch + c * V, src + lb[l] + c * V);
}


// Iterate (line, pos, global offset) over the bundle in a coalesced order and call fn.
template <bool SFLAV, class FN>
__device__ __forceinline__ void for_points(const LineGeom& g, const int64_t* lb, int nvalid, int logL, FN fn) {
  const int np = g.n + 1;
  if (SFLAV) {
    const int tot = np << logL;
    for (int i = threadIdx.x; i < tot; i += blockDim.x) {
      const int pos = i >> logL;
      const int l = i & (g.L - 1);
      if (l < nvalid) fn(l, pos, lb[l] + (int64_t)pos * g.pstride);
    }
  } else {
    for (int l = 0; l < nvalid; ++l)
      for (int pos = threadIdx.x; pos < np; pos += blockDim.x) fn(l, pos, lb[l] + pos);
  }
}

__device__ __forceinline__ int log2_pow2(int L) { return __ffs(L) - 1; }

// Bulk L2 prefetch of a bundle's elements of narr arrays (null entries skipped), so that a later pointwise phase
// finds them in L2: S flavour one segment of L elements per line position (when L elements are a multiple of 16
// bytes), X flavour one padded row per line.  Segments stay within the padded rows.
template <typename T, bool SFLAV>
__device__ __forceinline__ void prefetch_bundle(const LineGeom& g, const int64_t* lb, int nvalid,
                                                const T* const* arrs, int narr) {
  const int np = g.n + 1;
  if (SFLAV) {
    const uint32_t sb = (uint32_t)(g.L * sizeof(T));
    if ((sb & 15u) != 0) return;
    for (int i = threadIdx.x; i < narr * np; i += blockDim.x) {
      const T* base = arrs[i / np];
      if (base) prefetch_l2(base + lb[0] + (int64_t)(i % np) * g.pstride, sb);
    }
  } else {
    const uint32_t rb = (uint32_t)((np * sizeof(T) + 15) & ~(size_t)15);
    for (int i = threadIdx.x; i < narr * nvalid; i += blockDim.x) {
      const T* base = arrs[i / nvalid];
      if (base) prefetch_l2(base + lb[i % nvalid], rb);
    }
  }
}

// Four consecutive elements starting at a 16-byte aligned address.
__device__ __forceinline__ void ld4(const float* p, float (&r)[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  r[0] = t.x, r[1] = t.y, r[2] = t.z, r[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&r)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
  r[0] = a.x, r[1] = a.y, r[2] = b.x, r[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, const float (&r)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(r[0], r[1], r[2], r[3]);
}
__device__ __forceinline__ void st4(double* p, const double (&r)[4]) {
  *reinterpret_cast<double2*>(p) = make_double2(r[0], r[1]);
  *reinterpret_cast<double2*>(p + 2) = make_double2(r[2], r[3]);
}

}  // namespace

// Shot of tile t in a batched launch: the last s with tile0[s] <= t (tile0 ascending, tile0[0] = 0).
__device__ __forceinline__ int tile_shot(const int* __restrict__ tile0, int nshots, int t) {
  int lo = 0, hi = nshots - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tile0[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Block-wide copy of one shot's launch descriptor into shared memory.
template <class A>
__device__ __forceinline__ void copy_args(A* dst, const A* __restrict__ src) {
  static_assert(sizeof(A) % 8 == 0, "descriptor size");
  const uint64_t* s = reinterpret_cast<const uint64_t*>(src);
  uint64_t* d = reinterpret_cast<uint64_t*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(A) / 8); i += blockDim.x) d[i] = s[i];
}

}  // namespace lossk
