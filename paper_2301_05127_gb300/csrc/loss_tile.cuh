// Shared pieces of the FP32 truncated-convolution tile kernels (loss_fir.cuh): one tile is 32 neighbouring
// columns (one per lane) by one patch of a strided axis plus a halo of H = max(n_nb, K) positions on each side,
// staged in shared memory as rows of 32 floats.  Used by the 2-D z tiles and the 3-D elastic y / z tiles.
#ifndef LOSS_TILE_CUH_
#define LOSS_TILE_CUH_

#include <cuda_runtime.h>

#include "loss_fir.cuh"
#include "loss_line.cuh"
#include "loss_types.h"

namespace lossk {

// Shared-memory position of line position pos of z-tile column l (rows of 32 floats from position zb).
struct ZBun {
  int zb;
  __device__ __forceinline__ int at(int l, int pos) const { return (pos - zb) * 32 + l; }
};
// r^d for d < kFirPow - 1; the last entry is 0 (the value used for every d >= kFirPow - 1).  Strided over the
// block: the x blocks of rows with at most 255 intervals hold a single warp, fewer threads than entries.
__device__ __forceinline__ void fill_rpow(float* rpow, float r) {
  for (int i = threadIdx.x; i < kFirPow; i += blockDim.x) {
    float q = 1.0f;
    for (int d = 0; d < i; ++d) q *= r;
    rpow[i] = i == kFirPow - 1 ? 0.0f : q;
  }
}

// z tiles: junction corrections D_j = sum_m Wd[j][m] f_{jM+m}, accumulated in FP64, with the 32 columns on the
// lanes (conflict-free shared-memory rows).  Items (junction J, tap subset sub), ns = min(8, max(1, warps / 2))
// subsets per junction, go round the warps; the partial sums meet in shared memory.  Contains one barrier; dl is
// ready after the caller's next barrier.
// nwj: the warp count that fixes the tap subsets (the single-shot launch's), so that every launch shape sums in the
// same order.
__device__ inline void tile_junctions_z(const float* __restrict__ F, const ZBun& bun, int nvalid, int jg,
                                        const TileGeom& t, int nwj, const double* __restrict__ wsm,
                                        double* __restrict__ partf, float* __restrict__ dl) {
  const int col = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int ns = min(8, max(1, nwj >> 1));
  const int wl = 2 * t.Rd + 1;
  for (int it = w; it < 2 * ns; it += nw) {  // item = (junction J, tap subset sub); a lone warp takes both junctions
    const int J = it & 1, sub = it >> 1;
    const int j = jg + J;
    const int c = j * t.M;
    const int mlo = max(-t.Rd, -c);
    const int mhi = min(t.Rd, t.n - c);
    const double* wj = wsm + J * wl + t.Rd;
    double s = 0.0, s2 = 0.0;  // two independent accumulators halve the FP64 dependency chain
    if (col < nvalid) {
      int m = mlo + sub;
      for (; m + ns <= mhi; m += 2 * ns) {
        s = fma(wj[m], widen(F[bun.at(col, c + m)]), s);
        s2 = fma(wj[m + ns], widen(F[bun.at(col, c + m + ns)]), s2);
      }
      if (m <= mhi) s = fma(wj[m], widen(F[bun.at(col, c + m)]), s);
      s += s2;
    }
    partf[(J * ns + sub) * 32 + col] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 64; i += blockDim.x) {  // (junction, column) pairs; blocks may hold one warp
    const int JJ = i >> 5, cl = i & 31;
    double s = 0.0;
    for (int q = 0; q < ns; ++q) s += partf[(JJ * ns + q) * 32 + cl];
    dl[2 * cl + JJ] = (float)s;
  }
}

// Warm-up partial sums of a chunk's first C values: pa = sum_j r^(C-1-j) f_j (its part of the left sums of the
// chunks after it) and pb = sum_j r^j f_j (its part of the right sums of the chunks before it), in the Horner order
// of fir_left / fir_right.
template <int C>
__device__ __forceinline__ void chunk_partials(const float (&f)[C + 1], float r, float& pa, float& pb) {
  pa = 0.0f;
  pb = 0.0f;
#pragma unroll
  for (int j = 0; j < C; ++j) pa = f[j] + r * pa;
#pragma unroll
  for (int j = C - 1; j >= 0; --j) pb = f[j] + r * pb;
}

// e on the chunk [p0, p0 + len) of line l inside the patch starting at z0 (len <= C + 1), from its values fv and
// the warm-up sums sL = L_{p0} and qR = R_{p0 + len - 1} (fir_left / fir_right, or the neighbours' partial sums).
template <int C>
__device__ __forceinline__ void tile_chunk_e(const float (&fv)[C + 1], int p0, int len, int z0, const TileGeom& t,
                                             const float* __restrict__ dl, const float* __restrict__ rpow, float sL,
                                             float qR, float (&e)[C + 1]) {
  float s = sL;
#pragma unroll
  for (int j = 0; j <= C; ++j)
    if (j < len) {
      e[j] = s;
      s = fv[j] + t.r * s;
    }
  float q = qR;
#pragma unroll
  for (int j = C; j >= 0; --j)
    if (j < len) {
      e[j] = t.a * (q - e[j]);
      q = fv[j] + t.r * q;
    }
  // patch corrections; r^d runs along the chunk by multiplication from the table value at its near end (0 beyond
  // the table)
  const float DT = dl[0], DB = dl[1];
  const float A = (DT - t.rho * DB) * t.inv, B = (DB - t.rho * DT) * t.inv;
  const int d0 = p0 - z0;
  float qa = rpow[min(d0, kFirPow - 1)];                  // r^(d0 + j)
  float qb = rpow[min(t.M - d0 - (len - 1), kFirPow - 1)];  // r^(M - d0 - j), from j = len - 1 down
#pragma unroll
  for (int j = 0; j <= C; ++j)
    if (j < len) {
      e[j] += A * qa;
      qa *= t.r;
    }
#pragma unroll
  for (int j = C; j >= 0; --j)
    if (j < len) {
      e[j] += B * qb;
      qb *= t.r;
    }
}


}  // namespace lossk

#endif  // LOSS_TILE_CUH_
