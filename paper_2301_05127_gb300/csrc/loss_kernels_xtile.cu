// sm_103a FP32 x part of the 2-D acoustic step for rows of any length, in the truncated-convolution form
// (loss_fir.cuh): one warp per (row, x patch) item.
//
// The derivative at a point of patch l depends only on the field within K positions of it and on the junction
// corrections of the patch's two junctions, whose sums reach Rd = max(n_nb, K) positions beyond them. So a warp
// stages its patch plus Rd positions on each side of one row in shared memory and needs nothing from the other
// warps: no block barrier. The lanes take the patch's 8-position chunks (a second round for M > 256); the two
// junction sums are spread over the lanes and reduced with shuffles in FP64.
//
// Sub-step B (sigma from d_x v1 and the staged d_z v3) and the x part of A (v1 from d_x sigma) need the new sigma
// beyond the patch, so they are two launches: k_xt<B> over every item, then k_xt<A>. The per-point arithmetic is
// that of the whole-row kernel k_xp; this form serves rows that do not fit its shared-memory stages.
#include <cuda_runtime.h>

#include "../../include/loss.h"
#include "loss_fir.cuh"
#include "loss_line.cuh"
#include "loss_tile.cuh"
#include "loss_types.h"

namespace lossk {

constexpr int kXtWarps = 8;  // items per block

// Positions [xb, xb + W) of one row segment, stored from index 0.
struct SegBun {
  int xb;
  __device__ __forceinline__ int at(int, int pos) const { return pos - xb; }
};

__device__ __forceinline__ double warp_sum(double s) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// Junction corrections of junction j of the staged row segment: D = sum_m Wd[j][m] f_{jM+m}, m in [-Rd, Rd]
// clipped to the line, in FP64 over the lanes.
__device__ __forceinline__ float xt_junction(const float* __restrict__ S, const SegBun& bun, const TileGeom& t, int j,
                                             int lane) {
  const int c = j * t.M;
  const int mlo = max(-t.Rd, -c), mhi = min(t.Rd, t.n - c);
  const double* w = t.Wd + (size_t)j * (2 * t.Rd + 1) + t.Rd;
  double s = 0.0;
  for (int m = mlo + lane; m <= mhi; m += 32) s = fma(w[m], widen(S[bun.at(0, c + m)]), s);
  return (float)warp_sum(s);
}

template <bool B, bool KAHAN>
__global__ void __launch_bounds__(32 * kXtWarps, 4) k_xt(AcXArgs<float> a, TileGeom t, int nitems) {
  extern __shared__ __align__(16) float xsm[];
  __shared__ float rpow[kFirPow];
  fill_rpow(rpow, t.r);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int item = blockIdx.x * kXtWarps + warp;
  if (item >= nitems) return;
  const int row = item / t.p, l = item - row * t.p;
  const int n = t.n, M = t.M;
  const int x0 = l * M;
  const bool last = l == t.p - 1;
  const int xb = max(x0 - t.Rd, 0);
  const int xe = min(x0 + M + t.Rd, n);
  const int W = M + 2 * t.Rd + 1;
  float* S = xsm + (size_t)warp * ((W + 3) & ~3);
  const SegBun bun{xb};
  const int64_t rb = (int64_t)row * t.px;
  const float* f = B ? a.v1 : a.sigma;
  for (int pos = xb + lane; pos <= xe; pos += 32) S[pos - xb] = f[rb + pos];
  __syncwarp();
  const float dl[2] = {xt_junction(S, bun, t, l, lane), xt_junction(S, bun, t, l + 1, lane)};
  const int own = M + (last ? 1 : 0);  // the last patch also owns position n
  const int nch = (own + 7) >> 3;
  double amp = 0.0;
  bool srow = false;
  bool zlay = false;
  if (B) {
    amp = a.src.amp_tab ? a.src.amp_tab[a.src.clk->step] : a.src.amp;
    srow = a.src.on && amp != 0.0 && (unsigned)(row - a.src.zs + 12) < 25u;
    zlay = a.pml && a.zB.in(row);
  }
  for (int c = lane; c < nch; c += 32) {
    const int p0 = x0 + 8 * c;
    const int len = min(8, x0 + own - p0);
    float fv[9];
#pragma unroll
    for (int j = 0; j < 9; ++j)
      if (j < len) fv[j] = S[p0 + j - xb];
    const float sL = fir_left<float, FirLen<float>::K>(S, bun, 0, p0, n, t.r);
    const float qR = fir_right<float, FirLen<float>::K>(S, bun, 0, p0 + len - 1, n, t.r);
    float e[9];
    tile_chunk_e<8>(fv, p0, len, x0, t, dl, rpow, sL, qR, e);
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      if (j >= len) break;
      const int pos = p0 + j;
      const int64_t gi = rb + pos;
      const float gx = mulc(e[j], t.s3h, t.s3h_lo);
      if (B) {
        float inc = -mulc(gx, a.dt, a.dt_lo);
        if (a.pml && a.xB.in(pos)) inc = a.xB.step(a.phix, gi, pos, gx);
        const float gzv = a.tmp[gi];
        const float incz = zlay ? a.zB.step(a.phiz, gi, row, gzv) : -mulc(gzv, a.dt, a.dt_lo);
        float delta = a.kappa[gi] * (inc + incz);
        if (srow) {
          const int dx = pos - a.src.xs + 12;
          if ((unsigned)dx < 25u) delta += (float)(amp * a.src.g[row - a.src.zs + 12] * a.src.g[dx]);
        }
        float v = a.sigma[gi];
        if (KAHAN) {
          float cc = a.csig[gi];
          kahan_add(v, cc, delta);
          a.csig[gi] = cc;
        } else {
          v += delta;
        }
        a.sigma[gi] = v;
      } else {
        const float bb = a.b ? a.b[gi] : a.b0;
        float inc;
        if (a.pml && a.xA.in(pos)) {
          const float ih = a.dlt ? a.xA.half(a.psix, gi, pos, gx) : 0.0f;
          inc = a.xA.step(a.psix, gi, pos, gx);
          if (a.dlt) a.dlt[gi] = bb * (ih - 0.5f * inc);
        } else {
          inc = -mulc(gx, a.acoef, a.acoef_lo);
        }
        const float delta = a.b ? bb * inc : mulc(inc, a.b0, a.b0_lo);
        float v = a.v1[gi];
        if (KAHAN) {
          float cc = a.cv1[gi];
          kahan_add(v, cc, delta);
          a.cv1[gi] = cc;
        } else {
          v += delta;
        }
        a.v1[gi] = v;
      }
    }
  }
}

size_t xt_smem(const TileGeom& t) { return (size_t)kXtWarps * (((t.M + 2 * t.Rd + 1) + 3) & ~3) * sizeof(float); }

// Sub-step B (when do_B) and the x part of A over every (row, patch) item, as two launches on stream st.
template <bool KAHAN>
cudaError_t launch_xt(const AcXArgs<float>& a, const TileGeom& t, cudaStream_t st) {
  const int nitems = t.ncross * t.p;
  const int grid = (nitems + kXtWarps - 1) / kXtWarps;
  const size_t smem = xt_smem(t);
  if (a.do_B) {
    if (smem > 48 * 1024) {
      const cudaError_t e = cudaFuncSetAttribute(k_xt<true, KAHAN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
      if (e != cudaSuccess) return e;
    }
    k_xt<true, KAHAN><<<grid, 32 * kXtWarps, smem, st>>>(a, t, nitems);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(k_xt<false, KAHAN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_xt<false, KAHAN><<<grid, 32 * kXtWarps, smem, st>>>(a, t, nitems);
  return cudaGetLastError();
}

template cudaError_t launch_xt<false>(const AcXArgs<float>&, const TileGeom&, cudaStream_t);
template cudaError_t launch_xt<true>(const AcXArgs<float>&, const TileGeom&, cudaStream_t);

}  // namespace lossk
