// sm_103a FP32 kernels of the 2-D acoustic step in the truncated-convolution form (loss_fir.cuh), on tiles of
// one patch.
//
// Every output point of the LOSS derivative depends only on the field within its own patch, the K positions
// beyond each patch end (warm-up of the recursions) and the n_nb positions around the patch's two junctions
// (PMBC sums).  A thread block therefore takes one patch of a bundle of lines plus a halo of H >= max(n_nb, K)
// positions on each side; tiles are independent, so no block needs whole lines on chip:
//   z tiles: 32 neighbouring x columns x one patch of z (one 128-byte row segment per z position; a warp is one
//            chunk of C z positions for the 32 columns, so shared-memory accesses are conflict-free),
// The step is three launches: the fused x kernel on whole rows (sub-step B with d_x v1 and the staged d_z v3, then
// the x part of A with d_x sigma), Z1 (z part of A, d_z sigma) and Z2 (d_z v3 for the next step's B) on z tiles.
// A z tile owns the positions [jM, jM + M) of its patch, and the last patch also the line's last point.
#include <cuda_runtime.h>

#include "../../include/loss.h"
#include "loss_block.cuh"
#include "loss_fir.cuh"
#include "loss_line.cuh"
#include "loss_types.h"

namespace lossk {

// Shared-memory position of line position pos of z-tile column l (rows of 32 floats from position zb).
struct ZBun {
  int zb;
  __device__ __forceinline__ int at(int l, int pos) const { return (pos - zb) * 32 + l; }
};
// r^d for d < kFirPow - 1; the last entry is 0 (the value used for every d >= kFirPow - 1).
__device__ __forceinline__ void fill_rpow(float* rpow, float r) {
  if (threadIdx.x < kFirPow) {
    float q = 1.0f;
    for (int d = 0; d < (int)threadIdx.x; ++d) q *= r;
    rpow[threadIdx.x] = threadIdx.x == kFirPow - 1 ? 0.0f : q;
  }
}

// z tiles: junction corrections D_j = sum_m Wd[j][m] f_{jM+m}, accumulated in FP64, with the 32 columns on the
// lanes (conflict-free shared-memory rows).  Items (junction J, tap subset sub), ns = min(8, max(1, warps / 2))
// subsets per junction, go round the warps; the partial sums meet in shared memory.  Contains one barrier; dl is
// ready after the caller's next barrier.
__device__ void tile_junctions_z(const float* __restrict__ F, const ZBun& bun, int nvalid, int jg, const TileGeom& t,
                                 const double* __restrict__ wsm, double* __restrict__ partf, float* __restrict__ dl) {
  const int col = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int ns = min(8, max(1, nw >> 1));
  const int wl = 2 * t.Rd + 1;
  for (int it = w; it < 2 * ns; it += nw) {  // item = (junction J, tap subset sub); a lone warp takes both junctions
    const int J = it & 1, sub = it >> 1;
    const int j = jg + J;
    const int c = j * t.M;
    const int mlo = max(-t.Rd, -c);
    const int mhi = min(t.Rd, t.n - c);
    const double* wj = wsm + J * wl + t.Rd;
    double s = 0.0;
    if (col < nvalid)
      for (int m = mlo + sub; m <= mhi; m += ns) s = fma(wj[m], widen(F[bun.at(col, c + m)]), s);
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

// e on the chunk [p0, p0 + len) of line l inside the patch starting at z0 (len <= C + 1).
template <int C, class BUN>
__device__ __forceinline__ void tile_chunk(const float* __restrict__ F, const BUN& bun, int l, int p0, int len,
                                           int z0, const TileGeom& t, const float* __restrict__ dl,
                                           const float* __restrict__ rpow, float (&e)[C + 1]) {
  constexpr int K = FirLen<float>::K;
  float fv[C + 1];
#pragma unroll
  for (int j = 0; j <= C; ++j)
    if (j < len) fv[j] = F[bun.at(l, p0 + j)];
  float s = fir_left<float, K>(F, bun, l, p0, t.n, t.r);
#pragma unroll
  for (int j = 0; j <= C; ++j)
    if (j < len) {
      e[j] = s;
      s = fv[j] + t.r * s;
    }
  float q = fir_right<float, K>(F, bun, l, p0 + len - 1, t.n, t.r);
#pragma unroll
  for (int j = C; j >= 0; --j)
    if (j < len) {
      e[j] = t.a * (q - e[j]);
      q = fv[j] + t.r * q;
    }
  const float DT = dl[0], DB = dl[1];
  const float A = (DT - t.rho * DB) * t.inv, B = (DB - t.rho * DT) * t.inv;
  const int d0 = p0 - z0;
#pragma unroll
  for (int j = 0; j <= C; ++j)
    if (j < len) e[j] += A * rpow[min(d0 + j, kFirPow - 1)] + B * rpow[min(t.M - d0 - j, kFirPow - 1)];
}

// ---------------------------------------------------------------------------------------------------------------
// z tiles.  MODE 1 (Z1): v3 += b * (z part of A) from d_z sigma.  MODE 2 (Z2): tmp = d_z v3.
template <int MODE, bool KAHAN, int LOGC>
__global__ void __launch_bounds__(1024) k_tz(AcZArgs<float> a, TileGeom t) {
  constexpr int C = 1 << LOGC;
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ float rpow[kFirPow];
  __shared__ float dl[64];
  __shared__ double jpart[16 * 32];   // junction partial sums [2 x up to 8 subsets][32 columns]
  __shared__ double wsm[2 * 129];     // the two junctions' correction weights (Rd <= 64)
  const int l = blockIdx.x % t.p;                  // patch
  const int cg = blockIdx.x / t.p;                 // column group
  const int x0 = cg * 32;
  const int z0 = l * t.M;
  const int zb = z0 - t.H;
  const int rows = t.M + 2 * t.H + 1;
  const bool last = l == t.p - 1;
  float* F = reinterpret_cast<float*>(sm);         // [rows][32]
  float* SV = F + rows * 32;                       // MODE 1: v3 of the own rows [M + 1][32]
  float* SC = SV + (t.M + 1) * 32;                 //         compensation of v3
  const float* f = MODE == 1 ? a.sigma : a.v3;
  fill_rpow(rpow, t.r);
  {
    const int wl = 2 * t.Rd + 1;
    for (int i = threadIdx.x; i < 2 * wl; i += blockDim.x) wsm[i] = t.Wd[(size_t)l * wl + i];
  }
  for (int i = threadIdx.x; i < rows * 8; i += blockDim.x) {
    const int q = i >> 3, seg = i & 7;
    const int pos = zb + q;
    if (pos >= 0 && pos <= t.n) cp_async<16>(F + q * 32 + seg * 4, f + (int64_t)pos * t.px + x0 + seg * 4);
  }
  if (MODE == 1) {
    for (int i = threadIdx.x; i < (t.M + 1) * 8; i += blockDim.x) {
      const int q = i >> 3, seg = i & 7;
      const int pos = z0 + q;
      if (pos <= t.n) {
        cp_async<16>(SV + q * 32 + seg * 4, a.v3 + (int64_t)pos * t.px + x0 + seg * 4);
        if (KAHAN) cp_async<16>(SC + q * 32 + seg * 4, a.cv3 + (int64_t)pos * t.px + x0 + seg * 4);
      }
    }
  }
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  const ZBun bun{zb};
  const int nvalid = min(32, t.ncross - x0);
  tile_junctions_z(F, bun, nvalid, l, t, wsm, jpart, dl);
  __syncthreads();
  const int col = threadIdx.x & 31;
  const int c = threadIdx.x >> 5;
  const int p0 = z0 + c * C;
  int len = min(C, z0 + t.M - p0);
  if (last && p0 + len == t.n) ++len;  // the line's last point
  if (col >= nvalid || len <= 0) return;
  float e[C + 1];
  tile_chunk<C>(F, bun, col, p0, len, z0, t, dl + 2 * col, rpow, e);
  const int64_t base = x0 + col;
#pragma unroll
  for (int j = 0; j <= C; ++j) {
    if (j >= len) break;
    const int pos = p0 + j;
    const int64_t gi = (int64_t)pos * t.px + base;
    const float gz = t.s3h * e[j];
    if (MODE == 2) {
      a.tmp[gi] = gz;
      continue;
    }
    const float bb = a.b ? a.b[gi] : a.b0;
    float inc;
    if (a.pml && a.zA.in(pos)) {
      const float ih = a.dlt ? a.zA.half(a.psiz, gi, pos, gz) : 0.0f;
      inc = a.zA.step(a.psiz, gi, pos, gz);
      if (a.dlt) a.dlt[gi] = bb * (ih - 0.5f * inc);
    } else {
      inc = -a.acoef * gz;
    }
    const float delta = bb * inc;
    const int k = (pos - z0) * 32 + col;
    float v = SV[k];
    if (KAHAN) {
      float cc = SC[k];
      kahan_add(v, cc, delta);
      a.cv3[gi] = cc;
    } else {
      v += delta;
    }
    a.v3[gi] = v;
  }
}

// ---------------------------------------------------------------------------------------------------------------
// Fused x kernel (FP32): whole rows, sub-step B then the x part of A, as the line kernel, but with chunk-owned
// threads (8 positions each) and rows stored in 12-float slots per 8-position chunk, so that every shared-memory
// access of a chunk and of its warm-up neighbours is a 16-byte vector without bank conflicts, and all global
// traffic is 16-byte cp.async loads and 16-byte stores.
// Plain contiguous rows (bulk-copied): position pos at row[pos].
struct PlainBun {
  __device__ __forceinline__ int at(int, int pos) const { return pos; }
};
// Eight values of chunk s.  Lanes of chunks with (s >> 2) odd read the two 16-byte halves in the other order, so the
// eight lanes of a quarter warp (chunks 32 bytes apart) hit disjoint banks.
__device__ __forceinline__ void plain8(const float* __restrict__ row, int s, float (&v)[8]) {
  const int h = (s >> 2) & 1;
  const float4 a = *reinterpret_cast<const float4*>(row + s * 8 + 4 * h);
  const float4 b = *reinterpret_cast<const float4*>(row + s * 8 + 4 - 4 * h);
  const float4 lo = h ? b : a, hi = h ? a : b;
  v[0] = lo.x, v[1] = lo.y, v[2] = lo.z, v[3] = lo.w, v[4] = hi.x, v[5] = hi.y, v[6] = hi.z, v[7] = hi.w;
}
__device__ __forceinline__ void plain8_store(float* row, int s, const float (&v)[9]) {
  const int h = (s >> 2) & 1;
  const float4 lo = make_float4(v[0], v[1], v[2], v[3]), hi = make_float4(v[4], v[5], v[6], v[7]);
  *reinterpret_cast<float4*>(row + s * 8 + 4 * h) = h ? hi : lo;
  *reinterpret_cast<float4*>(row + s * 8 + 4 - 4 * h) = h ? lo : hi;
}
struct PlainLayout {
  PlainBun bun;
  __device__ __forceinline__ void eight(const float* row, int s, float (&v)[8]) const { plain8(row, s, v); }
  __device__ __forceinline__ void store8(float* row, int s, const float (&v)[9]) const { plain8_store(row, s, v); }
  __device__ __forceinline__ int chunk(int s) const { return s * 8; }
};

// Warm-up partial sums of chunk c (first eight values): PA = sum_j r^{7-j} f_{8c+j} (its part of the left sum of
// chunks c + 1 and c + 2) and PB = sum_j r^j f_{8c+j} (its part of the right sum of chunks c - 1 and c - 2), in
// the Horner order the consumers would use.
__device__ __forceinline__ void xf_partials(const float (&f)[8], float r, float& pa, float& pb) {
  pa = 0.0f;
  pb = 0.0f;
#pragma unroll
  for (int j = 0; j < 8; ++j) pa = f[j] + r * pa;
#pragma unroll
  for (int j = 7; j >= 0; --j) pb = f[j] + r * pb;
}

// e on chunk c of the row (positions 8c .. 8c + len - 1, len = 8, or 9 for the chunk ending at n).
template <class LAY>
__device__ __forceinline__ void xf_chunk(const float* __restrict__ row, const LAY& lay, int c, int len,
                                         const TileGeom& t, int M, unsigned mmagic, const float* __restrict__ dlf,
                                         const float* __restrict__ rpow, const float* __restrict__ PA,
                                         const float* __restrict__ PB, float (&e)[9]) {
  constexpr int K = FirLen<float>::K;  // 16 = two slots
  const int p0 = c << 3;
  const float r = t.r;
  float fv[9];
  {
    float v8[8];
    lay.eight(row, c, v8);
#pragma unroll
    for (int j = 0; j < 8; ++j) fv[j] = v8[j];
    fv[8] = (len > 8) ? row[lay.chunk(c + 1)] : 0.0f;
  }
  float s = 0.0f;
  if (p0 >= K) {
    // L = sum_{k=1..16} r^{k-1} f_{p0-k}: chunk c-1 gives the terms k = 1..8, chunk c-2 those of k = 9..16
    s = PA[c - 1] + rpow[8] * PA[c - 2];
  } else {
    s = fir_left<float, K>(row, lay.bun, 0, p0, t.n, r);
  }
#pragma unroll
  for (int j = 0; j < 9; ++j)
    if (j < len) {
      e[j] = s;
      s = fv[j] + r * s;
    }
  float q = 0.0f;
  const int pe = p0 + len - 1;
  if (len == 8 && pe + K <= t.n) {
    q = PB[c + 1] + rpow[8] * PB[c + 2];
  } else {
    q = fir_right<float, K>(row, lay.bun, 0, pe, t.n, r);
  }
#pragma unroll
  for (int j = 8; j >= 0; --j)
    if (j < len) {
      e[j] = t.a * (q - e[j]);
      q = fv[j] + r * q;
    }
  // patch corrections: the chunk (and its ninth point, the line's end) lies in one patch since M is a multiple
  // of 8; r^d runs along the chunk by multiplication from the table value at its near end (0 beyond the table)
  const int pt = min((int)div_magic(p0, mmagic), t.p - 1);
  const float DL = dlf[pt], DR = dlf[pt + 1];
  const float A = (DL - t.rho * DR) * t.inv, B = (DR - t.rho * DL) * t.inv;
  const int d0 = p0 - pt * M;
  const int dB = M - d0 - (len - 1);
  float qa = rpow[min(d0, kFirPow - 1)];  // r^(d0 + j)
  float qb = rpow[min(dB, kFirPow - 1)];  // r^(M - d0 - j), from j = len - 1 down
#pragma unroll
  for (int j = 0; j < 9; ++j)
    if (j < len) {
      e[j] += A * qa;
      qa *= r;
    }
#pragma unroll
  for (int j = 8; j >= 0; --j)
    if (j < len) {
      e[j] += B * qb;
      qb *= r;
    }
}

// Junction corrections of one row: D_j = sum_m Wd[j][m] f_{jM+m}, accumulated in FP64 (the weights hold the PMBC
// weights minus the convolution's own junction weights), G lanes per junction.
template <int G, class BUN>
__device__ void xf_junctions(const float* __restrict__ row, const BUN& bun, const TileGeom& t,
                             const double* __restrict__ wd, float* __restrict__ dlf) {
  const int g = threadIdx.x % G;
  const int lane = threadIdx.x & 31;
  const unsigned gmask = (((1u << G) - 1u) << (lane & ~(G - 1)));
  const int wl = 2 * t.Rd + 1;
  for (int j = threadIdx.x / G; j <= t.p; j += blockDim.x / G) {
    const int c = j * t.M;
    const int mlo = max(-t.Rd, -c);
    const int mhi = min(t.Rd, t.n - c);
    const double* wj = wd + (size_t)j * wl + t.Rd;
    double s = 0.0;
    for (int m = mlo + g; m <= mhi; m += G) s = fma(wj[m], widen(row[bun.at(0, c + m)]), s);
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(gmask, s, o, G);
    if (g == 0) dlf[j] = (float)s;
  }
}

// Layer segments of an x-axis memory variable staged with a row: positions [0, W) and [R0, R0 + SR) (R0 = the
// layer start n + 1 - W rounded down to 16 bytes).
struct MemSeg {
  int W, SL, R0, SR;
  __device__ __forceinline__ int at(int pos) const { return pos < W ? pos : SL + (pos - R0); }
  __device__ __forceinline__ int floats() const { return SL + SR; }
};
__device__ __forceinline__ MemSeg mem_seg(int n, int W) {
  MemSeg m;
  m.W = W;
  m.SL = (W + 3) & ~3;
  m.R0 = (n + 1 - W) & ~3;
  m.SR = (n + 1 - m.R0 + 3) & ~3;
  return m;
}
// PmlAxis::step / ::half with the memory value before the sub-step given and the coefficients from a staged table
// T[4][F] at slot sl (same arithmetic).
__device__ __forceinline__ float pml_step_s(const float* T, int F, int sl, float m0, float g, float* mem,
                                            int64_t gi) {
  const float m1 = T[sl] * m0 - T[F + sl] * g;
  mem[gi] = m1;
  return T[2 * F + sl] * (m1 - m0) - T[3 * F + sl] * g;
}
__device__ __forceinline__ float pml_half_s(const float* T, int F, int sl, float m0, float g) {
  const float m1 = T[sl] * m0 - T[F + sl] * g;
  return T[2 * F + sl] * (m1 - m0) - T[3 * F + sl] * g;
}

// Chunks of a row that go through the one-point-per-thread pass: the absorbing-layer chunks [0, cL) and [cR, nch)
// and, on rows of the source block, the chunks [s0, s1] between them that the source touches.  Ordinal k numbers
// them in that order; their derivative values wait in O[9 k + j].
struct SlowSet {
  int cL, cR, nr, s0, s1;  // nr = nch - cR
  __device__ __forceinline__ int count() const { return cL + nr + (s1 >= s0 ? s1 - s0 + 1 : 0); }
  __device__ __forceinline__ int chunk(int k) const {
    return k < cL ? k : (k < cL + nr ? cR + (k - cL) : s0 + (k - cL - nr));
  }
  __device__ __forceinline__ int ordinal(int c) const {
    if (c < cL) return c;
    if (c >= cR) return cL + (c - cR);
    return (c >= s0 && c <= s1) ? cL + nr + (c - s0) : -1;
  }
};
// W: layer width (0: no layer); src: the row crosses the source block, whose x extent is xs - 12 .. xs + 12.
__device__ __forceinline__ SlowSet slow_set(int n, int nch, int W, bool src, int xs) {
  SlowSet s;
  if (W > 0) {
    s.cL = min((W + 7) >> 3, nch);                             // chunks starting before W
    s.cR = max(min(max(n - W + 1, 0) >> 3, nch - 1), s.cL);  // first chunk reaching past n - W
  } else {
    s.cL = 0;
    s.cR = nch;
  }
  s.nr = nch - s.cR;
  s.s0 = 1;
  s.s1 = 0;
  if (src) {  // the last chunk also holds position n
    const int lo = xs - 12, hi = xs + 12;
    if (lo <= n) {
      s.s0 = max(lo < 0 ? 0 : min(lo >> 3, nch - 1), s.cL);
      s.s1 = min(hi < 0 ? -1 : hi >> 3, s.cR - 1);
    }
  }
  return s;
}

// One row of the fused x step (sub-step B, then the x part of A) from rows already in shared memory (layout LAY).
// Contains barriers: every thread of the block must call it.
template <bool KAHAN, class LAY>
__device__ __forceinline__ void xrow(const AcXArgs<float>& a, const TileGeom& t, unsigned mmagic, int row,
                                     const LAY& lay, float* V, float* D, const float* SK, const float* ST,
                                     const float* SC, const float* SV, float* O, const float* rpow,
                                     const double* wd, float* dlf, const MemSeg& ms, const float* segB,
                                     const float* segA, float* PA, float* PB, const float* tabs) {
  const int n = t.n, np = n + 1;
  const int M = t.M;
  const int64_t rb = (int64_t)row * t.px;
  const int nch = (n + 7) >> 3;
  const int c = threadIdx.x;
  const int len = (c == nch - 1) ? np - (c << 3) : 8;
  const int p0 = c << 3;
  const bool act = c < nch;
  // Points of chunks in an x absorbing layer or in the source block go through a second pass with one point per
  // thread (its table reads come from shared memory and its memory-variable loads are independent); the chunk pass
  // handles the others in registers, including the z memory variable of rows in a z layer.
  auto chunk_len = [&](int cc) { return (cc == nch - 1) ? np - (cc << 3) : 8; };
  const int F = ms.floats();
  if (a.do_B) {
    const double amp = a.src.amp_tab ? a.src.amp_tab[a.src.clk->step] : a.src.amp;
    const bool son = a.src.on && amp != 0.0;
    const bool zlay = a.pml && a.zB.in(row);
    const bool srow = son && (unsigned)(row - a.src.zs + 12) < 25u;
    const SlowSet SB = slow_set(n, nch, a.pml ? a.xB.width : 0, srow, a.src.xs);
    if (act) {
      float f8[8];
      lay.eight(V, c, f8);
      xf_partials(f8, t.r, PA[c], PB[c]);
    }
    xf_junctions<8>(V, lay.bun, t, wd, dlf);
    __syncthreads();
    if (act) {
      float e[9];
      xf_chunk(V, lay, c, len, t, M, mmagic, dlf, rpow, PA, PB, e);
      const int ob = SB.ordinal(c);
      if (ob >= 0) {
#pragma unroll
        for (int j = 0; j < 9; ++j)
          if (j < len) O[9 * ob + j] = t.s3h * e[j];
      } else {
        float sg[9], cs[9], kp[9], gz[9], iz[9];
        {
          float v8[8];
          lay.eight(D, c, v8);
#pragma unroll
          for (int j = 0; j < 8; ++j) sg[j] = v8[j];
          lay.eight(SK, c, v8);
#pragma unroll
          for (int j = 0; j < 8; ++j) kp[j] = v8[j];
          lay.eight(ST, c, v8);
#pragma unroll
          for (int j = 0; j < 8; ++j) gz[j] = v8[j];
          if (KAHAN) {
            lay.eight(SC, c, v8);
#pragma unroll
            for (int j = 0; j < 8; ++j) cs[j] = v8[j];
          }
          if (len > 8) {
            const int k8 = lay.chunk(c + 1);
            sg[8] = D[k8], kp[8] = SK[k8], gz[8] = ST[k8];
            if (KAHAN) cs[8] = SC[k8];
          }
        }
        if (zlay) {  // z memory variable of this row (PmlAxis::step, vectorised)
          float pz[9];
          load_run<8>(a.phiz + rb + p0, len, pz);
          const int n1z = a.zB.n + 1;
          const float T0 = a.zB.tab[row], T1 = a.zB.tab[n1z + row], T2 = a.zB.tab[2 * n1z + row],
                      T3 = a.zB.tab[3 * n1z + row];
#pragma unroll
          for (int j = 0; j < 9; ++j) {
            const float m1 = T0 * pz[j] - T1 * gz[j];
            iz[j] = T2 * (m1 - pz[j]) - T3 * gz[j];
            pz[j] = m1;
          }
          store_run<8>(a.phiz + rb + p0, len, pz);
        } else {
#pragma unroll
          for (int j = 0; j < 9; ++j) iz[j] = -a.dt * gz[j];
        }
#pragma unroll
        for (int j = 0; j < 9; ++j) {
          if (j >= len) break;
          const float delta = kp[j] * (-a.dt * (t.s3h * e[j]) + iz[j]);
          float v = sg[j];
          if (KAHAN) {
            float cc = cs[j];
            kahan_add(v, cc, delta);
            cs[j] = cc;
          } else {
            v += delta;
          }
          sg[j] = v;
        }
        lay.store8(D, c, sg);
        if (len > 8) D[lay.chunk(c + 1)] = sg[8];
        store_run<8>(a.sigma + rb + p0, len, sg);
        if (KAHAN) store_run<8>(a.csig + rb + p0, len, cs);
      }
    }
    __syncthreads();
    const int nsB = 9 * SB.count();
    for (int q = threadIdx.x; q < nsB; q += blockDim.x) {
      const int kq = q / 9, j = q - 9 * kq;
      const int ch = SB.chunk(kq);
      if (j >= chunk_len(ch)) continue;
      const int pos = (ch << 3) + j;
      const int64_t gi = rb + pos;
      const int k = lay.bun.at(0, pos);
      const float gx = O[q];
      const float gzv = ST[k];
      float inc = -a.dt * gx;
      if (a.pml && a.xB.in(pos)) {
        const int sl = ms.at(pos);
        inc = pml_step_s(tabs, F, sl, segB[sl], gx, a.phix, gi);
      }
      const float incz = zlay ? a.zB.step(a.phiz, gi, row, gzv) : -a.dt * gzv;
      float delta = SK[k] * (inc + incz);
      if (srow) {
        const int dx = pos - a.src.xs + 12;
        if ((unsigned)dx < 25u) delta += (float)(amp * a.src.g[row - a.src.zs + 12] * a.src.g[dx]);
      }
      float v = D[k];
      if (KAHAN) {
        float cc = SC[k];
        kahan_add(v, cc, delta);
        a.csig[gi] = cc;
      } else {
        v += delta;
      }
      D[k] = v;
      a.sigma[gi] = v;
    }
    __syncthreads();
  }
  const SlowSet SA = slow_set(n, nch, a.pml ? a.xA.width : 0, false, 0);
  if (act) {
    float f8[8];
    lay.eight(D, c, f8);
    xf_partials(f8, t.r, PA[c], PB[c]);
  }
  xf_junctions<8>(D, lay.bun, t, wd, dlf);
  __syncthreads();
  if (act) {
    float e[9];
    xf_chunk(D, lay, c, len, t, M, mmagic, dlf, rpow, PA, PB, e);
    const int oa = SA.ordinal(c);
    if (oa >= 0) {
#pragma unroll
      for (int j = 0; j < 9; ++j)
        if (j < len) O[9 * oa + j] = t.s3h * e[j];
    } else {
      float vv[9], cs[9], bb[9];
      {
        float v8[8];
        lay.eight(V, c, v8);
#pragma unroll
        for (int j = 0; j < 8; ++j) vv[j] = v8[j];
        if (KAHAN) {
          lay.eight(SV, c, v8);
#pragma unroll
          for (int j = 0; j < 8; ++j) cs[j] = v8[j];
        }
        if (len > 8) {
          vv[8] = V[lay.chunk(c + 1)];
          if (KAHAN) cs[8] = SV[lay.chunk(c + 1)];
        }
      }
#pragma unroll
      for (int j = 0; j < 9; ++j) bb[j] = (a.b && j < len) ? a.b[rb + p0 + j] : a.b0;
#pragma unroll
      for (int j = 0; j < 9; ++j) {
        if (j >= len) break;
        const float delta = bb[j] * (-a.acoef * (t.s3h * e[j]));
        float v = vv[j];
        if (KAHAN) {
          float cc = cs[j];
          kahan_add(v, cc, delta);
          cs[j] = cc;
        } else {
          v += delta;
        }
        vv[j] = v;
      }
      store_run<8>(a.v1 + rb + p0, len, vv);
      if (KAHAN) store_run<8>(a.cv1 + rb + p0, len, cs);
    }
  }
  __syncthreads();
  const int nsA = 9 * SA.count();
  for (int q = threadIdx.x; q < nsA; q += blockDim.x) {
    const int kq = q / 9, j = q - 9 * kq;
    const int ch = SA.chunk(kq);
    if (j >= chunk_len(ch)) continue;
    const int pos = (ch << 3) + j;
    const int64_t gi = rb + pos;
    const int k = lay.bun.at(0, pos);
    const float gx = O[q];
    const float bb = a.b ? a.b[gi] : a.b0;
    float inc;
    if (a.xA.in(pos)) {
      const int sl = ms.at(pos);
      const float m0 = segA[sl];
      const float ih = a.dlt ? pml_half_s(tabs + 8 * F, F, sl, m0, gx) : 0.0f;
      inc = pml_step_s(tabs + 4 * F, F, sl, m0, gx, a.psix, gi);
      if (a.dlt) a.dlt[gi] = bb * (ih - 0.5f * inc);
    } else {
      inc = -a.acoef * gx;
    }
    const float delta = bb * inc;
    float v = V[k];
    if (KAHAN) {
      float cc = SV[k];
      kahan_add(v, cc, delta);
      a.cv1[gi] = cc;
    } else {
      v += delta;
    }
    a.v1[gi] = v;
  }
}

// Dynamic shared memory of k_xp, in floats: 2 stages x 6 staged rows, the slow chunks' derivative values O, the
// junction-correction weights (FP64), 2 stages x 2 layer segments of the x memory variables, the warm-up partial
// sums, and the x layer's coefficient tables (B step, A step, A half step; 4 rows each) at the segment slots.
struct XpSmem {
  int RW, O, WS, SEG, PA, TAB, total;
};
__host__ __device__ inline XpSmem xp_layout(int n, int p, int Rd, int pw) {
  XpSmem L;
  L.RW = (n + 1 + 3) & ~3;
  const int W = pw > 0 ? pw : 4;
  const int SL = (W + 3) & ~3, R0 = (n + 1 - W) & ~3, SR = (n + 1 - R0 + 3) & ~3;  // as mem_seg
  const int nw = (p + 1) * (2 * Rd + 1);
  L.O = 12 * L.RW;
  L.WS = L.O + (((2 * ((pw + 7) / 8 + 2) + 5) * 9 + 3) & ~3);
  L.SEG = L.WS + 2 * ((nw + 1) & ~1);
  L.PA = L.SEG + 4 * (SL + SR);
  L.TAB = L.PA + ((2 * ((n + 7) / 8 + 8) + 3) & ~3);
  L.total = L.TAB + (pw > 0 ? 12 * (SL + SR) : 0);
  return L;
}

// Persistent, software-pipelined form: each block takes rows blockIdx.x, blockIdx.x + gridDim.x, ...; one thread
// bulk-copies (TMA) the next row's arrays into the other of two shared-memory stages while the block computes the
// current row, so HBM streams while the block computes.  Waits on the stage barriers are bounded: on a timeout
// the block records it in *err, waits (bounded) for its copy in flight and stops.
template <bool KAHAN>
__global__ void __launch_bounds__(256, 2) k_xp(AcXArgs<float> a, TileGeom t, unsigned mmagic, int* err) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ float rpow[kFirPow];
  __shared__ float dlf[65];
  __shared__ __align__(8) uint64_t bar[2];
  const int np = t.n + 1;
  const int RW = (np + 3) & ~3;           // floats per staged row
  const unsigned RB = (unsigned)RW * 4u;  // bytes per staged row (multiple of 16)
  const int nrows = t.ncross;
  const int G = gridDim.x;
  const unsigned narr = (a.do_B ? (KAHAN ? 5u : 4u) : 2u) + (KAHAN ? 1u : 0u);
  const PlainLayout lay{};
  float* base = reinterpret_cast<float*>(sm);
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_proxy_async();
  }
  fill_rpow(rpow, t.r);
  const XpSmem L = xp_layout(t.n, t.p, t.Rd, t.pw);
  double* WS = reinterpret_cast<double*>(base + L.WS);  // junction-correction weights, loaded once
  const int nw = (t.p + 1) * (2 * t.Rd + 1);
  for (int i = threadIdx.x; i < nw; i += blockDim.x) WS[i] = t.Wd[i];
  // layer segments of the x memory variables (phi_x for B, psi_x for A), two stages
  const bool segs = a.pml && t.pw > 0;
  const MemSeg ms = mem_seg(t.n, segs ? t.pw : 4);
  float* SEG = base + L.SEG;
  auto segp = [&](int st, int which) { return SEG + (size_t)(st * 2 + which) * ms.floats(); };
  float* PA = base + L.PA;  // warm-up partial sums per chunk
  float* PB = PA + ((t.n + 7) / 8 + 8);
  float* TAB = base + L.TAB;
  if (segs) {  // x-layer coefficients at the segment slots, loaded once
    const int F = ms.floats(), n1 = t.n + 1;
    for (int i = threadIdx.x; i < F; i += blockDim.x) {
      const int pos = i < ms.SL ? i : ms.R0 + (i - ms.SL);
      if (pos > t.n) continue;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        TAB[k * F + i] = a.xB.tab[k * n1 + pos];
        TAB[(4 + k) * F + i] = a.xA.tab[k * n1 + pos];
        TAB[(8 + k) * F + i] = a.xA.tabh ? a.xA.tabh[k * n1 + pos] : 0.0f;
      }
    }
  }
  __syncthreads();
  auto issue = [&](int row, int st) {
    float* S = base + (size_t)st * 6 * RW;
    const int64_t rb = (int64_t)row * t.px;
    mbar_expect_tx(&bar[st], narr * RB + (segs ? (a.do_B ? 2u : 1u) * (unsigned)ms.floats() * 4u : 0u));
    bulk_g2s(S, a.v1 + rb, RB, &bar[st]);
    bulk_g2s(S + RW, a.sigma + rb, RB, &bar[st]);
    if (a.do_B) {
      bulk_g2s(S + 2 * RW, a.kappa + rb, RB, &bar[st]);
      bulk_g2s(S + 3 * RW, a.tmp + rb, RB, &bar[st]);
      if (KAHAN) bulk_g2s(S + 4 * RW, a.csig + rb, RB, &bar[st]);
    }
    if (KAHAN) bulk_g2s(S + 5 * RW, a.cv1 + rb, RB, &bar[st]);
    if (segs) {
      if (a.do_B) {
        bulk_g2s(segp(st, 0), a.phix + rb, ms.SL * 4u, &bar[st]);
        bulk_g2s(segp(st, 0) + ms.SL, a.phix + rb + ms.R0, ms.SR * 4u, &bar[st]);
        if (a.zB.in(row)) prefetch_l2(a.phiz + rb, RB);
      }
      bulk_g2s(segp(st, 1), a.psix + rb, ms.SL * 4u, &bar[st]);
      bulk_g2s(segp(st, 1) + ms.SL, a.psix + rb + ms.R0, ms.SR * 4u, &bar[st]);
    }
  };
  if (threadIdx.x == 0 && (int)blockIdx.x < nrows) issue(blockIdx.x, 0);
  unsigned parity[2] = {0u, 0u};
  int i = 0;
  for (int row = blockIdx.x; row < nrows; row += G, ++i) {
    const int st = i & 1;
    const bool more = row + G < nrows;
    if (threadIdx.x == 0 && more) {
      fence_proxy_async();
      issue(row + G, st ^ 1);
    }
    const bool ok = mbar_wait(&bar[st], parity[st], 1u << 24);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicExch(err, 1);
        if (more) mbar_wait(&bar[st ^ 1], parity[st ^ 1], 1u << 24);
      }
      return;
    }
    parity[st] ^= 1u;
    float* S = base + (size_t)st * 6 * RW;
    xrow<KAHAN>(a, t, mmagic, row, lay, S, S + RW, S + 2 * RW, S + 3 * RW, S + 4 * RW, S + 5 * RW, base + L.O,
                rpow, WS, dlf, ms, segp(st, 0), segp(st, 1), PA, PB, TAB);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------------------------
// Host side.
size_t tile_smem_z(const TileGeom& t, int mode) {
  const int rows = t.M + 2 * t.H + 1;
  return (size_t)rows * 32 * 4 + (mode == 1 ? (size_t)2 * (t.M + 1) * 32 * 4 : 0);
}
template <class K>
static cudaError_t tile_launch(K kern, int grid, int threads, size_t smem, cudaStream_t st, void** argv) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaLaunchKernel((const void*)kern, dim3(grid), dim3(threads), argv, smem, st);
}

template <bool KAHAN>
cudaError_t launch_tz(const AcZArgs<float>& a, const TileGeom& t, int mode, int threads, cudaStream_t st) {
  AcZArgs<float> aa = a;
  TileGeom tt = t;
  void* argv[] = {&aa, &tt};
  const int grid = t.ntl * t.p;
  const size_t smem = tile_smem_z(t, mode);
  if (mode == 1) return tile_launch(k_tz<1, KAHAN, 4>, grid, threads, smem, st, argv);
  return tile_launch(k_tz<2, KAHAN, 4>, grid, threads, smem, st, argv);
}

size_t xp_smem(const TileGeom& t) { return (size_t)xp_layout(t.n, t.p, t.Rd, t.pw).total * 4; }

template <bool KAHAN>
cudaError_t launch_xp(const AcXArgs<float>& a, const TileGeom& t, unsigned mmagic, int* err, int num_sms,
                      cudaStream_t st) {
  AcXArgs<float> aa = a;
  TileGeom tt = t;
  unsigned mm = mmagic;
  int* e = err;
  void* argv[] = {&aa, &tt, &mm, &e};
  const int threads = (((t.n + 7) / 8 + 31) / 32) * 32;
  const int grid = t.ncross < 2 * num_sms ? t.ncross : 2 * num_sms;
  return tile_launch(k_xp<KAHAN>, grid, threads, xp_smem(t), st, argv);
}
template cudaError_t launch_xp<false>(const AcXArgs<float>&, const TileGeom&, unsigned, int*, int, cudaStream_t);
template cudaError_t launch_xp<true>(const AcXArgs<float>&, const TileGeom&, unsigned, int*, int, cudaStream_t);

template cudaError_t launch_tz<false>(const AcZArgs<float>&, const TileGeom&, int, int, cudaStream_t);
template cudaError_t launch_tz<true>(const AcZArgs<float>&, const TileGeom&, int, int, cudaStream_t);

}  // namespace lossk
