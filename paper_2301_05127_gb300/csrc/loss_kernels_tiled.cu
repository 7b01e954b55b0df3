// sm_103a FP32 kernels of the 2-D acoustic step in the truncated-convolution form (loss_fir.cuh).
//
// Every output point of the LOSS derivative depends only on:
//   - the field within its own patch;
//   - the K positions beyond each patch end (warm-up of the recursions);
//   - the n_nb positions around the patch's two junctions (PMBC sums, here FP64 junction corrections).
// So no block needs whole lines on chip:
//   - z tiles (k_tz): 32 neighbouring x columns x one patch of z plus a halo of H = max(n_nb, K) positions on
//     each side. There is one 128-byte row segment per z position, and a warp takes one chunk of C z positions
//     for the 32 columns, so shared-memory accesses are conflict-free. A z tile owns the positions
//     [jM, jM + M) of its patch; the last patch also owns the line's last point.
//   - x rows (k_xp): one block per row at a time, persistent over rows, with the next row's arrays bulk-copied
//     (TMA) into a second shared-memory stage while the current row is computed.
// The step is three launches:
//   - the fused x kernel on whole rows: sub-step B with d_x v1 and the staged d_z v3, then the x part of A with
//     d_x sigma;
//   - Z1: the z part of A, from d_z sigma;
//   - Z2: d_z v3 for the next step's B.
// The batched forms (k_xp_batch, k_tz_batch) advance the rows and tiles of many shots in one persistent launch
// each, with the same per-row and per-tile arithmetic.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "../../include/loss.h"
#include "loss_block.cuh"
#include "loss_fir.cuh"
#include "loss_line.cuh"
#include "loss_tile.cuh"
#include "loss_types.h"

namespace lossk {

// ---------------------------------------------------------------------------------------------------------------
// z tiles.  MODE 1 (Z1): v3 += b * (z part of A) from d_z sigma.  MODE 2 (Z2): tmp = d_z v3.
// Shared memory of one tile: the static parts below plus tile_smem_z() dynamic bytes.
struct TzShared {
  float rpow[kFirPow];
  float dl[64];
  double jpart[16 * 32];  // junction partial sums [2 x up to 8 subsets][32 columns]
  double wsm[2 * 129];    // the two junctions' correction weights (Rd <= 64)
};
// Tile `tile` (patch l = tile % p, column group tile / p) of one shot; nwj as tile_junctions_z.  Ends without a
// barrier: a caller that reuses the shared memory must synchronise first.
template <int MODE, bool KAHAN, int LOGC>
__device__ __forceinline__ void tz_tile(const AcZArgs<float>& a, const TileGeom& t, int tile, int nwj,
                                        unsigned char* sm, TzShared& ts) {
  constexpr int C = 1 << LOGC;
  const int l = tile % t.p;                        // patch
  const int cg = tile / t.p;                       // column group
  const int x0 = cg * 32;
  const int z0 = l * t.M;
  const int zb = z0 - t.H;
  const int rows = t.M + 2 * t.H + 1;
  const bool last = l == t.p - 1;
  float* F = reinterpret_cast<float*>(sm);         // [rows][32]
  float* SV = F + rows * 32;                       // MODE 1: v3 of the own rows [M + 1][32]
  float* SC = SV + (t.M + 1) * 32;                 //         compensation of v3
  const float* f = MODE == 1 ? a.sigma : a.v3;
  {
    const int wl = 2 * t.Rd + 1;
    for (int i = threadIdx.x; i < 2 * wl; i += blockDim.x) ts.wsm[i] = t.Wd[(size_t)l * wl + i];
  }
  // two copy groups: first the rows the junction sums read (2H + 1 around each patch end), then the others, so
  // that the FP64 junction sums run while the rest of the tile streams in
  const int jr = 2 * t.H + 1;
  auto copy_row = [&](int q, int seg) {
    const int pos = zb + q;
    if (pos >= 0 && pos <= t.n) cp_async<16>(F + q * 32 + seg * 4, f + (int64_t)pos * t.px + x0 + seg * 4);
  };
  for (int i = threadIdx.x; i < 2 * jr * 8; i += blockDim.x) {
    const int q = i >> 3, seg = i & 7;
    copy_row(q < jr ? q : t.M + (q - jr), seg);
  }
  cp_async_commit();
  for (int i = threadIdx.x; i < rows * 8; i += blockDim.x) {
    const int q = i >> 3, seg = i & 7;
    if (q < jr || (q >= t.M && q < t.M + jr)) continue;
    copy_row(q, seg);
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
  cp_async_wait<1>();
  __syncthreads();
  const ZBun bun{zb};
  const int nvalid = min(32, t.ncross - x0);
  tile_junctions_z(F, bun, nvalid, l, t, nwj, ts.wsm, ts.jpart, ts.dl);
  cp_async_wait<0>();
  __syncthreads();
  const int col = threadIdx.x & 31;
  const int c = threadIdx.x >> 5;
  const int p0 = z0 + c * C;
  int len = min(C, z0 + t.M - p0);     // len <= 0: warps beyond the patch (a batched block sized for a longer one)
  const int lenx = len + ((len > 0 && last && p0 + len == t.n) ? 1 : 0);  // with the line's last point
  // the warm-up sums of K = W C positions come from the W neighbouring chunks when they are whole chunks of this
  // patch, else directly from the tile (its halo reaches K beyond the patch)
  constexpr int W = FirLen<float>::K / C;
  float* PA = SV + (MODE == 1 ? 2 * (t.M + 1) * 32 : 0);  // [chunk][32]: partial sums, after the staged rows
  float* PB = PA + ((t.M + C - 1) / C) * 32;
  float fv[C + 1];
  const bool mine = len > 0 && col < nvalid;
  if (mine) {
#pragma unroll
    for (int j = 0; j <= C; ++j)
      if (j < lenx) fv[j] = F[bun.at(col, p0 + j)];
    if (len == C) chunk_partials<C>(fv, t.r, PA[c * 32 + col], PB[c * 32 + col]);
  }
  __syncthreads();
  if (!mine) return;
  len = lenx;
  const float rC = ts.rpow[C];
  float sL, qR;
  if (c >= W) {
    sL = PA[(c - 1) * 32 + col];
    if (W == 2) sL += rC * PA[(c - 2) * 32 + col];
  } else {
    sL = fir_left<float, FirLen<float>::K>(F, bun, col, p0, t.n, t.r);
  }
  if (len == C && (c + W + 1) * C <= t.M) {
    qR = PB[(c + 1) * 32 + col];
    if (W == 2) qR += rC * PB[(c + 2) * 32 + col];
  } else {
    qR = fir_right<float, FirLen<float>::K>(F, bun, col, p0 + len - 1, t.n, t.r);
  }
  // one body for whole chunks (len == C, a compile-time count) and one for the others
  auto finish = [&](auto lc) {
    const int len = decltype(lc)::value > 0 ? decltype(lc)::value : lenx;
    float e[C + 1];
    tile_chunk_e<C>(fv, p0, len, z0, t, ts.dl + 2 * col, ts.rpow, sL, qR, e);
    const int64_t base = x0 + col;
#pragma unroll
    for (int j = 0; j <= C; ++j) {
      if (j >= len) break;
      const int pos = p0 + j;
      const int64_t gi = (int64_t)pos * t.px + base;
      const float gz = mulc(e[j], t.s3h, t.s3h_lo);
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
        inc = -mulc(gz, a.acoef, a.acoef_lo);
      }
      const float delta = a.b ? bb * inc : mulc(inc, a.b0, a.b0_lo);
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
  };
  if (len == C) finish(std::integral_constant<int, C>{});
  else finish(std::integral_constant<int, 0>{});
}

// One shot: one block per tile, 32 x ceil(M / C) threads.
template <int MODE, bool KAHAN, int LOGC>
__global__ void __launch_bounds__(1024) k_tz(AcZArgs<float> a, TileGeom t) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ TzShared ts;
  fill_rpow(ts.rpow, t.r);
  tz_tile<MODE, KAHAN, LOGC>(a, t, blockIdx.x, blockDim.x >> 5, sm, ts);
}

// All shots in one persistent launch: tiles tile0[s] .. tile0[s + 1] - 1 belong to shot s; the block size is the
// largest of the shots' own (at most 512 threads).
template <int MODE, bool KAHAN, int LOGC>
__global__ void __launch_bounds__(512) k_tz_batch(const TzShot* __restrict__ tab, const int* __restrict__ tile0,
                                                   int nshots, int ntiles) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ TzShared ts;
  __shared__ __align__(16) unsigned char d_raw[sizeof(TzShot)];
  __shared__ int s_shot;
  const TzShot& d = *reinterpret_cast<const TzShot*>(d_raw);
  int cur = -1;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    if (threadIdx.x == 0) s_shot = tile_shot(tile0, nshots, tile);
    __syncthreads();
    const int shot = s_shot;
    if (shot != cur) {
      copy_args(reinterpret_cast<TzShot*>(d_raw), tab + shot);
      __syncthreads();
      fill_rpow(ts.rpow, d.t.r);
      cur = shot;
    }
    tz_tile<MODE, KAHAN, LOGC>(d.a, d.t, tile - tile0[shot], d.nwj, sm, ts);
    __syncthreads();
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
// tid / nt: the thread's index in its group and the group size (whole warps); a group that is not on skips.
template <int G, class BUN>
__device__ void xf_junctions(const float* __restrict__ row, const BUN& bun, const TileGeom& t,
                             const double* __restrict__ wd, float* __restrict__ dlf, int tid, int nt, bool on) {
  const int g = tid % G;
  const int lane = threadIdx.x & 31;
  const unsigned gmask = (((1u << G) - 1u) << (lane & ~(G - 1)));
  const int wl = 2 * t.Rd + 1;
  for (int j = on ? tid / G : t.p + 1; j <= t.p; j += nt / G) {
    const int c = j * t.M;
    const int mlo = max(-t.Rd, -c);
    const int mhi = min(t.Rd, t.n - c);
    const double* wj = wd + (size_t)j * wl + t.Rd;
    double s = 0.0, s2 = 0.0;  // two independent accumulators halve the FP64 dependency chain
    int m = mlo + g;
    for (; m + G <= mhi; m += 2 * G) {
      s = fma(wj[m], widen(row[bun.at(0, c + m)]), s);
      s2 = fma(wj[m + G], widen(row[bun.at(0, c + m + G)]), s2);
    }
    if (m <= mhi) s = fma(wj[m], widen(row[bun.at(0, c + m)]), s);
    s += s2;
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

// One row of the fused x step (sub-step B, then the x part of A) from rows already in shared memory (layout LAY),
// by a group of nt threads (whole warps; tid = index in the group).  Contains block-wide barriers: every thread of
// the block calls it, each group for its own row (or with on = false: barriers only).
template <bool KAHAN, bool SPLITLEN, class LAY, class MIDB>
__device__ __forceinline__ void xrow(const AcXArgs<float>& a, const TileGeom& t, unsigned mmagic, int row,
                                     const LAY& lay, float* V, float* D, const float* SK, const float* ST,
                                     const float* SC, const float* SV, float* O, const float* rpow,
                                     const double* wd, float* dlf, const MemSeg& ms, const float* segB,
                                     const float* segA, float* PA, float* PB, const float* tabs, int tid, int nt,
                                     bool on, const MIDB& midB) {
  const int n = t.n, np = n + 1;
  const int M = t.M;
  const int64_t rb = (int64_t)row * t.px;
  const int nch = (n + 7) >> 3;
  const int c = tid;
  const int len = (c == nch - 1) ? np - (c << 3) : 8;
  const int p0 = c << 3;
  const bool act = on && c < nch;
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
    xf_junctions<8>(V, lay.bun, t, wd, dlf, tid, nt, on);
    __syncthreads();
    if (act) {
      // SPLITLEN: one body per chunk length (8, or 9 for the chunk ending at n), so that the loops carry no
      // predicates; else one body for both (smaller code, for the register-bound batched kernel)
      const int len_rt = len;
      auto chunkB = [&](auto np) {
        const int len = decltype(np)::value > 0 ? decltype(np)::value : len_rt;
        float e[9];
        xf_chunk(V, lay, c, len, t, M, mmagic, dlf, rpow, PA, PB, e);
        const int ob = SB.ordinal(c);
        if (ob >= 0) {
#pragma unroll
          for (int j = 0; j < 9; ++j)
            if (j < len) O[9 * ob + j] = mulc(e[j], t.s3h, t.s3h_lo);
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
            for (int j = 0; j < 9; ++j) iz[j] = -mulc(gz[j], a.dt, a.dt_lo);
          }
#pragma unroll
          for (int j = 0; j < 9; ++j) {
            if (j >= len) break;
            const float delta = kp[j] * (-mulc(mulc(e[j], t.s3h, t.s3h_lo), a.dt, a.dt_lo) + iz[j]);
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
      };
      if (!SPLITLEN) chunkB(std::integral_constant<int, 0>{});
      else if (len == 9) chunkB(std::integral_constant<int, 9>{});
      else chunkB(std::integral_constant<int, 8>{});
    }
    __syncthreads();
    const int nsB = 9 * SB.count();
    for (int q = on ? tid : nsB; q < nsB; q += nt) {
      const int kq = q / 9, j = q - 9 * kq;
      const int ch = SB.chunk(kq);
      if (j >= chunk_len(ch)) continue;
      const int pos = (ch << 3) + j;
      const int64_t gi = rb + pos;
      const int k = lay.bun.at(0, pos);
      const float gx = O[q];
      const float gzv = ST[k];
      float inc = -mulc(gx, a.dt, a.dt_lo);
      if (a.pml && a.xB.in(pos)) {
        const int sl = ms.at(pos);
        inc = pml_step_s(tabs, F, sl, segB[sl], gx, a.phix, gi);
      }
      const float incz = zlay ? a.zB.step(a.phiz, gi, row, gzv) : -mulc(gzv, a.dt, a.dt_lo);
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
    midB();  // the B-only rows of this stage (kappa, d_z v3, sigma's compensation) are free from here on
  }
  const SlowSet SA = slow_set(n, nch, a.pml ? a.xA.width : 0, false, 0);
  if (act) {
    float f8[8];
    lay.eight(D, c, f8);
    xf_partials(f8, t.r, PA[c], PB[c]);
  }
  xf_junctions<8>(D, lay.bun, t, wd, dlf, tid, nt, on);
  __syncthreads();
  if (act) {
    const int len_rt = len;
    auto chunkA = [&](auto np) {
      const int len = decltype(np)::value > 0 ? decltype(np)::value : len_rt;
      float e[9];
      xf_chunk(D, lay, c, len, t, M, mmagic, dlf, rpow, PA, PB, e);
      const int oa = SA.ordinal(c);
      if (oa >= 0) {
#pragma unroll
        for (int j = 0; j < 9; ++j)
          if (j < len) O[9 * oa + j] = mulc(e[j], t.s3h, t.s3h_lo);
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
          const float gj = mulc(mulc(e[j], t.s3h, t.s3h_lo), a.acoef, a.acoef_lo);
          const float delta = a.b ? bb[j] * -gj : -mulc(gj, a.b0, a.b0_lo);
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
    };
    if (!SPLITLEN) chunkA(std::integral_constant<int, 0>{});
    else if (len == 9) chunkA(std::integral_constant<int, 9>{});
    else chunkA(std::integral_constant<int, 8>{});
  }
  __syncthreads();
  const int nsA = 9 * SA.count();
  for (int q = on ? tid : nsA; q < nsA; q += nt) {
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
      inc = -mulc(gx, a.acoef, a.acoef_lo);
    }
    const float delta = a.b ? bb * inc : mulc(inc, a.b0, a.b0_lo);
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

__host__ __device__ inline int xp_mem_floats(int n, int W) {  // MemSeg::floats() of mem_seg(n, W)
  const int R0 = (n + 1 - W) & ~3;
  return ((W + 3) & ~3) + ((n + 1 - R0 + 3) & ~3);
}
// Sizes in floats of the parts, from which xp_place() builds the offsets.
struct XpParts {
  int RW, ocap, ws, F, pa, tab;
};
__host__ __device__ inline XpParts xp_parts(int n, int p, int Rd, int pw) {
  XpParts q;
  q.RW = (n + 1 + 3) & ~3;
  q.ocap = ((2 * ((pw + 7) / 8 + 2) + 5) * 9 + 3) & ~3;
  q.ws = 2 * ((((p + 1) * (2 * Rd + 1)) + 1) & ~1);
  q.F = xp_mem_floats(n, pw > 0 ? pw : 4);
  q.pa = (n + 7) / 8 + 8;
  q.tab = pw > 0 ? 12 * q.F : 0;
  return q;
}
// na: rows staged per stage (6 with compensation arrays, else 4).
__host__ __device__ inline XpSmem xp_place(const XpParts& q, int na) {
  XpSmem L;
  L.NA = na;
  L.DL = 0;
  L.RW = q.RW;
  L.O = 2 * na * q.RW;
  L.WS = L.O + q.ocap;
  L.SEG = L.WS + q.ws;
  L.F = q.F;
  L.PA = L.SEG + 4 * q.F;
  L.PB = L.PA + q.pa;
  L.TAB = L.PA + ((2 * q.pa + 3) & ~3);
  L.total = L.TAB + q.tab;
  return L;
}
__host__ __device__ inline XpSmem xp_layout(int n, int p, int Rd, int pw, bool kahan) {
  return xp_place(xp_parts(n, p, Rd, pw), kahan ? 6 : 4);
}

// Junction-correction weights (unless WS is null) and x-layer coefficients of one shot into shared memory (no
// barrier).
__device__ __forceinline__ void xp_stage_shot(const AcXArgs<float>& a, const TileGeom& t, const MemSeg& ms, bool segs,
                                              double* WS, float* TAB) {
  const int nw = (t.p + 1) * (2 * t.Rd + 1);
  if (WS)
    for (int i = threadIdx.x; i < nw; i += blockDim.x) WS[i] = t.Wd[i];
  if (segs) {
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
}

// Bytes that xp_issue copies for one row.
template <bool KAHAN>
__device__ __forceinline__ unsigned xp_row_bytes(const AcXArgs<float>& a, const TileGeom& t, const MemSeg& ms,
                                                 bool segs) {
  const unsigned RB = (unsigned)((t.n + 1 + 3) & ~3) * 4u;
  const unsigned narr = (a.do_B ? (KAHAN ? 5u : 4u) : 2u) + (KAHAN ? 1u : 0u);
  return narr * RB + (segs ? (a.do_B ? 2u : 1u) * (unsigned)ms.floats() * 4u : 0u);
}
// Bulk copies (one thread) of row `row` of one shot into a stage: six rows at S + k * stride and the two layer
// segments, completing on *bar (whose expected bytes the caller has raised by xp_row_bytes).  part 1: the rows only
// sub-step B reads (kappa, d_z v3, sigma's compensation, the phi_x segments); part 2: the others; 0: all.
template <bool KAHAN>
__device__ __forceinline__ void xp_issue(const AcXArgs<float>& a, const TileGeom& t, const MemSeg& ms, bool segs,
                                         int row, float* S, int stride, float* seg0, float* seg1, uint64_t* bar,
                                         int part = 0) {
  const int RW = (t.n + 1 + 3) & ~3;
  const unsigned RB = (unsigned)RW * 4u;
  const int64_t rb = (int64_t)row * t.px;
  if (part != 1) {
    bulk_g2s(S, a.v1 + rb, RB, bar);
    bulk_g2s(S + stride, a.sigma + rb, RB, bar);
    if (KAHAN) bulk_g2s(S + 5 * stride, a.cv1 + rb, RB, bar);
    if (segs) {
      bulk_g2s(seg1, a.psix + rb, ms.SL * 4u, bar);
      bulk_g2s(seg1 + ms.SL, a.psix + rb + ms.R0, ms.SR * 4u, bar);
    }
  }
  if (part != 2 && a.do_B) {
    bulk_g2s(S + 2 * stride, a.kappa + rb, RB, bar);
    bulk_g2s(S + 3 * stride, a.tmp + rb, RB, bar);
    if (KAHAN) bulk_g2s(S + 4 * stride, a.csig + rb, RB, bar);
    if (segs) {
      bulk_g2s(seg0, a.phix + rb, ms.SL * 4u, bar);
      bulk_g2s(seg0 + ms.SL, a.phix + rb + ms.R0, ms.SR * 4u, bar);
      if (a.zB.in(row)) prefetch_l2(a.phiz + rb, RB);
    }
  }
}

__device__ __forceinline__ void xp_init_barriers(uint64_t* bar) {
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_proxy_async();
  }
}

// Persistent, software-pipelined form: each block takes rows blockIdx.x, blockIdx.x + gridDim.x, ...; one thread
// bulk-copies (TMA) the next row's arrays into the other of two shared-memory stages while the block computes the
// current row, so HBM streams while the block computes.  Waits on the stage barriers are bounded: on a timeout
// the block records it in *err, waits (bounded) for its copy in flight and stops.
// WIDE: rows of 2050 to 4097 points, one chunk per thread in blocks of up to 512 threads, one block per SM.
template <bool KAHAN, bool WIDE>
__global__ void __launch_bounds__(WIDE ? 512 : 256, WIDE ? 1 : 2) k_xp(AcXArgs<float> a, TileGeom t, unsigned mmagic,
                                                                       int* err, unsigned polls) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ float rpow[kFirPow];
  __shared__ float dlf[65];
  __shared__ __align__(8) uint64_t bar[2];
  const int nrows = t.ncross;
  const int G = gridDim.x;
  const PlainLayout lay{};
  float* base = reinterpret_cast<float*>(sm);
  xp_init_barriers(bar);
  fill_rpow(rpow, t.r);
  const XpSmem L = xp_layout(t.n, t.p, t.Rd, t.pw, KAHAN);
  double* WS = reinterpret_cast<double*>(base + L.WS);
  const bool segs = a.pml && t.pw > 0;
  const MemSeg ms = mem_seg(t.n, segs ? t.pw : 4);
  float* SEG = base + L.SEG;
  auto segp = [&](int st, int which) { return SEG + (size_t)(st * 2 + which) * L.F; };
  float* PA = base + L.PA;  // warm-up partial sums per chunk
  float* PB = base + L.PB;
  float* TAB = base + L.TAB;
  xp_stage_shot(a, t, ms, segs, WS, TAB);  // loaded once
  __syncthreads();
  // Copies of a row into a stage: part 1 arms the stage's barrier with the row's bytes (part 0: all at once).
  auto issue = [&](int row, int st, int part) {
    if (part != 2) mbar_expect_tx(&bar[st], xp_row_bytes<KAHAN>(a, t, ms, segs));
    xp_issue<KAHAN>(a, t, ms, segs, row, base + (size_t)st * L.NA * L.RW, L.RW, segp(st, 0), segp(st, 1), &bar[st],
                    part);
  };
  // With sub-step B the rows only B reads are copied earlier: those of row + 2G go into the current stage as soon
  // as B is done with it, the rest of a row at the start of the row before it.
  const bool split = a.do_B != 0;
  if (threadIdx.x == 0 && (int)blockIdx.x < nrows) {
    issue(blockIdx.x, 0, 0);
    if (split && (int)blockIdx.x + G < nrows) issue(blockIdx.x + G, 1, 1);
  }
  unsigned parity[2] = {0u, 0u};
  int i = 0;
  for (int row = blockIdx.x; row < nrows; row += G, ++i) {
    const int st = i & 1;
    const bool more = row + G < nrows;
    if (threadIdx.x == 0 && more) {
      fence_proxy_async();
      issue(row + G, st ^ 1, split ? 2 : 0);
    }
    const bool ok = mbar_wait(&bar[st], parity[st], polls);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {  // let the copies in flight land (bounded) before the block leaves
        atomicExch(err, 1);
        mbar_wait(&bar[st], parity[st], kDrainPolls);
        if (more) mbar_wait(&bar[st ^ 1], parity[st ^ 1], kDrainPolls);
      }
      return;
    }
    parity[st] ^= 1u;
    float* S = base + (size_t)st * L.NA * L.RW;
    const bool more2 = split && row + 2 * G < nrows;
    auto midB = [&] {
      if (threadIdx.x == 0 && more2) {
        fence_proxy_async();
        issue(row + 2 * G, st, 1);
      }
    };
    xrow<KAHAN, true>(a, t, mmagic, row, lay, S, S + L.RW, S + 2 * L.RW, S + 3 * L.RW, S + 4 * L.RW, S + 5 * L.RW,
                base + L.O, rpow, WS, dlf, ms, segp(st, 0), segp(st, 1), PA, PB, TAB, threadIdx.x, blockDim.x, true,
                midB);
    __syncthreads();
  }
}

// All shots in one persistent launch.  Work comes in units of R consecutive rows of one shot (R = XpShot::R, the
// rows that R groups of blockDim / R threads compute side by side, so that short rows fill the block); the units
// of shot s are unit0[s] .. unit0[s + 1] - 1, and block b takes the units bunit[b] .. bunit[b + 1] - 1 (about the
// same number of points per block), the first of them in shot bshot[b].  The pipeline is that of k_xp; a stage
// records the shot of its unit, the descriptors of the (at most two) live shots sit in two slots (shot s in slot
// s & 1), and a block restages the weights and layer tables when its units move on to the next shot.  Shared
// memory of a stage: array k of group g at S + k * RR + g * RW (RR = R * RW); per group its own O, warm-up sums,
// layer segments and junction corrections.
template <bool KAHAN>
__global__ void __launch_bounds__(256, 2) k_xp_batch(const XpShot* __restrict__ shots, const int* __restrict__ unit0,
                                                     const int* __restrict__ bunit, const int* __restrict__ bshot,
                                                     XpSmem L, int* err, unsigned polls) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ float rpow[kFirPow];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ __align__(16) unsigned char slot[2][sizeof(XpShot)];
  __shared__ int stage_shot[2];
  const int u0 = bunit[blockIdx.x], u1 = bunit[blockIdx.x + 1];
  if (u0 >= u1) return;
  const PlainLayout lay{};
  float* base = reinterpret_cast<float*>(sm);
  xp_init_barriers(bar);
  float* TAB = base + L.TAB;
  float* dlf = base + L.DL;  // junction corrections, 65 per group
  auto desc = [&](int s) -> const XpShot& { return *reinterpret_cast<const XpShot*>(slot[s & 1]); };
  // per-shot geometry of the stage and group regions
  struct Geo {
    int R, RW, RR, F, ocap, pa;
  };
  auto geo = [&](const XpShot& d) {
    Geo q;
    q.R = d.R;
    q.RW = (d.t.n + 1 + 3) & ~3;
    q.RR = q.R * q.RW;
    q.F = xp_mem_floats(d.t.n, (d.a.pml && d.t.pw > 0) ? d.t.pw : 4);
    q.ocap = ((2 * ((d.t.pw + 7) / 8 + 2) + 5) * 9 + 3) & ~3;
    q.pa = (d.t.n + 7) / 8 + 8;
    return q;
  };
  auto segp = [&](int st, int which, const Geo& q, int g) {
    return base + L.SEG + (size_t)(st * 2 + which) * L.F + (size_t)g * q.F;
  };
  // thread 0's view of the shot of the units it issues
  int is = bshot[blockIdx.x];
  int iend = 0;
  auto load_desc = [&](int s) {
    const uint64_t* src = reinterpret_cast<const uint64_t*>(shots + s);
    uint64_t* dst = reinterpret_cast<uint64_t*>(slot[s & 1]);
    for (int w = 0; w < (int)(sizeof(XpShot) / 8); ++w) dst[w] = src[w];
  };
  if (threadIdx.x == 0) {
    load_desc(is);
    iend = unit0[is + 1];
  }
  fill_rpow(rpow, shots[is].t.r);
  auto issue = [&](int u, int st) {  // thread 0
    while (u >= iend) {
      ++is;
      load_desc(is);
      iend = unit0[is + 1];
    }
    stage_shot[st] = is;
    const XpShot& d = desc(is);
    const Geo q = geo(d);
    const bool segs = d.a.pml && d.t.pw > 0;
    const MemSeg ms = mem_seg(d.t.n, segs ? d.t.pw : 4);
    const int r0 = (u - d.unit0) * q.R;
    const int nr = min(q.R, d.t.ncross - r0);
    mbar_expect_tx(&bar[st], (unsigned)nr * xp_row_bytes<KAHAN>(d.a, d.t, ms, segs));
    for (int g = 0; g < nr; ++g)
      xp_issue<KAHAN>(d.a, d.t, ms, segs, r0 + g, base + (size_t)st * L.NA * L.RW + (size_t)g * q.RW, q.RR,
                      segp(st, 0, q, g), segp(st, 1, q, g), &bar[st]);
  };
  if (threadIdx.x == 0) issue(u0, 0);
  unsigned parity[2] = {0u, 0u};
  int loaded = -1;
  int i = 0;
  for (int u = u0; u < u1; ++u, ++i) {
    const int st = i & 1;
    const bool more = u + 1 < u1;
    if (threadIdx.x == 0 && more) {
      fence_proxy_async();
      issue(u + 1, st ^ 1);
    }
    const bool ok = mbar_wait(&bar[st], parity[st], polls);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {  // let the copies in flight land (bounded) before the block leaves
        atomicExch(err, 1);
        mbar_wait(&bar[st], parity[st], kDrainPolls);
        if (more) mbar_wait(&bar[st ^ 1], parity[st ^ 1], kDrainPolls);
      }
      return;
    }
    parity[st] ^= 1u;
    const int s = stage_shot[st];
    const XpShot& d = desc(s);
    const Geo q = geo(d);
    const bool segs = d.a.pml && d.t.pw > 0;
    const MemSeg ms = mem_seg(d.t.n, segs ? d.t.pw : 4);
    if (s != loaded) {  // the junction weights are read from global memory (L1) here, not staged
      xp_stage_shot(d.a, d.t, ms, segs, nullptr, TAB);
      loaded = s;
      __syncthreads();
    }
    const int nt = blockDim.x / q.R;
    const int g = threadIdx.x / nt;
    const int row = (u - d.unit0) * q.R + g;
    float* S = base + (size_t)st * L.NA * L.RW + (size_t)g * q.RW;
    float* PAg = base + L.PA + (size_t)g * 2 * q.pa;
    xrow<KAHAN, false>(d.a, d.t, d.mmagic, row, lay, S, S + q.RR, S + 2 * q.RR, S + 3 * q.RR, S + 4 * q.RR, S + 5 * q.RR,
                base + L.O + (size_t)g * q.ocap, rpow, d.t.Wd, dlf + g * 65, ms, segp(st, 0, q, g), segp(st, 1, q, g),
                PAg, PAg + q.pa, TAB, threadIdx.x - g * nt, nt, row < d.t.ncross, [] {});
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------------------------
// Host side.
// Dynamic shared memory of a z tile: the rows, (Z1) the own rows of v3 and its compensation, and two partial sums
// per chunk (2^logc positions) and column.
size_t tile_smem_z(const TileGeom& t, int mode, int logc) {
  const int rows = t.M + 2 * t.H + 1;
  const int C = 1 << logc;
  return (size_t)rows * 32 * 4 + (mode == 1 ? (size_t)2 * (t.M + 1) * 32 * 4 : 0) +
         (size_t)2 * ((t.M + C - 1) / C) * 32 * 4;
}
template <class K>
static cudaError_t tile_launch(K kern, int grid, int threads, size_t smem, cudaStream_t st, void** argv) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaLaunchKernel((const void*)kern, dim3(grid), dim3(threads), argv, smem, st);
}

// logc: log2 of the z positions one warp row takes (3 or 4).
template <bool KAHAN>
cudaError_t launch_tz(const AcZArgs<float>& a, const TileGeom& t, int mode, int threads, int logc, cudaStream_t st) {
  AcZArgs<float> aa = a;
  TileGeom tt = t;
  void* argv[] = {&aa, &tt};
  const int grid = t.ntl * t.p;
  const size_t smem = tile_smem_z(t, mode, logc);
  if (logc == 3) {
    if (mode == 1) return tile_launch(k_tz<1, KAHAN, 3>, grid, threads, smem, st, argv);
    return tile_launch(k_tz<2, KAHAN, 3>, grid, threads, smem, st, argv);
  }
  if (mode == 1) return tile_launch(k_tz<1, KAHAN, 4>, grid, threads, smem, st, argv);
  return tile_launch(k_tz<2, KAHAN, 4>, grid, threads, smem, st, argv);
}

size_t xp_smem(const TileGeom& t, bool kahan) { return (size_t)xp_layout(t.n, t.p, t.Rd, t.pw, kahan).total * 4; }

// Rows per work unit of a batched x launch of `threads` threads: as many groups of whole warps as the row's
// chunks leave room for, at most kXpMaxGroups.
int xp_rows_per_unit(int n, int threads) {
  const int need = 32 * (((n + 7) / 8 + 31) / 32);
  int R = 1;
  while (R < kXpMaxGroups && 2 * R * need <= threads && (threads / (2 * R)) % 32 == 0) R *= 2;
  return R;
}

// Layout of a batched x launch: every part as large as the largest shot's, the per-group parts times the shot's
// rows per unit R (rs[i]); no staged weights, and the junction corrections of the groups after the tables.
XpSmem xp_batch_layout(const std::vector<TileGeom>& ts, const std::vector<int>& rs, bool kahan) {
  int RW = 0, ocap = 0, F = 0, pa = 0, tab = 0, R = 1;
  for (size_t i = 0; i < ts.size(); ++i) {
    const TileGeom& t = ts[i];
    const XpParts q = xp_parts(t.n, t.p, t.Rd, t.pw);
    RW = std::max(RW, rs[i] * q.RW);
    ocap = std::max(ocap, rs[i] * q.ocap);
    F = std::max(F, rs[i] * q.F);
    pa = std::max(pa, rs[i] * 2 * q.pa);
    tab = std::max(tab, 12 * q.F);
    R = std::max(R, rs[i]);
  }
  XpSmem L;
  L.NA = kahan ? 6 : 4;
  L.RW = (RW + 3) & ~3;
  L.O = 2 * L.NA * L.RW;
  L.WS = L.O + ((ocap + 3) & ~3);
  L.SEG = L.WS;
  L.F = (F + 3) & ~3;
  L.PA = L.SEG + 4 * L.F;
  L.PB = L.PA;  // per group: PA at 2 g pa, PB at 2 g pa + pa
  L.TAB = L.PA + ((pa + 3) & ~3);
  L.DL = L.TAB + ((tab + 3) & ~3);
  L.total = L.DL + ((R * 65 + 3) & ~3);
  return L;
}

template <bool KAHAN>
cudaError_t launch_xp_batch(const XpShot* shots, const int* unit0, const int* bunit, const int* bshot,
                            const XpSmem& L, int threads, int grid, int* err, unsigned polls, cudaStream_t st) {
  if (grid <= 0) return cudaSuccess;
  XpSmem l = L;
  void* argv[] = {(void*)&shots, (void*)&unit0, (void*)&bunit, (void*)&bshot, (void*)&l, (void*)&err, (void*)&polls};
  return tile_launch(k_xp_batch<KAHAN>, grid, threads, (size_t)L.total * 4, st, argv);
}
template <bool KAHAN>
cudaError_t xp_batch_per_sm(const XpSmem& L, int threads, int* per_sm) {
  cudaError_t e = cudaFuncSetAttribute(k_xp_batch<KAHAN>, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total * 4);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_xp_batch<KAHAN>, threads, (size_t)L.total * 4);
}
template <int MODE, bool KAHAN>
static auto tz_batch_kernel(int logc) {
  return logc == 3 ? k_tz_batch<MODE, KAHAN, 3> : k_tz_batch<MODE, KAHAN, 4>;
}
template <bool KAHAN>
cudaError_t launch_tz_batch(const TzShot* tab, const int* tile0, int nshots, int ntiles, int mode, int threads,
                            int logc, size_t smem, int grid, cudaStream_t st) {
  if (grid <= 0 || ntiles <= 0) return cudaSuccess;
  void* argv[] = {(void*)&tab, (void*)&tile0, (void*)&nshots, (void*)&ntiles};
  if (mode == 1) return tile_launch(tz_batch_kernel<1, KAHAN>(logc), grid, threads, smem, st, argv);
  return tile_launch(tz_batch_kernel<2, KAHAN>(logc), grid, threads, smem, st, argv);
}
template <bool KAHAN>
cudaError_t tz_batch_per_sm(int mode, int threads, int logc, size_t smem, int* per_sm) {
  auto kern = mode == 1 ? tz_batch_kernel<1, KAHAN>(logc) : tz_batch_kernel<2, KAHAN>(logc);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, threads, smem);
}
template cudaError_t launch_xp_batch<false>(const XpShot*, const int*, const int*, const int*, const XpSmem&, int, int,
                                            int*, unsigned, cudaStream_t);
template cudaError_t launch_xp_batch<true>(const XpShot*, const int*, const int*, const int*, const XpSmem&, int, int,
                                           int*, unsigned, cudaStream_t);
template cudaError_t xp_batch_per_sm<false>(const XpSmem&, int, int*);
template cudaError_t xp_batch_per_sm<true>(const XpSmem&, int, int*);
template cudaError_t launch_tz_batch<false>(const TzShot*, const int*, int, int, int, int, int, size_t, int,
                                            cudaStream_t);
template cudaError_t launch_tz_batch<true>(const TzShot*, const int*, int, int, int, int, int, size_t, int,
                                           cudaStream_t);
template cudaError_t tz_batch_per_sm<false>(int, int, int, size_t, int*);
template cudaError_t tz_batch_per_sm<true>(int, int, int, size_t, int*);

template <bool KAHAN>
cudaError_t launch_xp(const AcXArgs<float>& a, const TileGeom& t, unsigned mmagic, int* err, unsigned polls,
                      int num_sms, cudaStream_t st) {
  AcXArgs<float> aa = a;
  TileGeom tt = t;
  unsigned mm = mmagic;
  int* e = err;
  unsigned pl = polls;
  void* argv[] = {&aa, &tt, &mm, &e, &pl};
  const int threads = (((t.n + 7) / 8 + 31) / 32) * 32;
  if (threads > 256) {
    const int grid = t.ncross < num_sms ? t.ncross : num_sms;
    return tile_launch(k_xp<KAHAN, true>, grid, threads, xp_smem(t, KAHAN), st, argv);
  }
  const int grid = t.ncross < 2 * num_sms ? t.ncross : 2 * num_sms;
  return tile_launch(k_xp<KAHAN, false>, grid, threads, xp_smem(t, KAHAN), st, argv);
}
template cudaError_t launch_xp<false>(const AcXArgs<float>&, const TileGeom&, unsigned, int*, unsigned, int,
                                      cudaStream_t);
template cudaError_t launch_xp<true>(const AcXArgs<float>&, const TileGeom&, unsigned, int*, unsigned, int,
                                     cudaStream_t);

template cudaError_t launch_tz<false>(const AcZArgs<float>&, const TileGeom&, int, int, int, cudaStream_t);
template cudaError_t launch_tz<true>(const AcZArgs<float>&, const TileGeom&, int, int, int, cudaStream_t);

}  // namespace lossk
