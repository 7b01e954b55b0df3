// sm_103a kernels of the 2-D acoustic LOSS step and of the stand-alone derivative.
//
// Time stepping (paper Sec. 3.3, Strang "half A, full B, half A", with the exponential ADE-PML sub-flows in
// the absorbing layers).  Consecutive half steps of A share the same stress, so n steps are one half A,
// n - 1 alternations (full B, full A), a full B and a half A.  The library keeps the velocities half a step
// ahead between calls (staggered state), so one step is:
//   X kernel (lines along x):  sigma += -dt kappa (d_x v1 + d_z v3) + source           [sub-step B]
//                              v1    += -dt b d_x sigma                                   [A, x part]
//   Z kernel (lines along z):  v3    += -dt b d_z sigma                                   [A, z part]
//                              tmp    = d_z v3                       (feeds the next step's B)
// Inside a PML layer the increments -tau g are replaced by the exact exponential flow of the memory variables
// (PmlAxis::step): Phi_x, Phi_z advance in the B part of the X kernel, Psi_x in its A part, Psi_z in the Z
// kernel, each exactly once per sub-step.
//
// Each block holds whole grid lines (all patches) on chip, so the PMBC halo of every junction is read from
// shared memory and each field is read from and written to HBM once per kernel.  All global -> shared traffic
// is issued up front with cp.async in two groups: the lines the first solve needs, then the operands of the
// pointwise updates, which arrive while the block solves.
#include <cuda_runtime.h>

#include "loss_block.cuh"
#include "loss_line.cuh"
#include "loss_types.h"

namespace lossk {


// ---------------------------------------------------------------------------------------------------------------
// Stand-alone derivative d1 (and d2) along one axis; optional phi output.
template <typename T, int LOGC, bool SFLAV>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 512 : 1024) k_deriv(DerivArgs<T> a) {
  constexpr int C = 1 << LOGC;
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ ChunkClasses<T, C> cc;
  const LineGeom& g = a.g;
  const bool want_d2 = a.d2 != nullptr;
  Carve<T> cv(sm, g, want_d2 ? 3 : 2, 0);
  T* F = cv.buf[0];
  T* O = cv.buf[1];
  T* O2 = cv.buf[2];
  const Bundle<LOGC, SFLAV> bun{g.pitch};
  const WorkMap<SFLAV> wm{g.L, g.p, g.NC};
  const int logL = log2_pow2(g.L);
  const int nvalid = bundle_bases<SFLAV>(g, blockIdx.x, cv.lb);
  chunk_classes_init<T, C>(&cc, g.M, g.NC, a.tb.t32, a.tb.t64, a.minf);
  __syncthreads();
  stage_padded<T, SFLAV>(a.f, F, bun, g, cv.lb, nvalid, logL);
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  pmbc_phi<T, 16>(F, bun, g.L, nvalid, g.n, g.p, g.M, g.n_nb, a.tb.W, cv.phi);
  __syncthreads();
  const int p1 = g.p + 1;
  if (a.phi_out) {
    for (int i = threadIdx.x; i < nvalid * p1; i += blockDim.x) {
      const int l = i / p1;
      int64_t line;
      if (SFLAV) {
        const int outer = blockIdx.x / g.nxb;
        line = (int64_t)outer * a.lines_per_outer + (blockIdx.x - outer * g.nxb) * g.L + l;
      } else {
        line = (int64_t)blockIdx.x * g.L + l;
      }
      a.phi_out[line * p1 + (i - l * p1)] = cv.phi[i] * a.s1d;
    }
  }
  if (a.d1 == nullptr) return;
  solve_bundle<T, C, SFLAV>(F, O, cv.sA, &cc, bun, wm, nvalid, g.M, a.tb.t32, a.tb.t64, a.minf, RhsD1{},
                            BndPhi<T>{cv.phi, p1});
  for_points<SFLAV>(g, cv.lb, nvalid, logL, [&](int l, int pos, int64_t gi) {
    a.d1[gi] = a.s1 * O[bun.at(l, pos)];
  });
  if (!want_d2) return;
  solve_bundle<T, C, SFLAV>(F, O2, cv.sA, &cc, bun, wm, nvalid, g.M, a.tb.t32, a.tb.t64, a.minf, RhsD2{},
                            BndD2<T, Bundle<LOGC, SFLAV>>{F, O, cv.phi, p1, g.M, bun});
  // Output: interior slots from the solve; at a junction the average of the two patches' end values
  // (d2 h^2/6)_avg = (f_{j-1} - 2 f_j + f_{j+1} + e_{j-1} - e_{j+1}) / 2; at the two line ends the single value.
  for_points<SFLAV>(g, cv.lb, nvalid, logL, [&](int l, int pos, int64_t gi) {
    const int j = div_magic(pos, g.mmagic);
    T s;
    if (pos != j * g.M) {
      s = O2[bun.at(l, pos)];
    } else {
      const T ej = (T)cv.phi[l * p1 + j];
      if (pos == 0) {
        s = (F[bun.at(l, 1)] - F[bun.at(l, 0)]) - T(2) * ej - O[bun.at(l, 1)];
      } else if (pos == g.n) {
        s = (F[bun.at(l, pos - 1)] - F[bun.at(l, pos)]) + T(2) * ej + O[bun.at(l, pos - 1)];
      } else {
        const T fm = F[bun.at(l, pos - 1)], f0 = F[bun.at(l, pos)], fp = F[bun.at(l, pos + 1)];
        s = T(0.5) * (((fm - f0) + (fp - f0)) + (O[bun.at(l, pos - 1)] - O[bun.at(l, pos + 1)]));
      }
    }
    a.d2[gi] = a.s2 * s;
  });
}

// ---------------------------------------------------------------------------------------------------------------
// Source amplitude of this step: the immediate value, or the entry of the per-step table at the device clock.
__device__ __forceinline__ double source_amp(const SourceArgs& s) {
  return s.amp_tab ? s.amp_tab[s.clk->step] : s.amp;
}

// X kernel of the 2-D acoustic step: sub-step B on whole x lines, then the x part of sub-step A.  One tile is
// one bundle `bid` of rows; cc must hold the chunk classes of this geometry.
template <typename T, int LOGC, bool KAHAN>
__device__ __forceinline__ void ac_x_tile(const AcXArgs<T>& a, int bid, unsigned char* sm,
                                          const ChunkClasses<T, 1 << LOGC>& cc) {
  constexpr int C = 1 << LOGC;
  const LineGeom& g = a.g;
  Carve<T> cv(sm, g, 3, 4);
  T* V = cv.buf[0];  // v1 (old)
  T* D = cv.buf[1];  // sigma, then sigma after B
  T* O = cv.buf[2];  // solve output
  T* SK = cv.stg[0];  // kappa
  T* ST = cv.stg[1];  // d_z v3
  T* SC = cv.stg[2];  // compensation of sigma
  T* SV = cv.stg[3];  // compensation of v1
  const Bundle<LOGC, false> bun{g.pitch};
  const WorkMap<false> wm{g.L, g.p, g.NC};
  const int nvalid = bundle_bases<false>(g, bid, cv.lb);
  const int p1 = g.p + 1;
  const int sp = g.spitch;
  const double amp = source_amp(a.src);
  const bool son = a.src.on && amp != 0.0;
  __syncthreads();
  stage_padded<T, false>(a.v1, V, bun, g, cv.lb, nvalid, 0);
  stage_padded<T, false>(a.sigma, D, bun, g, cv.lb, nvalid, 0);
  cp_async_commit();
  if (a.do_B) {
    stage_rows<T>(a.kappa, SK, g, cv.lb, nvalid);
    stage_rows<T>(a.tmp, ST, g, cv.lb, nvalid);
    if constexpr (KAHAN) stage_rows<T>(a.csig, SC, g, cv.lb, nvalid);
  }
  if constexpr (KAHAN) stage_rows<T>(a.cv1, SV, g, cv.lb, nvalid);
  cp_async_commit();
  if (a.do_B) {
    cp_async_wait<1>();
    __syncthreads();
    pmbc_phi<T, 16>(V, bun, g.L, nvalid, g.n, g.p, g.M, g.n_nb, a.tb.W, cv.phi);
    __syncthreads();
    solve_bundle<T, C, false>(V, O, cv.sA, &cc, bun, wm, nvalid, g.M, a.tb.t32, a.tb.t64, a.minf, RhsD1{},
                              BndPhi<T>{cv.phi, p1});
    cp_async_wait<0>();
    __syncthreads();
    const int64_t r0 = (int64_t)bid * g.L;
    const int np = g.n + 1;
    for (int l = 0; l < nvalid; ++l) {
      const int z = (int)((r0 + l) / g.ny1);
      const bool zlay = a.pml && a.zB.in(z);
      const bool srow = son && (unsigned)(z - a.src.zs + 12) < 25u;
      const int64_t rb = cv.lb[l];
      const T* stl = ST + l * sp;
      const T* skl = SK + l * sp;
      const T* scl = SC + l * sp;
      // scalar update of one point (PML layers, source block, line tail)
      auto one = [&](int pos) {
        const int64_t gi = rb + pos;
        const T gx = mulc(O[bun.at(l, pos)], a.s3h, a.s3h_lo);  // d_x v1
        const T gz = stl[pos];                   // d_z v3
        T inc = (a.pml && a.xB.in(pos)) ? a.xB.step(a.phix, gi, pos, gx) : -mulc(gx, a.dt, a.dt_lo);
        inc += zlay ? a.zB.step(a.phiz, gi, z, gz) : -mulc(gz, a.dt, a.dt_lo);
        T delta = skl[pos] * inc;
        if (srow) {
          const int dx = pos - a.src.xs + 12;
          if ((unsigned)dx < 25u) delta += (T)(amp * a.src.g[z - a.src.zs + 12] * a.src.g[dx]);
        }
        const int k = bun.at(l, pos);
        T sg = D[k];
        if constexpr (KAHAN) {
          float c = scl[pos];
          kahan_add(sg, c, delta);
          a.csig[gi] = c;
        } else {
          sg += delta;
        }
        a.sigma[gi] = sg;
        D[k] = sg;
      };
      // four points per thread, lanes on consecutive positions (conflict-free on the padded buffers)
      const int T4 = 4 * blockDim.x;
      for (int q0 = threadIdx.x; q0 < np; q0 += T4) {
        T gz[4], kp[4], cc[4], ox[4], sg[4];
        bool fastp[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int pos = q0 + t * blockDim.x;
          fastp[t] = pos < np && !zlay && !(a.pml && a.xB.in(pos)) && !(srow && (unsigned)(pos - a.src.xs + 12) < 25u);
          if (fastp[t]) {
            const int k = bun.at(l, pos);
            gz[t] = stl[pos];
            kp[t] = skl[pos];
            if constexpr (KAHAN) cc[t] = scl[pos];
            ox[t] = O[k];
            sg[t] = D[k];
          }
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int pos = q0 + t * blockDim.x;
          if (!fastp[t]) {
            if (pos < np) one(pos);
            continue;
          }
          const T delta = kp[t] * -mulc(mulc(ox[t], a.s3h, a.s3h_lo) + gz[t], a.dt, a.dt_lo);
          if constexpr (KAHAN) {
            kahan_add(sg[t], cc[t], delta);
            a.csig[rb + pos] = cc[t];
          } else {
            sg[t] += delta;
          }
          a.sigma[rb + pos] = sg[t];
          D[bun.at(l, pos)] = sg[t];
        }
      }
    }
    __syncthreads();
  } else {
    cp_async_wait<0>();
    __syncthreads();
  }
  pmbc_phi<T, 16>(D, bun, g.L, nvalid, g.n, g.p, g.M, g.n_nb, a.tb.W, cv.phi);
  __syncthreads();
  solve_bundle<T, C, false>(D, O, cv.sA, &cc, bun, wm, nvalid, g.M, a.tb.t32, a.tb.t64, a.minf, RhsD1{},
                            BndPhi<T>{cv.phi, p1});
  {
    const int np = g.n + 1;
    for (int l = 0; l < nvalid; ++l) {
      const int64_t rb = cv.lb[l];
      const T* svl = SV + l * sp;
      auto one = [&](int pos) {
        const int64_t gi = rb + pos;
        const T gx = mulc(O[bun.at(l, pos)], a.s3h, a.s3h_lo);  // d_x sigma
        const T bb = a.b ? a.b[gi] : a.b0;
        T inc;
        if (a.pml && a.xA.in(pos)) {
          const T ih = a.dlt ? a.xA.half(a.psix, gi, pos, gx) : T(0);
          inc = a.xA.step(a.psix, gi, pos, gx);
          if (a.dlt) a.dlt[gi] = bb * (ih - T(0.5) * inc);
        } else {
          inc = -mulc(gx, a.acoef, a.acoef_lo);
        }
        const T delta = a.b ? bb * inc : mulc(inc, a.b0, a.b0_lo);
        T v = V[bun.at(l, pos)];
        if constexpr (KAHAN) {
          float c = svl[pos];
          kahan_add(v, c, delta);
          a.cv1[gi] = c;
        } else {
          v += delta;
        }
        a.v1[gi] = v;
      };
      const int T4 = 4 * blockDim.x;
            for (int q0 = threadIdx.x; q0 < np; q0 += T4) {
        T ox[4], vv[4], cc[4];
        bool fastp[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int pos = q0 + t * blockDim.x;
          fastp[t] = pos < np && !a.b && !(a.pml && a.xA.in(pos));
          if (fastp[t]) {
            const int k = bun.at(l, pos);
            ox[t] = O[k];
            vv[t] = V[k];
            if constexpr (KAHAN) cc[t] = svl[pos];
          }
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int pos = q0 + t * blockDim.x;
          if (!fastp[t]) {
            if (pos < np) one(pos);
            continue;
          }
          const T delta = mulc(ox[t], a.sc, a.sc_lo);
          if constexpr (KAHAN) {
            kahan_add(vv[t], cc[t], delta);
            a.cv1[rb + pos] = cc[t];
          } else {
            vv[t] += delta;
          }
          a.v1[rb + pos] = vv[t];
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------------------------
// Z kernel of the 2-D acoustic step: z part of sub-step A on whole z lines, then tmp = d_z v3.  One tile is one
// bundle `bid` of neighbouring z lines.
template <typename T, int LOGC, bool KAHAN>
__device__ __forceinline__ void ac_z_tile(const AcZArgs<T>& a, int bid, unsigned char* sm,
                                          const ChunkClasses<T, 1 << LOGC>& cc) {
  constexpr int C = 1 << LOGC;
  const LineGeom& g = a.g;
  Carve<T> cv(sm, g, 2, 0);
  T* S = cv.buf[0];  // sigma, then v3 (new)
  T* O = cv.buf[1];
  const Bundle<LOGC, true> bun{g.pitch};
  const WorkMap<true> wm{g.L, g.p, g.NC};
  const int logL = log2_pow2(g.L);
  const int nvalid = bundle_bases<true>(g, bid, cv.lb);
  const int np = g.n + 1;
  const int p1 = g.p + 1;
  __syncthreads();
  {
    // L2 prefetch of the bundle's segments of every array read later (segments of L elements start on
    // L * sizeof(T)-byte boundaries of the padded layout).
    const T* arrs[3] = {a.v3, a.b, a.cv3};
    const uint32_t sb = (uint32_t)(g.L * sizeof(T));
    if ((sb & 15u) == 0)
      for (int i = threadIdx.x; i < 3 * np; i += blockDim.x) {
        const T* base = arrs[i / np];
        if (base) prefetch_l2(base + cv.lb[0] + (int64_t)(i % np) * g.pstride, sb);
      }
  }
  stage_padded<T, true>(a.sigma, S, bun, g, cv.lb, nvalid, logL);
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  pmbc_phi<T, 16>(S, bun, g.L, nvalid, g.n, g.p, g.M, g.n_nb, a.tb.W, cv.phi);
  __syncthreads();
  solve_bundle<T, C, true>(S, O, cv.sA, &cc, bun, wm, nvalid, g.M, a.tb.t32, a.tb.t64, a.minf, RhsD1{},
                           BndPhi<T>{cv.phi, p1});
  // update of v3; lines are handled in groups of four neighbouring x (16-byte vectors) where possible
  const int lg = g.L >= 4 ? logL - 2 : 0;   // log2 of the number of 4-line groups per position
  const int wl = g.L >= 4 ? 4 : g.L;        // lines per item
  auto one = [&](int l, int pos) {
    const int64_t gi = cv.lb[l] + (int64_t)pos * g.pstride;
    const T gz = mulc(O[bun.at(l, pos)], a.s3h, a.s3h_lo);  // d_z sigma
    const T bb = a.b ? a.b[gi] : a.b0;
    T inc;
    if (a.pml && a.zA.in(pos)) {
      const T ih = a.dlt ? a.zA.half(a.psiz, gi, pos, gz) : T(0);
      inc = a.zA.step(a.psiz, gi, pos, gz);
      if (a.dlt) a.dlt[gi] = bb * (ih - T(0.5) * inc);
    } else {
      inc = -mulc(gz, a.acoef, a.acoef_lo);
    }
    const T delta = a.b ? bb * inc : mulc(inc, a.b0, a.b0_lo);
    T vv = a.v3[gi];
    if constexpr (KAHAN) {
      float cc = a.cv3[gi];
      kahan_add(vv, cc, delta);
      a.cv3[gi] = cc;
    } else {
      vv += delta;
    }
    a.v3[gi] = vv;
    S[bun.at(l, pos)] = vv;
  };
  const int items = np << lg;
    for (int i = threadIdx.x; i < items; i += blockDim.x) {
    const int pos = i >> lg;
    const int l0 = (i & ((1 << lg) - 1)) * wl;
    if (g.L < 4 || l0 + 3 >= nvalid || a.b || (a.pml && a.zA.in(pos))) {
      for (int t = 0; t < wl; ++t)
        if (l0 + t < nvalid) one(l0 + t, pos);
      continue;
    }
    const int64_t gi = cv.lb[l0] + (int64_t)pos * g.pstride;
    const int k = bun.at(l0, pos);
    T v[4], c[4], o[4];
    ld4(a.v3 + gi, v);
    if constexpr (KAHAN) ld4(a.cv3 + gi, c);
    ld4(O + k, o);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const T delta = mulc(o[t], a.sc, a.sc_lo);
      if constexpr (KAHAN) {
        kahan_add(v[t], c[t], delta);
      } else {
        v[t] += delta;
      }
    }
    st4(a.v3 + gi, v);
    if constexpr (KAHAN) st4(a.cv3 + gi, c);
    st4(S + k, v);
  }
  __syncthreads();
  if (!a.do_tmp) return;
  pmbc_phi<T, 16>(S, bun, g.L, nvalid, g.n, g.p, g.M, g.n_nb, a.tb.W, cv.phi);
  __syncthreads();
  solve_bundle<T, C, true>(S, O, cv.sA, &cc, bun, wm, nvalid, g.M, a.tb.t32, a.tb.t64, a.minf, RhsD1{},
                           BndPhi<T>{cv.phi, p1});
  for (int i = threadIdx.x; i < items; i += blockDim.x) {
    const int pos = i >> lg;
    const int l0 = (i & ((1 << lg) - 1)) * wl;
    if (g.L < 4 || l0 + 3 >= nvalid) {
      for (int t = 0; t < wl; ++t)
        if (l0 + t < nvalid) a.tmp[cv.lb[l0 + t] + (int64_t)pos * g.pstride] = mulc(O[bun.at(l0 + t, pos)], a.s3h, a.s3h_lo);
      continue;
    }
    T o[4];
    ld4(O + bun.at(l0, pos), o);
#pragma unroll
    for (int t = 0; t < 4; ++t) o[t] = mulc(o[t], a.s3h, a.s3h_lo);
    st4(a.tmp + cv.lb[l0] + (int64_t)pos * g.pstride, o);
  }
}

// ---------------------------------------------------------------------------------------------------------------
// Kernels: one launch per shot (a tile per block), and one persistent launch over the tiles of all shots of a
// handle (tile t of the concatenated tile list; the block copies the shot's descriptor into shared memory and
// rebuilds its chunk classes when the shot changes).  The batched kernels read the descriptor from shared memory
// instead of the parameter bank, which costs registers, so their blocks are capped at kBatchThreads threads.
template <typename T, int LOGC, bool KAHAN>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 512 : 1024) k_ac_x(AcXArgs<T> a) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ ChunkClasses<T, 1 << LOGC> cc;
  chunk_classes_init<T, 1 << LOGC>(&cc, a.g.M, a.g.NC, a.tb.t32, a.tb.t64, a.minf);
  ac_x_tile<T, LOGC, KAHAN>(a, blockIdx.x, sm, cc);
}

template <typename T, int LOGC, bool KAHAN>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 512 : 1024) k_ac_z(AcZArgs<T> a) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ ChunkClasses<T, 1 << LOGC> cc;
  chunk_classes_init<T, 1 << LOGC>(&cc, a.g.M, a.g.NC, a.tb.t32, a.tb.t64, a.minf);
  ac_z_tile<T, LOGC, KAHAN>(a, blockIdx.x, sm, cc);
}

template <typename T, int LOGC, bool KAHAN>
__global__ void __launch_bounds__(kBatchThreads)
    k_ac_x_batch(const AcXArgs<T>* __restrict__ tab, const int* __restrict__ tile0, int nshots, int ntiles) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ ChunkClasses<T, 1 << LOGC> cc;
  __shared__ __align__(16) unsigned char sa_raw[sizeof(AcXArgs<T>)];
  __shared__ int s_shot;
  AcXArgs<T>& sa = *reinterpret_cast<AcXArgs<T>*>(sa_raw);
  int cur = -1;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    if (threadIdx.x == 0) s_shot = tile_shot(tile0, nshots, t);
    __syncthreads();
    const int shot = s_shot;
    if (shot != cur) {
      copy_args(&sa, tab + shot);
      __syncthreads();
      chunk_classes_init<T, 1 << LOGC>(&cc, sa.g.M, sa.g.NC, sa.tb.t32, sa.tb.t64, sa.minf);
      cur = shot;
    }
    ac_x_tile<T, LOGC, KAHAN>(sa, t - tile0[shot], sm, cc);
    __syncthreads();
  }
}

template <typename T, int LOGC, bool KAHAN>
__global__ void __launch_bounds__(kBatchThreads)
    k_ac_z_batch(const AcZArgs<T>* __restrict__ tab, const int* __restrict__ tile0, int nshots, int ntiles) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ ChunkClasses<T, 1 << LOGC> cc;
  __shared__ __align__(16) unsigned char sa_raw[sizeof(AcZArgs<T>)];
  __shared__ int s_shot;
  AcZArgs<T>& sa = *reinterpret_cast<AcZArgs<T>*>(sa_raw);
  int cur = -1;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    if (threadIdx.x == 0) s_shot = tile_shot(tile0, nshots, t);
    __syncthreads();
    const int shot = s_shot;
    if (shot != cur) {
      copy_args(&sa, tab + shot);
      __syncthreads();
      chunk_classes_init<T, 1 << LOGC>(&cc, sa.g.M, sa.g.NC, sa.tb.t32, sa.tb.t64, sa.minf);
      cur = shot;
    }
    ac_z_tile<T, LOGC, KAHAN>(sa, t - tile0[shot], sm, cc);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------------------------
// Receiver gather.  mode 0: out[r] = f[idx[r]].  mode 1 (velocities, staggered state): out holds v_{n+1/2} and
// f holds v_{n+3/2}; the integer-time value is v_{n+1/2} + (v_{n+3/2} - v_{n+1/2}) / 2 plus, inside absorbing
// layers where the exponential sub-flow is not linear in the step length, the corrections d0..d2 (may be null).
template <typename T>
__global__ void k_gather(const T* __restrict__ f, const int64_t* __restrict__ idx, int64_t n, T* __restrict__ out,
                         int mode, const T* __restrict__ d0, const T* __restrict__ d1, const T* __restrict__ d2) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = idx[r];
    const T v = f[q];
    if (mode == 0) {
      out[r] = v;
    } else {
      T c = T(0);
      if (d0) c += d0[q];
      if (d1) c += d1[q];
      if (d2) c += d2[q];
      out[r] = out[r] + T(0.5) * (v - out[r]) + c;
    }
  }
}

// All receiver gathers of one phase of a batched step: job blockIdx.y, trace row from the shot's device clock.
template <typename T>
__global__ void k_gather_batch(const GatherJob<T>* __restrict__ jobs) {
  const GatherJob<T>& j = jobs[blockIdx.y];
  T* out = j.trace + j.clk->row * j.n_rcv + j.off;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < j.cnt; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = j.idx[r];
    const T v = j.f[q];
    if (j.mode == 0) {
      out[r] = v;
    } else {
      T c = T(0);
      if (j.d[0]) c += j.d[0][q];
      if (j.d[1]) c += j.d[1][q];
      if (j.d[2]) c += j.d[2][q];
      out[r] = out[r] + T(0.5) * (v - out[r]) + c;
    }
  }
}

// End of a batched step: advance every shot's device clock.
__global__ void k_tick(StepClock* __restrict__ c, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    c[i].step += 1;
    c[i].row += c[i].row_inc;
  }
}

// ---------------------------------------------------------------------------------------------------------------
// Host launchers.
size_t smem_bytes(const LineGeom& g, int nbuf, int nstage, size_t esize) {
  const size_t nw = (size_t)g.L * g.p * g.NC;
  size_t b = (size_t)nbuf * g.buf * esize;
  b = (b + 15) & ~size_t(15);
  b += (size_t)nstage * g.stage * esize;
  b = (b + 15) & ~size_t(15);
  b += 2 * nw * esize;
  b = (b + 15) & ~size_t(15);
  b += (size_t)g.L * (g.p + 1) * sizeof(double);
  b = (b + 15) & ~size_t(15);
  b += (size_t)g.L * sizeof(int64_t);
  return b + 16;
}

template <class K>
static cudaError_t launch(K kern, int grid, int threads, size_t smem, cudaStream_t st, void* args) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* argv[] = {args};
  return cudaLaunchKernel((const void*)kern, dim3(grid), dim3(threads), argv, smem, st);
}

template <typename T>
cudaError_t launch_deriv(const DerivArgs<T>& a, int logc, bool sflav, int threads, cudaStream_t st) {
  const size_t smem = smem_bytes(a.g, a.d2 ? 3 : 2, 0, sizeof(T));
  DerivArgs<T> args = a;
  if (sflav) {
    if (logc == 3 && sizeof(T) == 4) return launch(k_deriv<T, 3, true>, a.g.nbundles, threads, smem, st, &args);
    return launch(k_deriv<T, 4, true>, a.g.nbundles, threads, smem, st, &args);
  }
  if (logc == 3 && sizeof(T) == 4) return launch(k_deriv<T, 3, false>, a.g.nbundles, threads, smem, st, &args);
  return launch(k_deriv<T, 4, false>, a.g.nbundles, threads, smem, st, &args);
}

template <typename T, bool KAHAN>
cudaError_t launch_ac_x(const AcXArgs<T>& a, int logc, int threads, cudaStream_t st) {
  const size_t smem = smem_bytes(a.g, 3, 4, sizeof(T));
  AcXArgs<T> args = a;
  if (logc == 3 && sizeof(T) == 4) return launch(k_ac_x<T, 3, KAHAN>, a.g.nbundles, threads, smem, st, &args);
  return launch(k_ac_x<T, 4, KAHAN>, a.g.nbundles, threads, smem, st, &args);
}

template <typename T, bool KAHAN>
cudaError_t launch_ac_z(const AcZArgs<T>& a, int logc, int threads, cudaStream_t st) {
  const size_t smem = smem_bytes(a.g, 2, 0, sizeof(T));
  AcZArgs<T> args = a;
  if (logc == 3 && sizeof(T) == 4) return launch(k_ac_z<T, 3, KAHAN>, a.g.nbundles, threads, smem, st, &args);
  return launch(k_ac_z<T, 4, KAHAN>, a.g.nbundles, threads, smem, st, &args);
}

// Persistent launches: as many blocks as fit on the device at once (at most one per tile), each looping over
// tiles.  The grid size and the shared-memory attribute are set up front (outside any graph capture).
template <class K>
static cudaError_t persistent_grid(K kern, int ntiles, int threads, size_t smem, int num_sms, int* grid) {
  *grid = 0;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  *grid = ntiles < per_sm * num_sms ? ntiles : per_sm * num_sms;
  return cudaSuccess;
}

template <typename T, bool KAHAN>
cudaError_t batch_grid_ac_x(int logc, int threads, size_t smem, int ntiles, int num_sms, int* grid) {
  if (logc == 3 && sizeof(T) == 4) return persistent_grid(k_ac_x_batch<T, 3, KAHAN>, ntiles, threads, smem, num_sms, grid);
  return persistent_grid(k_ac_x_batch<T, 4, KAHAN>, ntiles, threads, smem, num_sms, grid);
}

template <typename T, bool KAHAN>
cudaError_t batch_grid_ac_z(int logc, int threads, size_t smem, int ntiles, int num_sms, int* grid) {
  if (logc == 3 && sizeof(T) == 4) return persistent_grid(k_ac_z_batch<T, 3, KAHAN>, ntiles, threads, smem, num_sms, grid);
  return persistent_grid(k_ac_z_batch<T, 4, KAHAN>, ntiles, threads, smem, num_sms, grid);
}

template <typename T, bool KAHAN>
cudaError_t launch_ac_x_batch(const AcXArgs<T>* tab, const int* tile0, int nshots, int ntiles, int logc, int threads,
                              size_t smem, int grid, cudaStream_t st) {
  if (ntiles <= 0 || grid <= 0) return cudaSuccess;
  void* argv[] = {(void*)&tab, (void*)&tile0, (void*)&nshots, (void*)&ntiles};
  const void* kern = (logc == 3 && sizeof(T) == 4) ? (const void*)k_ac_x_batch<T, 3, KAHAN>
                                                    : (const void*)k_ac_x_batch<T, 4, KAHAN>;
  return cudaLaunchKernel(kern, dim3(grid), dim3(threads), argv, smem, st);
}

template <typename T, bool KAHAN>
cudaError_t launch_ac_z_batch(const AcZArgs<T>* tab, const int* tile0, int nshots, int ntiles, int logc, int threads,
                              size_t smem, int grid, cudaStream_t st) {
  if (ntiles <= 0 || grid <= 0) return cudaSuccess;
  void* argv[] = {(void*)&tab, (void*)&tile0, (void*)&nshots, (void*)&ntiles};
  const void* kern = (logc == 3 && sizeof(T) == 4) ? (const void*)k_ac_z_batch<T, 3, KAHAN>
                                                    : (const void*)k_ac_z_batch<T, 4, KAHAN>;
  return cudaLaunchKernel(kern, dim3(grid), dim3(threads), argv, smem, st);
}

template <typename T>
cudaError_t launch_gather_batch(const GatherJob<T>* jobs, int njobs, int64_t max_cnt, cudaStream_t st) {
  if (njobs <= 0 || max_cnt <= 0) return cudaSuccess;
  const int threads = 256;
  const int64_t bx = (max_cnt + threads - 1) / threads;
  k_gather_batch<T><<<dim3((unsigned)(bx < 1024 ? bx : 1024), (unsigned)njobs), threads, 0, st>>>(jobs);
  return cudaGetLastError();
}

cudaError_t launch_tick(StepClock* c, int n, cudaStream_t st) {
  k_tick<<<(n + 127) / 128, 128, 0, st>>>(c, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gather(const T* f, const int64_t* idx, int64_t n, T* out, int mode, const T* d0, const T* d1,
                          const T* d2, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int threads = 256;
  const int grid = (int)((n + threads - 1) / threads < 4096 ? (n + threads - 1) / threads : 4096);
  k_gather<T><<<grid, threads, 0, st>>>(f, idx, n, out, mode, d0, d1, d2);
  return cudaGetLastError();
}

template cudaError_t launch_deriv<float>(const DerivArgs<float>&, int, bool, int, cudaStream_t);
template cudaError_t launch_deriv<double>(const DerivArgs<double>&, int, bool, int, cudaStream_t);
template cudaError_t launch_ac_x<float, false>(const AcXArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_ac_x<float, true>(const AcXArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_ac_x<double, false>(const AcXArgs<double>&, int, int, cudaStream_t);
template cudaError_t launch_ac_z<float, false>(const AcZArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_ac_z<float, true>(const AcZArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_ac_z<double, false>(const AcZArgs<double>&, int, int, cudaStream_t);
template cudaError_t launch_ac_x_batch<float, false>(const AcXArgs<float>*, const int*, int, int, int, int, size_t, int,
                                    cudaStream_t);
template cudaError_t launch_ac_x_batch<float, true>(const AcXArgs<float>*, const int*, int, int, int, int, size_t, int,
                                    cudaStream_t);
template cudaError_t launch_ac_x_batch<double, false>(const AcXArgs<double>*, const int*, int, int, int, int, size_t, int,
                                    cudaStream_t);
template cudaError_t launch_ac_z_batch<float, false>(const AcZArgs<float>*, const int*, int, int, int, int, size_t, int,
                                    cudaStream_t);
template cudaError_t launch_ac_z_batch<float, true>(const AcZArgs<float>*, const int*, int, int, int, int, size_t, int,
                                    cudaStream_t);
template cudaError_t launch_ac_z_batch<double, false>(const AcZArgs<double>*, const int*, int, int, int, int, size_t, int,
                                    cudaStream_t);
template cudaError_t batch_grid_ac_x<float, false>(int, int, size_t, int, int, int*);
template cudaError_t batch_grid_ac_x<float, true>(int, int, size_t, int, int, int*);
template cudaError_t batch_grid_ac_x<double, false>(int, int, size_t, int, int, int*);
template cudaError_t batch_grid_ac_z<float, false>(int, int, size_t, int, int, int*);
template cudaError_t batch_grid_ac_z<float, true>(int, int, size_t, int, int, int*);
template cudaError_t batch_grid_ac_z<double, false>(int, int, size_t, int, int, int*);
template cudaError_t launch_gather_batch<float>(const GatherJob<float>*, int, int64_t, cudaStream_t);
template cudaError_t launch_gather_batch<double>(const GatherJob<double>*, int, int64_t, cudaStream_t);
template cudaError_t launch_gather<float>(const float*, const int64_t*, int64_t, float*, int, const float*,
                                          const float*, const float*, cudaStream_t);
template cudaError_t launch_gather<double>(const double*, const int64_t*, int64_t, double*, int, const double*,
                                           const double*, const double*, cudaStream_t);

}  // namespace lossk
