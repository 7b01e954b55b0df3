// sm_103a kernels of the 3-D elastic LOSS step (paper Sec. 2 velocity-stress system, Sec. 3.3 Strang
// splitting with the exponential ADE-PML sub-flows).
//
// With the velocities half a step ahead (staggered state), one step is five line passes, each of which holds
// whole lines of three fields along one axis on chip, closes them with the PMBC and solves them:
//   BX (x lines):  TA = X[v1,x], TB = X[v2,x], TC = X[v3,x]
//   BY (y lines):  TD = X[v2,y], TB += X[v1,y], TE = X[v3,y]
//   BZ (z lines):  sigma_ii += lambda (TA + TD + X[v3,z]) + 2 mu X_ii,  sigma_12 += mu TB,
//                  sigma_13 += mu (TC + X[v1,z]),  sigma_23 += mu (TE + X[v2,z]),  + source      [sub-step B]
//                  then, on the new stresses still on chip: UA = Y[s13,z], UB = Y[s23,z], UC = Y[s33,z]
//   AX (x lines):  UA += Y[s11,x], UB += Y[s12,x], UC += Y[s13,x]
//   AY (y lines):  v1 += b (UA + Y[s12,y]), v2 += b (UB + Y[s22,y]), v3 += b (UC + Y[s23,y])   [sub-step A]
// X[f,a] = dt * d_a f and Y[f,a] = tau_A * d_a f outside the absorbing layers; inside, the exact integral of the
// stretched derivative over the sub-step, -PmlAxis::step(...), which also advances that term's memory variable.
#include <cuda_runtime.h>

#include "../../include/loss.h"
#include "loss_block.cuh"
#include "loss_fir.cuh"
#include "loss_line.cuh"
#include "loss_tile.cuh"
#include "loss_types.h"

namespace lossk {

enum { EL_BX = 0, EL_BY = 1, EL_BZ = 2, EL_AX = 3, EL_AY = 4 };

size_t smem_bytes(const LineGeom& g, int nbuf, int nstage, size_t esize);  // loss_kernels_acoustic.cu

// tau times the (stretched) derivative g along this pass's axis at line position pos.
template <typename T>
__device__ __forceinline__ T eff(int pml, const PmlAxis<T>& pa, T* mem, int64_t gi, int pos, T g, T tau, T tau_lo) {
  return (pml && pa.in(pos)) ? -pa.step(mem, gi, pos, g) : mulc(g, tau, tau_lo);
}

// Velocity-sub-step term: returns tau * (stretched derivative); in a layer with receiver corrections on, also
// stores b (X(tau/2) - X(tau)/2), the amount by which the first half of the step differs from half of it.
template <typename T>
__device__ __forceinline__ T effA(const ElArgs<T>& a, int term, int64_t gi, int pos, T g, T tau) {
  if (!(a.pml && a.pA.in(pos))) return mulc(g, tau, a.acoef_lo);
  T xh = T(0);
  const bool rec = a.dlt[term] != nullptr;
  if (rec) xh = -a.pA.half(a.memA[term], gi, pos, g);
  const T xf = -a.pA.step(a.memA[term], gi, pos, g);
  if (rec) a.dlt[term][gi] = (a.b ? a.b[gi] : a.b0) * (xh - T(0.5) * xf);
  return xf;
}

// u += delta in registers (compensated with c when KAHAN); the caller loads and stores.
template <typename T, bool KAHAN>
__device__ __forceinline__ void upd_r(T& u, T& c, T delta) {
  if constexpr (KAHAN) {
    float cc = c;
    kahan_add(u, cc, delta);
    c = cc;
  } else {
    u += delta;
  }
}


template <typename T, int LOGC, bool SFLAV, int PASS, bool KAHAN>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 512 : 1024) k_el(ElArgs<T> a) {
  constexpr int C = 1 << LOGC;
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ ChunkClasses<T, C> cc;
  const LineGeom& g = a.g;
  Carve<T> cv(sm, g, 6, 0);
  T* F[3] = {cv.buf[0], cv.buf[1], cv.buf[2]};
  T* O[3] = {cv.buf[3], cv.buf[4], cv.buf[5]};
  const Bundle<LOGC, SFLAV> bun{g.pitch};
  const WorkMap<SFLAV> wm{g.L, g.p, g.NC};
  const int logL = SFLAV ? (__ffs(g.L) - 1) : 0;
  const int nvalid = bundle_bases<SFLAV>(g, blockIdx.x, cv.lb);
  const int p1 = g.p + 1;
  chunk_classes_init<T, C>(&cc, g.M, g.NC, a.tb.t32, a.tb.t64, a.minf);
  __syncthreads();
  if (!SFLAV) {
    // the arrays the pointwise phase reads, into L2 while the rows are staged and solved (one bulk prefetch per
    // row; on the y / z bundles the per-position 32-byte segments cost more than they save, measured)
    const T* pre[20];
    int np_ = 0;
    T* const* tt = a.tmp;
    if (PASS == EL_BY) {
      pre[np_++] = tt[1];
    } else if (PASS == EL_BZ && a.do_B) {
      const int fs[6] = {LOSS_FIELD_S11, LOSS_FIELD_S22, LOSS_FIELD_S12, LOSS_FIELD_S13, LOSS_FIELD_S23,
                         LOSS_FIELD_S33};
      pre[np_++] = tt[0], pre[np_++] = tt[1], pre[np_++] = tt[2], pre[np_++] = tt[3], pre[np_++] = tt[4];
      pre[np_++] = a.lam, pre[np_++] = a.mu;
      for (int f = 0; f < 6; ++f) {
        pre[np_++] = a.fld[fs[f]];
        if (KAHAN) pre[np_++] = a.cmp[fs[f]];
      }
    } else if (PASS == EL_AX) {
      pre[np_++] = tt[5], pre[np_++] = tt[6], pre[np_++] = tt[7];
    } else if (PASS == EL_AY) {
      pre[np_++] = tt[5], pre[np_++] = tt[6], pre[np_++] = tt[7], pre[np_++] = a.b;
      for (int f = LOSS_FIELD_V1; f <= LOSS_FIELD_V3; ++f) {
        pre[np_++] = a.fld[f];
        if (KAHAN) pre[np_++] = a.cmp[f];
      }
    }
    prefetch_bundle<T, SFLAV>(g, cv.lb, nvalid, pre, np_);
  }
  // the first field in a copy group of its own: its PMBC sums and solve run while the other two stream in
  stage_padded<T, SFLAV>(a.src[0], F[0], bun, g, cv.lb, nvalid, logL);
  cp_async_commit();
  for (int s = 1; s < 3; ++s) stage_padded<T, SFLAV>(a.src[s], F[s], bun, g, cv.lb, nvalid, logL);
  cp_async_commit();
  cp_async_wait<1>();
  __syncthreads();
  auto derive = [&](int s) {
    pmbc_phi<T, 16>(F[s], bun, g.L, nvalid, g.n, g.p, g.M, g.n_nb, a.tb.W, cv.phi);
    __syncthreads();
    solve_bundle<T, C, SFLAV>(F[s], O[s], cv.sA, &cc, bun, wm, nvalid, g.M, a.tb.t32, a.tb.t64, a.minf, RhsD1{},
                              BndPhi<T>{cv.phi, p1});
  };
  derive(0);
  cp_async_wait<0>();
  __syncthreads();
  for (int s = 1; s < 3; ++s) derive(s);
  const T dt = a.dt, ta = a.acoef;
  T* const* t = a.tmp;
  if (PASS == EL_BX) {
    for_points<SFLAV>(g, cv.lb, nvalid, logL, [&](int l, int pos, int64_t gi) {
      const int k = bun.at(l, pos);
      t[0][gi] = eff(a.pml, a.pB, a.memB[0], gi, pos, mulc(O[0][k], a.s3h, a.s3h_lo), dt, a.dt_lo);
      t[1][gi] = eff(a.pml, a.pB, a.memB[1], gi, pos, mulc(O[1][k], a.s3h, a.s3h_lo), dt, a.dt_lo);
      t[2][gi] = eff(a.pml, a.pB, a.memB[2], gi, pos, mulc(O[2][k], a.s3h, a.s3h_lo), dt, a.dt_lo);
    });
  } else if (PASS == EL_BY) {
    for_points<SFLAV>(g, cv.lb, nvalid, logL, [&](int l, int pos, int64_t gi) {
      const int k = bun.at(l, pos);
      const T t1 = t[1][gi];  // loaded before any store (see EL_BZ)
      const T x0 = eff(a.pml, a.pB, a.memB[0], gi, pos, mulc(O[0][k], a.s3h, a.s3h_lo), dt, a.dt_lo);
      const T x1 = eff(a.pml, a.pB, a.memB[1], gi, pos, mulc(O[1][k], a.s3h, a.s3h_lo), dt, a.dt_lo);
      const T x2 = eff(a.pml, a.pB, a.memB[2], gi, pos, mulc(O[2][k], a.s3h, a.s3h_lo), dt, a.dt_lo);
      t[1][gi] = t1 + x0;
      t[3][gi] = x1;
      t[4][gi] = x2;
    });
  } else if (PASS == EL_BZ) {
    if (a.do_B) {
      const int outer = blockIdx.x / g.nxb;           // y index of the bundle
      const int x0 = (blockIdx.x - outer * g.nxb) * g.L;
      for_points<SFLAV>(g, cv.lb, nvalid, logL, [&](int l, int pos, int64_t gi) {
        const int k = bun.at(l, pos);
        // every global operand of the point first (the arrays may alias as far as the compiler knows, so loads
        // after the first store would wait for it), then the arithmetic, then the stores
        const int fs[6] = {LOSS_FIELD_S11, LOSS_FIELD_S22, LOSS_FIELD_S12, LOSS_FIELD_S13, LOSS_FIELD_S23,
                           LOSS_FIELD_S33};
        T u[6], cu[6];
#pragma unroll
        for (int f = 0; f < 6; ++f) {
          u[f] = a.fld[fs[f]][gi];
          cu[f] = KAHAN ? a.cmp[fs[f]][gi] : T(0);
        }
        const T xa = t[0][gi], xd = t[3][gi], tc = t[2][gi], tb = t[1][gi], te = t[4][gi];
        const T lam = a.lam ? a.lam[gi] : a.lam0;
        const T mu = a.mu ? a.mu[gi] : a.mu0;
        const T x13 = eff(a.pml, a.pB, a.memB[0], gi, pos, mulc(O[0][k], a.s3h, a.s3h_lo), dt, a.dt_lo);  // v1 along z
        const T x23 = eff(a.pml, a.pB, a.memB[1], gi, pos, mulc(O[1][k], a.s3h, a.s3h_lo), dt, a.dt_lo);  // v2 along z
        const T x33 = eff(a.pml, a.pB, a.memB[2], gi, pos, mulc(O[2][k], a.s3h, a.s3h_lo), dt, a.dt_lo);  // v3 along z
        // constant moduli enter through mulc (their rounding errors would bias every update the same way)
        auto mlam = [&](T x) { return a.lam ? lam * x : mulc(x, a.lam0, a.lam0_lo); };
        auto mmu = [&](T x) { return a.mu ? mu * x : mulc(x, a.mu0, a.mu0_lo); };
        const T ltr = mlam(xa + xd + x33);
        T s11 = ltr + T(2) * mmu(xa), s22 = ltr + T(2) * mmu(xd), s33 = ltr + T(2) * mmu(x33);
        T s13 = mmu(tc + x13);
        if (a.srcp.on) {
          const int dz = pos - a.srcp.zs + 12, dy = outer - a.srcp.ys + 12, dx = x0 + l - a.srcp.xs + 12;
          if ((unsigned)dz < 25u && (unsigned)dy < 25u && (unsigned)dx < 25u) {
            const T sv = (T)(a.srcp.amp * a.srcp.g[dz] * a.srcp.g[dy] * a.srcp.g[dx]);
            if (a.src_explosive) s11 += sv, s22 += sv, s33 += sv;
            if (a.src_shear) s13 += sv;
          }
        }
        const T d[6] = {s11, s22, mmu(tb), s13, mmu(te + x23), s33};
#pragma unroll
        for (int f = 0; f < 6; ++f) upd_r<T, KAHAN>(u[f], cu[f], d[f]);
#pragma unroll
        for (int f = 0; f < 6; ++f) {
          a.fld[fs[f]][gi] = u[f];
          if (KAHAN) a.cmp[fs[f]][gi] = cu[f];
        }
        // new stresses needed by the velocity sub-step's z derivatives stay on chip
        F[0][k] = u[3];
        F[1][k] = u[4];
        F[2][k] = u[5];
      });
      __syncthreads();
      if (a.do_A)
        for (int s = 0; s < 3; ++s) derive(s);
    }
    if (a.do_A) {
      for_points<SFLAV>(g, cv.lb, nvalid, logL, [&](int l, int pos, int64_t gi) {
        const int k = bun.at(l, pos);
        t[5][gi] = effA(a, 0, gi, pos, mulc(O[0][k], a.s3h, a.s3h_lo), ta);
        t[6][gi] = effA(a, 1, gi, pos, mulc(O[1][k], a.s3h, a.s3h_lo), ta);
        t[7][gi] = effA(a, 2, gi, pos, mulc(O[2][k], a.s3h, a.s3h_lo), ta);
      });
    }
  } else if (PASS == EL_AX) {
    for_points<SFLAV>(g, cv.lb, nvalid, logL, [&](int l, int pos, int64_t gi) {
      const int k = bun.at(l, pos);
      const T t5 = t[5][gi], t6 = t[6][gi], t7 = t[7][gi];  // loaded before any store (see EL_BZ)
      const T y0 = effA(a, 0, gi, pos, mulc(O[0][k], a.s3h, a.s3h_lo), ta);
      const T y1 = effA(a, 1, gi, pos, mulc(O[1][k], a.s3h, a.s3h_lo), ta);
      const T y2 = effA(a, 2, gi, pos, mulc(O[2][k], a.s3h, a.s3h_lo), ta);
      t[5][gi] = t5 + y0;
      t[6][gi] = t6 + y1;
      t[7][gi] = t7 + y2;
    });
  } else if (PASS == EL_AY) {
    const int outer = blockIdx.x / g.nxb;  // z index of the bundle
    const int x0 = (blockIdx.x - outer * g.nxb) * g.L;
    for_points<SFLAV>(g, cv.lb, nvalid, logL, [&](int l, int pos, int64_t gi) {
      const int k = bun.at(l, pos);
      const T b = a.b ? a.b[gi] : a.b0;
      T force = T(0);  // body force (FORCE_X/Y/Z sources), already multiplied by the sub-step length
      if (a.srcp.on) {
        const int dz = outer - a.srcp.zs + 12, dy = pos - a.srcp.ys + 12, dx = x0 + l - a.srcp.xs + 12;
        if ((unsigned)dz < 25u && (unsigned)dy < 25u && (unsigned)dx < 25u)
          force = (T)(a.srcp.amp * a.srcp.g[dz] * a.srcp.g[dy] * a.srcp.g[dx]);
      }
      const T f0 = (a.force_mask & 1) ? force : T(0), f1 = (a.force_mask & 2) ? force : T(0),
              f2 = (a.force_mask & 4) ? force : T(0);
      T u[3], cu[3];
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        u[f] = a.fld[LOSS_FIELD_V1 + f][gi];
        cu[f] = KAHAN ? a.cmp[LOSS_FIELD_V1 + f][gi] : T(0);
      }
      const T t5 = t[5][gi], t6 = t[6][gi], t7 = t[7][gi];
      auto mb = [&](T x) { return a.b ? b * x : mulc(x, a.b0, a.b0_lo); };
      const T d0 = mb(t5 + effA(a, 0, gi, pos, mulc(O[0][k], a.s3h, a.s3h_lo), ta) + f0);
      const T d1 = mb(t6 + effA(a, 1, gi, pos, mulc(O[1][k], a.s3h, a.s3h_lo), ta) + f1);
      const T d2 = mb(t7 + effA(a, 2, gi, pos, mulc(O[2][k], a.s3h, a.s3h_lo), ta) + f2);
      upd_r<T, KAHAN>(u[0], cu[0], d0);
      upd_r<T, KAHAN>(u[1], cu[1], d1);
      upd_r<T, KAHAN>(u[2], cu[2], d2);
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        a.fld[LOSS_FIELD_V1 + f][gi] = u[f];
        if (KAHAN) a.cmp[LOSS_FIELD_V1 + f][gi] = cu[f];
      }
    });
  }
}

// ---------------------------------------------------------------------------------------------------------------
// y and z passes of the FP32 step on one-patch tiles, in the truncated-convolution form of loss_fir.cuh (the 2-D z
// tiles' arithmetic): a block takes 32 neighbouring x columns by one patch of the pass axis plus a halo of
// H = max(n_nb, K) positions on each side, for one index of the remaining axis.  It stages the pass's three source
// fields (128-byte row segments), forms the FP64 junction corrections of the patch's two junctions for each field,
// computes the three derivatives of its chunk in registers and applies the pass's pointwise update:
//   ET_BY (y):  TB += X[v1,y], TD = X[v2,y], TE = X[v3,y]
//   ET_BZ (z):  the stress sub-step (as EL_BZ with do_B) from TA..TE and X[v1..v3, z], + source
//   ET_AZ (z):  UA = Y[s13,z], UB = Y[s23,z], UC = Y[s33,z] (from the new stresses)
//   ET_AY (y):  v_i += b (U_i + Y[s_i2, y]) (as EL_AY), + body force
// Tiles are independent: no block holds a whole line.  The z part of the velocity sub-step is a pass of its own
// (the line kernel computes it on the stresses BZ leaves on chip; a tile has no neighbour's new stresses).
// Junction corrections of the three staged fields of a tile: D[s][J] = sum_m Wd[J][m] f_s[jM + m] for the tile's two
// junctions J, accumulated in FP64 with the 32 columns on the lanes.  Items (field, junction, tap subset) go round
// the warps (ns = min(8, max(1, warps / 6)) subsets per field and junction); partial sums meet in partf.  Contains
// no barrier: partf is complete after the caller's next barrier, and elt_junction_reduce then forms dl.
__device__ __forceinline__ void elt_junction_parts(const float* __restrict__ F, int fstride, const ZBun& bun,
                                                   int nvalid, int l, const TileGeom& t, int ns,
                                                   const double* __restrict__ wsm, double* __restrict__ partf) {
  const int col = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int wl = 2 * t.Rd + 1;
  for (int it = w; it < 6 * ns; it += nw) {  // item = ((field, junction), subset)
    const int fj = it % 6, sub = it / 6;
    const int s = fj >> 1, J = fj & 1;
    const int c = (l + J) * t.M;
    const int mlo = max(-t.Rd, -c);
    const int mhi = min(t.Rd, t.n - c);
    const double* wj = wsm + J * wl + t.Rd;
    const float* Fs = F + s * fstride;
    double a = 0.0, b = 0.0;  // two independent accumulators halve the FP64 dependency chain
    if (col < nvalid) {
      int m = mlo + sub;
      for (; m + ns <= mhi; m += 2 * ns) {
        a = fma(wj[m], widen(Fs[bun.at(col, c + m)]), a);
        b = fma(wj[m + ns], widen(Fs[bun.at(col, c + m + ns)]), b);
      }
      if (m <= mhi) a = fma(wj[m], widen(Fs[bun.at(col, c + m)]), a);
    }
    partf[(fj * ns + sub) * 32 + col] = a + b;
  }
}
__device__ __forceinline__ void elt_junction_reduce(const double* __restrict__ partf, int ns, float* __restrict__ dl) {
  for (int i = threadIdx.x; i < 6 * 32; i += blockDim.x) {  // (field, junction) x column
    const int fj = i >> 5, cl = i & 31;
    double acc = 0.0;
    for (int q = 0; q < ns; ++q) acc += partf[(fj * ns + q) * 32 + cl];
    dl[(fj >> 1) * 64 + 2 * cl + (fj & 1)] = (float)acc;
  }
}

// 8-position chunks up to M = 64 (at most 8 warps, 3 blocks per SM), 16-position chunks up to M = 256.
template <int PASS, bool KAHAN, int LOGC>
__global__ void __launch_bounds__(LOGC == 3 ? 256 : 512, LOGC == 3 ? 3 : 1) k_elt(ElArgs<float> a, ElTile g) {
  constexpr int C = 1 << LOGC;
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ float rpow[kFirPow];
  __shared__ float dl[3 * 64];
  __shared__ double partf[6 * 8 * 32];
  __shared__ double wsm[2 * 129];
  const TileGeom& t = g.t;
  const int l = blockIdx.x % t.p;
  const int rest = blockIdx.x / t.p;
  const int cg = rest % g.ncg;
  const int outer = rest / g.ncg;
  const int x0 = cg * 32;
  const int z0 = l * t.M;  // the patch along the pass axis
  const int zb = z0 - t.H;
  const int rows = t.M + 2 * t.H + 1;
  const int nch = (t.M + C - 1) / C;
  const bool last = l == t.p - 1;
  const int64_t obase = (int64_t)outer * g.ostride + x0;
  const int fstride = rows * 32;
  float* F = reinterpret_cast<float*>(sm);  // three fields, [rows][32] each
  float* PA = F + 3 * fstride;              // [field][chunk][32] warm-up partial sums
  float* PB = PA + 3 * nch * 32;
  fill_rpow(rpow, t.r);
  {
    const int wl = 2 * t.Rd + 1;
    for (int i = threadIdx.x; i < 2 * wl; i += blockDim.x) wsm[i] = t.Wd[(size_t)l * wl + i];
  }
  for (int s = 0; s < 3; ++s) {
    const float* f = a.src[s] + obase;
    float* Fs = F + s * fstride;
    for (int i = threadIdx.x; i < rows * 8; i += blockDim.x) {
      const int q = i >> 3, seg = i & 7;
      const int pos = zb + q;
      if (pos >= 0 && pos <= t.n) cp_async<16>(Fs + q * 32 + seg * 4, f + (int64_t)pos * t.px + seg * 4);
    }
  }
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  const ZBun bun{zb};
  const int nvalid = min(32, g.nx - x0);
  const int ns = min(8, max(1, (int)(blockDim.x >> 5) / 6));
  const int col = threadIdx.x & 31;
  const int c = threadIdx.x >> 5;
  const int p0 = z0 + c * C;
  const int len = min(C, z0 + t.M - p0);
  const int lenx = len + ((len > 0 && last && p0 + len == t.n) ? 1 : 0);  // with the line's last point
  const bool mine = len > 0 && col < nvalid;
  // one phase for the FP64 junction sums and the warm-up partial sums of all three fields
  elt_junction_parts(F, fstride, bun, nvalid, l, t, ns, wsm, partf);
  if (mine && len == C) {
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      float fv[C + 1];
#pragma unroll
      for (int j = 0; j < C; ++j) fv[j] = F[s * fstride + bun.at(col, p0 + j)];
      chunk_partials<C>(fv, t.r, PA[(s * nch + c) * 32 + col], PB[(s * nch + c) * 32 + col]);
    }
  }
  __syncthreads();
  elt_junction_reduce(partf, ns, dl);
  __syncthreads();
  constexpr int W = FirLen<float>::K / C;
  const float rC = rpow[C];
  float e[3][C + 1];
  if (mine) {
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const float* Fs = F + s * fstride;
      const float* PAs = PA + s * nch * 32;
      const float* PBs = PB + s * nch * 32;
      float fv[C + 1];
#pragma unroll
      for (int j = 0; j <= C; ++j)
        if (j < lenx) fv[j] = Fs[bun.at(col, p0 + j)];
      float sL, qR;
      if (c >= W) {
        sL = PAs[(c - 1) * 32 + col];
        if (W == 2) sL += rC * PAs[(c - 2) * 32 + col];
      } else {
        sL = fir_left<float, FirLen<float>::K>(Fs, bun, col, p0, t.n, t.r);
      }
      if (lenx == C && (c + W + 1) * C <= t.M) {
        qR = PBs[(c + 1) * 32 + col];
        if (W == 2) qR += rC * PBs[(c + 2) * 32 + col];
      } else {
        qR = fir_right<float, FirLen<float>::K>(Fs, bun, col, p0 + lenx - 1, t.n, t.r);
      }
      tile_chunk_e<C>(fv, p0, lenx, z0, t, dl + s * 64 + 2 * col, rpow, sL, qR, e[s]);
    }
  }
  if (!mine) return;
  const float dt = a.dt, ta = a.acoef, s3h = t.s3h;
  float* const* tt = a.tmp;
#pragma unroll
  for (int j = 0; j <= C; ++j) {
    if (j >= lenx) break;
    const int pos = p0 + j;
    const int64_t gi = obase + (int64_t)pos * t.px + col;
    const float g0 = mulc(e[0][j], s3h, t.s3h_lo), g1 = mulc(e[1][j], s3h, t.s3h_lo),
                g2 = mulc(e[2][j], s3h, t.s3h_lo);
    if (PASS == ET_BY) {
      const float t1 = tt[1][gi];
      const float y0 = eff(a.pml, a.pB, a.memB[0], gi, pos, g0, dt, a.dt_lo);
      const float y1 = eff(a.pml, a.pB, a.memB[1], gi, pos, g1, dt, a.dt_lo);
      const float y2 = eff(a.pml, a.pB, a.memB[2], gi, pos, g2, dt, a.dt_lo);
      tt[1][gi] = t1 + y0;
      tt[3][gi] = y1;
      tt[4][gi] = y2;
    } else if (PASS == ET_BZ) {
      // every global operand of the point first, then the arithmetic, then the stores
      const int fs[6] = {LOSS_FIELD_S11, LOSS_FIELD_S22, LOSS_FIELD_S12, LOSS_FIELD_S13, LOSS_FIELD_S23,
                         LOSS_FIELD_S33};
      float u[6], cu[6];
#pragma unroll
      for (int f = 0; f < 6; ++f) {
        u[f] = a.fld[fs[f]][gi];
        cu[f] = KAHAN ? a.cmp[fs[f]][gi] : 0.0f;
      }
      const float xa = tt[0][gi], xd = tt[3][gi], tc = tt[2][gi], tb = tt[1][gi], te = tt[4][gi];
      const float lam = a.lam ? a.lam[gi] : a.lam0;
      const float mu = a.mu ? a.mu[gi] : a.mu0;
      const float x13 = eff(a.pml, a.pB, a.memB[0], gi, pos, g0, dt, a.dt_lo);  // v1 along z
      const float x23 = eff(a.pml, a.pB, a.memB[1], gi, pos, g1, dt, a.dt_lo);  // v2 along z
      const float x33 = eff(a.pml, a.pB, a.memB[2], gi, pos, g2, dt, a.dt_lo);  // v3 along z
      auto mlam = [&](float x) { return a.lam ? lam * x : mulc(x, a.lam0, a.lam0_lo); };
      auto mmu = [&](float x) { return a.mu ? mu * x : mulc(x, a.mu0, a.mu0_lo); };
      const float ltr = mlam(xa + xd + x33);
      float s11 = ltr + 2.0f * mmu(xa), s22 = ltr + 2.0f * mmu(xd), s33 = ltr + 2.0f * mmu(x33);
      float s13 = mmu(tc + x13);
      if (a.srcp.on) {
        const int dz = pos - a.srcp.zs + 12, dy = outer - a.srcp.ys + 12, dx = x0 + col - a.srcp.xs + 12;
        if ((unsigned)dz < 25u && (unsigned)dy < 25u && (unsigned)dx < 25u) {
          const float sv = (float)(a.srcp.amp * a.srcp.g[dz] * a.srcp.g[dy] * a.srcp.g[dx]);
          if (a.src_explosive) s11 += sv, s22 += sv, s33 += sv;
          if (a.src_shear) s13 += sv;
        }
      }
      const float d[6] = {s11, s22, mmu(tb), s13, mmu(te + x23), s33};
#pragma unroll
      for (int f = 0; f < 6; ++f) upd_r<float, KAHAN>(u[f], cu[f], d[f]);
#pragma unroll
      for (int f = 0; f < 6; ++f) {
        a.fld[fs[f]][gi] = u[f];
        if (KAHAN) a.cmp[fs[f]][gi] = cu[f];
      }
    } else if (PASS == ET_AZ) {
      tt[5][gi] = effA(a, 0, gi, pos, g0, ta);
      tt[6][gi] = effA(a, 1, gi, pos, g1, ta);
      tt[7][gi] = effA(a, 2, gi, pos, g2, ta);
    } else {  // ET_AY
      const float b = a.b ? a.b[gi] : a.b0;
      float force = 0.0f;  // body force (FORCE_X/Y/Z sources), already multiplied by the sub-step length
      if (a.srcp.on) {
        const int dz = outer - a.srcp.zs + 12, dy = pos - a.srcp.ys + 12, dx = x0 + col - a.srcp.xs + 12;
        if ((unsigned)dz < 25u && (unsigned)dy < 25u && (unsigned)dx < 25u)
          force = (float)(a.srcp.amp * a.srcp.g[dz] * a.srcp.g[dy] * a.srcp.g[dx]);
      }
      const float f0 = (a.force_mask & 1) ? force : 0.0f, f1 = (a.force_mask & 2) ? force : 0.0f,
                  f2 = (a.force_mask & 4) ? force : 0.0f;
      float u[3], cu[3];
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        u[f] = a.fld[LOSS_FIELD_V1 + f][gi];
        cu[f] = KAHAN ? a.cmp[LOSS_FIELD_V1 + f][gi] : 0.0f;
      }
      const float t5 = tt[5][gi], t6 = tt[6][gi], t7 = tt[7][gi];
      auto mb = [&](float x) { return a.b ? b * x : mulc(x, a.b0, a.b0_lo); };
      const float d0 = mb(t5 + effA(a, 0, gi, pos, g0, ta) + f0);
      const float d1 = mb(t6 + effA(a, 1, gi, pos, g1, ta) + f1);
      const float d2 = mb(t7 + effA(a, 2, gi, pos, g2, ta) + f2);
      upd_r<float, KAHAN>(u[0], cu[0], d0);
      upd_r<float, KAHAN>(u[1], cu[1], d1);
      upd_r<float, KAHAN>(u[2], cu[2], d2);
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        a.fld[LOSS_FIELD_V1 + f][gi] = u[f];
        if (KAHAN) a.cmp[LOSS_FIELD_V1 + f][gi] = cu[f];
      }
    }
  }
}

size_t elt_smem(const ElTile& g, int logc) {
  const int rows = g.t.M + 2 * g.t.H + 1;
  const int nch = (g.t.M + (1 << logc) - 1) >> logc;
  return (size_t)3 * rows * 32 * 4 + (size_t)6 * nch * 32 * 4;
}

template <int PASS, bool KAHAN>
static cudaError_t launch_elt_pass(const ElArgs<float>& a, const ElTile& g, int logc, cudaStream_t st) {
  ElArgs<float> aa = a;
  ElTile gg = g;
  void* argv[] = {&aa, &gg};
  const int threads = 32 * ((g.t.M + (1 << logc) - 1) >> logc);
  const int grid = g.t.p * g.ncg * g.nouter;
  const size_t smem = elt_smem(g, logc);
  auto kern = logc == 3 ? k_elt<PASS, KAHAN, 3> : k_elt<PASS, KAHAN, 4>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaLaunchKernel((const void*)kern, dim3(grid), dim3(threads), argv, smem, st);
}

template <bool KAHAN>
cudaError_t launch_elt(const ElArgs<float>& a, const ElTile& g, int pass, int logc, cudaStream_t st) {
  switch (pass) {
    case ET_BY: return launch_elt_pass<ET_BY, KAHAN>(a, g, logc, st);
    case ET_BZ: return launch_elt_pass<ET_BZ, KAHAN>(a, g, logc, st);
    case ET_AZ: return launch_elt_pass<ET_AZ, KAHAN>(a, g, logc, st);
    default: return launch_elt_pass<ET_AY, KAHAN>(a, g, logc, st);
  }
}
template cudaError_t launch_elt<false>(const ElArgs<float>&, const ElTile&, int, int, cudaStream_t);
template cudaError_t launch_elt<true>(const ElArgs<float>&, const ElTile&, int, int, cudaStream_t);

// ---------------------------------------------------------------------------------------------------------------
template <class K>
static cudaError_t launch_el_k(K kern, int grid, int threads, size_t smem, cudaStream_t st, void* args) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* argv[] = {args};
  return cudaLaunchKernel((const void*)kern, dim3(grid), dim3(threads), argv, smem, st);
}

template <typename T, int PASS, bool KAHAN>
static cudaError_t launch_el_pass(const ElArgs<T>& a, int logc, int threads, cudaStream_t st) {
  constexpr bool SF = (PASS == EL_BY || PASS == EL_BZ || PASS == EL_AY);
  const size_t smem = smem_bytes(a.g, 6, 0, sizeof(T));
  ElArgs<T> args = a;
  if (logc == 3 && sizeof(T) == 4) return launch_el_k(k_el<T, 3, SF, PASS, KAHAN>, a.g.nbundles, threads, smem, st, &args);
  return launch_el_k(k_el<T, 4, SF, PASS, KAHAN>, a.g.nbundles, threads, smem, st, &args);
}

template <typename T, bool KAHAN>
cudaError_t launch_el(const ElArgs<T>& a, int pass, int logc, int threads, cudaStream_t st) {
  switch (pass) {
    case EL_BX: return launch_el_pass<T, EL_BX, KAHAN>(a, logc, threads, st);
    case EL_BY: return launch_el_pass<T, EL_BY, KAHAN>(a, logc, threads, st);
    case EL_BZ: return launch_el_pass<T, EL_BZ, KAHAN>(a, logc, threads, st);
    case EL_AX: return launch_el_pass<T, EL_AX, KAHAN>(a, logc, threads, st);
    default: return launch_el_pass<T, EL_AY, KAHAN>(a, logc, threads, st);
  }
}

template cudaError_t launch_el<float, false>(const ElArgs<float>&, int, int, int, cudaStream_t);
template cudaError_t launch_el<float, true>(const ElArgs<float>&, int, int, int, cudaStream_t);
template cudaError_t launch_el<double, false>(const ElArgs<double>&, int, int, int, cudaStream_t);

}  // namespace lossk
