// sm_103a kernels of the 2-D acoustic LOSS step and of the stand-alone derivative.
//
// Time stepping (paper Sec. 3.3, Strang "half A, full B, half A", with the exponential ADE-PML sub-flows in
// the absorbing layers).  Consecutive half steps of A
// share the same stress, so n steps are one half A, n - 1 alternations (full B, full A), a full B and a half
// A.  The library keeps the velocities half a step ahead between calls (staggered state), so one step is:
//   X kernel (lines along x):  sigma += -dt kappa (d_x v1 + d_z v3) + source           [sub-step B]
//                              v1    += -dt b d_x sigma                                   [A, x part]
//   Z kernel (lines along z):  v3    += -dt b d_z sigma                                   [A, z part]
//                              tmp    = d_z v3                       (feeds the next step's B)
// Inside a PML layer the increments -tau g are replaced by the exact exponential flow of the memory variables
// (PmlAxis::step): Phi_x, Phi_z advance in the B part of the X kernel, Psi_x in its A part, Psi_z in the Z
// kernel, each exactly once per sub-step.
// Each kernel holds whole grid lines (all patches) on chip, so the PMBC halo of every junction is read from
// shared memory and each field is read from and written to HBM once per kernel.
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

// Shared-memory carve-up: nbuf line buffers, two summary arrays, phi, line bases.
template <typename T>
struct Carve {
  T* buf[3];
  T* sA;
  T* sB;
  double* phi;
  int64_t* lb;
  __device__ Carve(unsigned char* sm, const LineGeom& g, int nbuf) {
    T* p = reinterpret_cast<T*>(sm);
    for (int i = 0; i < 3; ++i) {
      buf[i] = p;
      if (i < nbuf) p += g.buf;
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

// Load whole lines of a global field into a shared buffer.
template <typename T, bool SFLAV, class BUN>
__device__ __forceinline__ void load_lines(const T* __restrict__ src, T* dst, const BUN& bun, const LineGeom& g,
                                           const int64_t* lb, int nvalid) {
  const int np = g.n + 1;
  if (SFLAV) {
    const int tot = np * g.L;
    for (int i = threadIdx.x; i < tot; i += blockDim.x) {
      const int pos = i / g.L;
      const int l = i - pos * g.L;
      if (l < nvalid) dst[bun.at(l, pos)] = src[lb[l] + (int64_t)pos * g.pstride];
    }
  } else {
    const int tot = np * nvalid;
    for (int i = threadIdx.x; i < tot; i += blockDim.x) {
      const int l = i / np;
      const int pos = i - l * np;
      dst[bun.at(l, pos)] = src[lb[l] + pos];
    }
  }
}

// Iterate (line, pos, global offset) over the bundle in a coalesced order and call fn.
template <bool SFLAV, class FN>
__device__ __forceinline__ void for_points(const LineGeom& g, const int64_t* lb, int nvalid, FN fn) {
  const int np = g.n + 1;
  if (SFLAV) {
    const int tot = np * g.L;
    for (int i = threadIdx.x; i < tot; i += blockDim.x) {
      const int pos = i / g.L;
      const int l = i - pos * g.L;
      if (l < nvalid) fn(l, pos, lb[l] + (int64_t)pos * g.pstride);
    }
  } else {
    const int tot = np * nvalid;
    for (int i = threadIdx.x; i < tot; i += blockDim.x) {
      const int l = i / np;
      const int pos = i - l * np;
      fn(l, pos, lb[l] + pos);
    }
  }
}

// Scaled first derivative e at (line, pos): phi at junctions and ends, the solve elsewhere.
template <typename T, class BUN>
__device__ __forceinline__ T e_at(const T* O, const double* phi, const BUN& bun, int p1, int M, int l, int pos) {
  const int j = pos / M;
  return (pos - j * M == 0) ? (T)phi[l * p1 + j] : O[bun.at(l, pos)];
}

}  // namespace

// ---------------------------------------------------------------------------------------------------------------
// Stand-alone derivative d1 (and d2) along one axis; optional phi output.
template <typename T, int LOGC, bool SFLAV>
__global__ void __launch_bounds__(1024) k_deriv(DerivArgs<T> a) {
  constexpr int C = 1 << LOGC;
  extern __shared__ __align__(16) unsigned char sm[];
  const LineGeom& g = a.g;
  const bool want_d2 = a.d2 != nullptr;
  Carve<T> cv(sm, g, want_d2 ? 3 : 2);
  T* F = cv.buf[0];
  T* O = cv.buf[1];
  T* O2 = cv.buf[2];
  const Bundle<LOGC, SFLAV> bun{g.pitch};
  const WorkMap<SFLAV> wm{g.L, g.p, g.NC};
  const int nvalid = bundle_bases<SFLAV>(g, blockIdx.x, cv.lb);
  __syncthreads();
  load_lines<T, SFLAV>(a.f, F, bun, g, cv.lb, nvalid);
  __syncthreads();
  pmbc_phi<T, 8>(F, bun, g.L, nvalid, g.n, g.p, g.M, g.n_nb, a.tb.W, cv.phi);
  __syncthreads();
  if (a.phi_out) {
    const int p1 = g.p + 1;
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
  solve_bundle<T, C, SFLAV>(F, O, cv.sA, cv.sB, bun, wm, nvalid, g.M, a.tb.t32, a.tb.t64, a.minf, RhsD1{},
                            BndPhi<T>{cv.phi, g.p + 1});
  const int p1 = g.p + 1;
  for_points<SFLAV>(g, cv.lb, nvalid, [&](int l, int pos, int64_t gi) {
    a.d1[gi] = a.s1 * e_at(O, cv.phi, bun, p1, g.M, l, pos);
  });
  if (!want_d2) return;
  solve_bundle<T, C, SFLAV>(F, O2, cv.sA, cv.sB, bun, wm, nvalid, g.M, a.tb.t32, a.tb.t64, a.minf, RhsD2{},
                            BndD2<T, Bundle<LOGC, SFLAV>>{F, O, cv.phi, p1, g.M, bun});
  // Output: interior slots from the solve; at a junction the average of the two patches' end values
  // (d2 h^2/6)_avg = (f_{j-1} - 2 f_j + f_{j+1} + e_{j-1} - e_{j+1}) / 2; at the two line ends the single value.
  for_points<SFLAV>(g, cv.lb, nvalid, [&](int l, int pos, int64_t gi) {
    const int j = pos / g.M;
    T s;
    if (pos - j * g.M != 0) {
      s = O2[bun.at(l, pos)];
    } else {
      const T ej = (T)cv.phi[l * p1 + j];
      if (pos == 0) {
        s = (F[bun.at(l, 1)] - F[bun.at(l, 0)]) - T(2) * ej - e_at(O, cv.phi, bun, p1, g.M, l, 1);
      } else if (pos == g.n) {
        s = (F[bun.at(l, pos - 1)] - F[bun.at(l, pos)]) + T(2) * ej + e_at(O, cv.phi, bun, p1, g.M, l, pos - 1);
      } else {
        const T fm = F[bun.at(l, pos - 1)], f0 = F[bun.at(l, pos)], fp = F[bun.at(l, pos + 1)];
        s = T(0.5) * (((fm - f0) + (fp - f0)) + (e_at(O, cv.phi, bun, p1, g.M, l, pos - 1) -
                                                 e_at(O, cv.phi, bun, p1, g.M, l, pos + 1)));
      }
    }
    a.d2[gi] = a.s2 * s;
  });
}

// ---------------------------------------------------------------------------------------------------------------
// X kernel of the 2-D acoustic step: sub-step B on whole x lines, then the x part of sub-step A.
template <typename T, int LOGC, bool KAHAN>
__global__ void __launch_bounds__(1024) k_ac_x(AcXArgs<T> a) {
  constexpr int C = 1 << LOGC;
  extern __shared__ __align__(16) unsigned char sm[];
  const LineGeom& g = a.g;
  Carve<T> cv(sm, g, 3);
  T* V = cv.buf[0];  // v1 (old)
  T* D = cv.buf[1];  // sigma after B
  T* O = cv.buf[2];  // solve output
  const Bundle<LOGC, false> bun{g.pitch};
  const WorkMap<false> wm{g.L, g.p, g.NC};
  const int nvalid = bundle_bases<false>(g, blockIdx.x, cv.lb);
  const int p1 = g.p + 1;
  __syncthreads();
  load_lines<T, false>(a.v1, V, bun, g, cv.lb, nvalid);
  if (!a.do_B) load_lines<T, false>(a.sigma, D, bun, g, cv.lb, nvalid);
  __syncthreads();
  if (a.do_B) {
    pmbc_phi<T, 8>(V, bun, g.L, nvalid, g.n, g.p, g.M, g.n_nb, a.tb.W, cv.phi);
    __syncthreads();
    solve_bundle<T, C, false>(V, O, cv.sA, cv.sB, bun, wm, nvalid, g.M, a.tb.t32, a.tb.t64, a.minf, RhsD1{},
                              BndPhi<T>{cv.phi, p1});
    const int64_t r0 = (int64_t)blockIdx.x * g.L;
    for_points<false>(g, cv.lb, nvalid, [&](int l, int pos, int64_t gi) {
      const int z = (int)((r0 + l) / g.ny1);
      const T gx = a.s3h * e_at(O, cv.phi, bun, p1, g.M, l, pos);  // d_x v1
      const T gz = a.tmp[gi];                                        // d_z v3
      T inc;
      if (a.pml && (a.xB.in(pos) || a.zB.in(z))) {
        inc = a.xB.in(pos) ? a.xB.step(a.phix, gi, pos, gx) : -a.dt * gx;
        inc += a.zB.in(z) ? a.zB.step(a.phiz, gi, z, gz) : -a.dt * gz;
      } else {
        inc = -a.dt * (gx + gz);
      }
      T delta = a.kappa[gi] * inc;
      if (a.src.on) {
        const int dz = z - a.src.zs + 12, dx = pos - a.src.xs + 12;
        if ((unsigned)dz < 25u && (unsigned)dx < 25u) delta += (T)(a.src.amp * a.src.g[dz] * a.src.g[dx]);
      }
      T s = a.sigma[gi];
      if constexpr (KAHAN) {
        float c = a.csig[gi];
        kahan_add(s, c, delta);
        a.csig[gi] = c;
      } else {
        s += delta;
      }
      a.sigma[gi] = s;
      D[bun.at(l, pos)] = s;
    });
    __syncthreads();
  }
  pmbc_phi<T, 8>(D, bun, g.L, nvalid, g.n, g.p, g.M, g.n_nb, a.tb.W, cv.phi);
  __syncthreads();
  solve_bundle<T, C, false>(D, O, cv.sA, cv.sB, bun, wm, nvalid, g.M, a.tb.t32, a.tb.t64, a.minf, RhsD1{},
                            BndPhi<T>{cv.phi, p1});
  for_points<false>(g, cv.lb, nvalid, [&](int l, int pos, int64_t gi) {
    const T gx = a.s3h * e_at(O, cv.phi, bun, p1, g.M, l, pos);  // d_x sigma
    const T inc = (a.pml && a.xA.in(pos)) ? a.xA.step(a.psix, gi, pos, gx) : -a.acoef * gx;
    const T delta = a.b[gi] * inc;
    T v = V[bun.at(l, pos)];
    if constexpr (KAHAN) {
      float c = a.cv1[gi];
      kahan_add(v, c, delta);
      a.cv1[gi] = c;
    } else {
      v += delta;
    }
    a.v1[gi] = v;
  });
}

// ---------------------------------------------------------------------------------------------------------------
// Z kernel of the 2-D acoustic step: z part of sub-step A on whole z lines, then tmp = d_z v3.
template <typename T, int LOGC, bool KAHAN>
__global__ void __launch_bounds__(1024) k_ac_z(AcZArgs<T> a) {
  constexpr int C = 1 << LOGC;
  extern __shared__ __align__(16) unsigned char sm[];
  const LineGeom& g = a.g;
  Carve<T> cv(sm, g, 2);
  T* S = cv.buf[0];  // sigma, then v3 (new)
  T* O = cv.buf[1];
  const Bundle<LOGC, true> bun{g.pitch};
  const WorkMap<true> wm{g.L, g.p, g.NC};
  const int nvalid = bundle_bases<true>(g, blockIdx.x, cv.lb);
  const int p1 = g.p + 1;
  __syncthreads();
  load_lines<T, true>(a.sigma, S, bun, g, cv.lb, nvalid);
  __syncthreads();
  pmbc_phi<T, 8>(S, bun, g.L, nvalid, g.n, g.p, g.M, g.n_nb, a.tb.W, cv.phi);
  __syncthreads();
  solve_bundle<T, C, true>(S, O, cv.sA, cv.sB, bun, wm, nvalid, g.M, a.tb.t32, a.tb.t64, a.minf, RhsD1{},
                           BndPhi<T>{cv.phi, p1});
  for_points<true>(g, cv.lb, nvalid, [&](int l, int pos, int64_t gi) {
    const T gz = a.s3h * e_at(O, cv.phi, bun, p1, g.M, l, pos);  // d_z sigma
    const T inc = (a.pml && a.zA.in(pos)) ? a.zA.step(a.psiz, gi, pos, gz) : -a.acoef * gz;
    const T delta = a.b[gi] * inc;
    T v = a.v3[gi];
    if constexpr (KAHAN) {
      float c = a.cv3[gi];
      kahan_add(v, c, delta);
      a.cv3[gi] = c;
    } else {
      v += delta;
    }
    a.v3[gi] = v;
    S[bun.at(l, pos)] = v;
  });
  __syncthreads();
  if (!a.do_tmp) return;
  pmbc_phi<T, 8>(S, bun, g.L, nvalid, g.n, g.p, g.M, g.n_nb, a.tb.W, cv.phi);
  __syncthreads();
  solve_bundle<T, C, true>(S, O, cv.sA, cv.sB, bun, wm, nvalid, g.M, a.tb.t32, a.tb.t64, a.minf, RhsD1{},
                           BndPhi<T>{cv.phi, p1});
  for_points<true>(g, cv.lb, nvalid, [&](int l, int pos, int64_t gi) {
    a.tmp[gi] = a.s3h * e_at(O, cv.phi, bun, p1, g.M, l, pos);
  });
}

// ---------------------------------------------------------------------------------------------------------------
// Receiver gather: mode 0 out[r] = f[idx[r]]; mode 1 out[r] = (out[r] + f[idx[r]]) / 2 (integer-time velocity
// from the two staggered half-step values).
template <typename T>
__global__ void k_gather(const T* __restrict__ f, const int64_t* __restrict__ idx, int64_t n, T* __restrict__ out,
                         int mode) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const T v = f[idx[r]];
    out[r] = mode ? T(0.5) * (out[r] + v) : v;
  }
}

// ---------------------------------------------------------------------------------------------------------------
// Host launchers.
size_t smem_bytes(const LineGeom& g, int nbuf, size_t esize) {
  const size_t nw = (size_t)g.L * g.p * g.NC;
  size_t b = (size_t)nbuf * g.buf * esize;
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
  const size_t smem = smem_bytes(a.g, a.d2 ? 3 : 2, sizeof(T));
  DerivArgs<T> args = a;
  if (sflav) {
    if (logc == 4) return launch(k_deriv<T, 4, true>, a.g.nbundles, threads, smem, st, &args);
    return launch(k_deriv<T, 5, true>, a.g.nbundles, threads, smem, st, &args);
  }
  if (logc == 4) return launch(k_deriv<T, 4, false>, a.g.nbundles, threads, smem, st, &args);
  return launch(k_deriv<T, 5, false>, a.g.nbundles, threads, smem, st, &args);
}

template <typename T, bool KAHAN>
cudaError_t launch_ac_x(const AcXArgs<T>& a, int logc, int threads, cudaStream_t st) {
  const size_t smem = smem_bytes(a.g, 3, sizeof(T));
  AcXArgs<T> args = a;
  if (logc == 4) return launch(k_ac_x<T, 4, KAHAN>, a.g.nbundles, threads, smem, st, &args);
  return launch(k_ac_x<T, 5, KAHAN>, a.g.nbundles, threads, smem, st, &args);
}

template <typename T, bool KAHAN>
cudaError_t launch_ac_z(const AcZArgs<T>& a, int logc, int threads, cudaStream_t st) {
  const size_t smem = smem_bytes(a.g, 2, sizeof(T));
  AcZArgs<T> args = a;
  if (logc == 4) return launch(k_ac_z<T, 4, KAHAN>, a.g.nbundles, threads, smem, st, &args);
  return launch(k_ac_z<T, 5, KAHAN>, a.g.nbundles, threads, smem, st, &args);
}

template <typename T>
cudaError_t launch_gather(const T* f, const int64_t* idx, int64_t n, T* out, int mode, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int threads = 256;
  const int grid = (int)((n + threads - 1) / threads < 4096 ? (n + threads - 1) / threads : 4096);
  k_gather<T><<<grid, threads, 0, st>>>(f, idx, n, out, mode);
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
template cudaError_t launch_gather<float>(const float*, const int64_t*, int64_t, float*, int, cudaStream_t);
template cudaError_t launch_gather<double>(const double*, const int64_t*, int64_t, double*, int, cudaStream_t);

}  // namespace lossk
