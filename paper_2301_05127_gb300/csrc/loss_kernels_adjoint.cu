// sm_103a kernels of the discrete adjoint of the LOSS time step (gradient of a seismogram misfit).  The paper
// has no adjoint; these kernels transpose the step the forward kernels take.
//
// Transposed LOSS derivative along one line (D = (3/h) P, P f = e):  forward, every patch solves
// e_{i-1} + 4 e_i + e_{i+1} = f_{i+1} - f_{i-1} for its interior unknowns with the junction values
// e_j = phi_j = sum_m W[j][m] f_{jM+m} (PMBC, Sec. 3.2).  With ebar the adjoint of e (all points):
//   w = T^{-1} ebar on every patch interior (T = tridiag(1, 4, 1) is symmetric; w = 0 at junctions),
//   phibar_j = ebar_j - w_{j-1} - w_{j+1},
//   (P^T ebar)_k = w_{k-1} - w_{k+1} + sum_j W[j][k - jM] phibar_j,
// so D^T needs the same tridiagonal solve as D (identity right-hand side, zero boundary values) and the PMBC
// weights applied as a scatter instead of a gather.  The junction sums are accumulated in FP64.
//
// One adjoint term per launch (k_adj, modes in AdjArgs): the forward derivative of the term is recomputed on
// chip (the gradient needs the forward increment), the term's adjoint input is formed pointwise, passed through
// the transposed PML sub-flow (m' = E m + P g, X = Q m + R g; transpose m_adj = E m'_adj + Q X_adj,
// g_adj = P m'_adj + R X_adj), and D^T of the result is added to the output adjoint field.
#include <cuda_runtime.h>

#include "../../include/loss.h"
#include "loss_block.cuh"
#include "loss_line.cuh"
#include "loss_types.h"

namespace lossk {

size_t smem_bytes(const LineGeom& g, int nbuf, int nstage, size_t esize);  // loss_kernels_acoustic.cu

template <typename T, int LOGC, bool SFLAV>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 512 : 1024) k_adj(AdjArgs<T> a) {
  constexpr int C = 1 << LOGC;
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ ChunkClasses<T, C> cc;
  const LineGeom& g = a.g;
  Carve<T> cv(sm, g, 4, 0);
  T* F = cv.buf[0];   // forward field
  T* O = cv.buf[1];   // e of the forward field
  T* Gb = cv.buf[2];  // adjoint of e
  T* Wb = cv.buf[3];  // w
  const Bundle<LOGC, SFLAV> bun{g.pitch};
  const WorkMap<SFLAV> wm{g.L, g.p, g.NC};
  const int logL = SFLAV ? log2_pow2(g.L) : 0;
  const int nvalid = bundle_bases<SFLAV>(g, blockIdx.x, cv.lb);
  const int p1 = g.p + 1;
  const int n1 = g.n + 1;
  chunk_classes_init<T, C>(&cc, g.M, g.NC, a.tb.t32, a.tb.t64, a.minf);
  __syncthreads();
  if (a.mode != 0) {
    stage_padded<T, SFLAV>(a.ffwd, F, bun, g, cv.lb, nvalid, logL);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    pmbc_phi<T, 16>(F, bun, g.L, nvalid, g.n, g.p, g.M, g.n_nb, a.tb.W, cv.phi);
    __syncthreads();
    solve_bundle<T, C, SFLAV>(F, O, cv.sA, &cc, bun, wm, nvalid, g.M, a.tb.t32, a.tb.t64, a.minf, RhsD1{},
                              BndPhi<T>{cv.phi, p1});
  }
  // adjoint of the derivative at every point of the bundle
  for_points<SFLAV>(g, cv.lb, nvalid, logL, [&](int l, int pos, int64_t gi) {
    const int k = bun.at(l, pos);
    if (a.mode == 0) {
      Gb[k] = a.in3[gi];
      return;
    }
    const T gf = a.s3h * O[k];  // forward derivative
    const bool lay = a.pml && a.pa.in(pos);
    T E = T(0), P = T(0), Q = T(0), R = -a.tau;
    T m = T(0);
    if (lay) {
      E = a.pa.tab[pos];
      P = -a.pa.tab[n1 + pos];
      const T ib = a.pa.tab[2 * n1 + pos];
      Q = (E - T(1)) * ib;
      R = P * ib - a.pa.tab[3 * n1 + pos];
      m = a.memf[gi];
    }
    const T Z = a.sgn * (Q * m + R * gf);
    // the accumulated gradients and the adjoint memory variable are loaded with the other operands, before any
    // store (the arrays may alias as far as the compiler knows)
    const double g1o = a.g1 ? a.g1[gi] : 0.0;
    const double g2o = a.g2 ? a.g2[gi] : 0.0;
    const T mbo = lay ? a.memb[gi] : T(0);
    T ssum = T(0);
    if (a.in[0]) ssum += a.in[0][gi];
    if (a.in[1]) ssum += a.in[1][gi];
    if (a.in[2]) ssum += a.in[2][gi];
    const T a3 = a.in3 ? a.in3[gi] : T(0);
    const T c1 = a.c1 ? a.c1[gi] : a.c1s;
    const T c2 = a.cw2 * (a.c2 ? a.c2[gi] : a.c2s);
    const T xb = a.sgn * (c1 * ssum + c2 * a3);  // adjoint of X
    // receiver term: the integer-time velocity adds the first half (tau / 2) of the sub-flow
    T Qh = T(0), Rh = T(0), xhb = T(0), Zh = T(0), rv = T(0);
    if (a.rv) {
      rv = a.rv[gi];
      Rh = T(-0.5) * a.tau;
      if (lay) {
        const T Eh = a.pa.tabh[pos];
        const T Ph = -a.pa.tabh[n1 + pos];
        const T ibh = a.pa.tabh[2 * n1 + pos];
        Qh = (Eh - T(1)) * ibh;
        Rh = Ph * ibh - a.pa.tabh[3 * n1 + pos];
      }
      Zh = a.sgn * (Qh * m + Rh * gf);
      xhb = a.sgn * (c2 * rv);
    }
    if (a.g1) a.g1[gi] = g1o + (double)Z * (double)ssum;
    if (a.g2) a.g2[gi] = g2o + ((double)Z * (double)(a.gw2 * a3) + (double)Zh * (double)rv);
    T gb;
    if (lay) {
      const T mb = mbo;
      a.memb[gi] = E * mb + Q * xb + Qh * xhb;
      gb = P * mb + R * xb + Rh * xhb;
    } else {
      gb = R * xb + Rh * xhb;
    }
    Gb[k] = gb;
  });
  __syncthreads();
  solve_bundle<T, C, SFLAV>(Gb, Wb, cv.sA, &cc, bun, wm, nvalid, g.M, a.tb.t32, a.tb.t64, a.minf, RhsId{},
                            BndZero<T>{});
  for (int i = threadIdx.x; i < nvalid * p1; i += blockDim.x) {
    const int l = i / p1;
    const int c = (i - l * p1) * g.M;
    double v = (double)Gb[bun.at(l, c)];
    if (c > 0) v -= (double)Wb[bun.at(l, c - 1)];
    if (c < g.n) v -= (double)Wb[bun.at(l, c + 1)];
    cv.phi[i] = v;
  }
  __syncthreads();
  const int wlen = 2 * g.n_nb + 1;
  for_points<SFLAV>(g, cv.lb, nvalid, logL, [&](int l, int pos, int64_t gi) {
    const int jlo = pos <= g.n_nb ? 0 : (pos - g.n_nb + g.M - 1) / g.M;
    const int jhi = min(g.p, (pos + g.n_nb) / g.M);
    double acc = 0.0;
    for (int j = jlo; j <= jhi; ++j) acc += __ldg(a.tb.W + (size_t)j * wlen + g.n_nb + (pos - j * g.M)) * cv.phi[l * p1 + j];
    const T wm1 = pos > 0 ? Wb[bun.at(l, pos - 1)] : T(0);
    const T wp1 = pos < g.n ? Wb[bun.at(l, pos + 1)] : T(0);
    a.out[gi] += (T)(a.s3hd * ((double)(wm1 - wp1) + acc));
  });
}

// Residual injection of one adjoint step (trace row `row`): job blockIdx.y.
template <typename T>
__global__ void k_inject(const InjectJob<T>* __restrict__ jobs, int64_t row, int64_t row_stride, int phase) {
  const InjectJob<T>& j = jobs[blockIdx.y];
  const double* rr = j.r + row * row_stride;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < j.cnt; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = j.idx[r];
    const T v = (T)rr[r];
    if (phase == 0) {
      if (j.rv) atomicAdd(j.rv + q, v);
      else atomicAdd(j.lam + q, v);
    } else if (j.rv) {
      atomicAdd(j.lam + q, v);
      j.rv[q] = T(0);
    }
  }
}

template <typename T>
cudaError_t launch_adj(const AdjArgs<T>& a, int logc, bool sflav, int threads, cudaStream_t st) {
  const size_t smem = smem_bytes(a.g, 4, 0, sizeof(T));
  AdjArgs<T> args = a;
  void* argv[] = {&args};
  const void* kern;
  if (sflav)
    kern = (logc == 3 && sizeof(T) == 4) ? (const void*)k_adj<T, 3, true> : (const void*)k_adj<T, 4, true>;
  else
    kern = (logc == 3 && sizeof(T) == 4) ? (const void*)k_adj<T, 3, false> : (const void*)k_adj<T, 4, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaLaunchKernel(kern, dim3(a.g.nbundles), dim3(threads), argv, smem, st);
}

template <typename T>
cudaError_t launch_inject(const InjectJob<T>* jobs, int njobs, int64_t max_cnt, int64_t row, int64_t row_stride,
                          int phase, cudaStream_t st) {
  if (njobs <= 0 || max_cnt <= 0) return cudaSuccess;
  const int threads = 256;
  const int64_t bx = (max_cnt + threads - 1) / threads;
  k_inject<T><<<dim3((unsigned)(bx < 1024 ? bx : 1024), (unsigned)njobs), threads, 0, st>>>(jobs, row, row_stride,
                                                                                            phase);
  return cudaGetLastError();
}

template cudaError_t launch_adj<float>(const AdjArgs<float>&, int, bool, int, cudaStream_t);
template cudaError_t launch_adj<double>(const AdjArgs<double>&, int, bool, int, cudaStream_t);
template cudaError_t launch_inject<float>(const InjectJob<float>*, int, int64_t, int64_t, int64_t, int, cudaStream_t);
template cudaError_t launch_inject<double>(const InjectJob<double>*, int, int64_t, int64_t, int64_t, int,
                                           cudaStream_t);

}  // namespace lossk
