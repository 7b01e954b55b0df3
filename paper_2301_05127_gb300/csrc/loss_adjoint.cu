// Host side of the discrete adjoint: loss_gradient (misfit and its gradient with respect to vp, vs, rho) and
// loss_derivative_adjoint (stand-alone D^T).  The paper has no adjoint; see loss_kernels_adjoint.cu.
//
// The forward run is the library's own staggered time step: with S_n = (sigma_n, v_{n+1/2}, Psi_{n+1/2}, Phi_n)
// the state between steps, step n is B(dt) (sigma_n -> sigma_{n+1} from v_{n+1/2}, Phi_n -> Phi_{n+1}) followed
// by A(dt) (v_{n+1/2} -> v_{n+3/2} from sigma_{n+1}, Psi_{n+1/2} -> Psi_{n+3/2}); trace row n holds
// sigma_{n+1} and v_{n+1} = v_{n+1/2} + (first half of the A flow), i.e. the integer-time values.  The adjoint
// step n maps the adjoint of S_{n+1} to that of S_n:
//   1. residual of trace row n: stress receivers into the stress adjoints, velocity receivers into rv;
//   2. every velocity-sub-step term (A) transposed: adjoint memory, D^T into the stress adjoints, gradient of b;
//   3. velocity receivers into the velocity adjoints (their direct part);
//   4. every stress-sub-step term (B) transposed: adjoint memory, D^T into the velocity adjoints, gradients of
//      lambda and mu (kappa).
// Forward values come from the states S_n and S_{n+1}, recomputed segment by segment from checkpoints taken
// every C steps (C = ceil(sqrt(n_steps)) by default): memory ~ (n/C + C) states instead of n.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "loss_host.h"

namespace lossk {

#define LOSS_TRY(expr)              \
  do {                              \
    loss_status_t st_ = (expr);     \
    if (st_ != LOSS_OK) return st_; \
  } while (0)

static loss_status_t err(loss_ctx* h, loss_status_t st, const std::string& msg) {
  h->err = msg;
  return st;
}

// Arrays of the staggered state between steps.  with_all: also the compensation terms and the carried
// derivative temporary (everything needed to continue stepping bit for bit).
static std::vector<void*> state_arrays(Shot& s, bool with_all) {
  std::vector<void*> v;
  for (int f = 0; f < LOSS_NUM_FIELDS; ++f)
    if (field_used(s, f)) v.push_back(s.field[f]);
  if (s.pml_on) {
    if (s.d.physics == LOSS_ELASTIC) {
      for (int i = 0; i < 18; ++i) v.push_back(s.pmem[i]);
    } else {
      for (int k = 0; k < 3; ++k) {
        if (s.dim == 2 && k == 1) continue;
        v.push_back(s.psi[k]);
        v.push_back(s.phi[k]);
      }
    }
  }
  if (with_all) {
    if (s.kahan)
      for (int f = 0; f < LOSS_NUM_FIELDS; ++f)
        if (field_used(s, f)) v.push_back(s.comp[f]);
    if (s.d.physics == LOSS_ACOUSTIC) v.push_back(s.tmp[0]);
  }
  return v;
}

// Position of an array of state_arrays(s, *) in the snapshot (fields first, then memory variables).
static int snap_field(const Shot& s, int f) {
  int k = 0;
  for (int g = 0; g < f; ++g)
    if (field_used(s, g)) ++k;
  return k;
}
static int snap_mem(const Shot& s, int slot) {  // elastic: pmem index; acoustic: 2*slot_index + (0 psi, 1 phi)
  int nf = 0;
  for (int g = 0; g < LOSS_NUM_FIELDS; ++g)
    if (field_used(s, g)) ++nf;
  return nf + slot;
}

static loss_status_t copy_arrays(loss_ctx* h, const std::vector<void*>& src, char* dst, size_t fb, bool to_store) {
  for (size_t i = 0; i < src.size(); ++i) {
    void* a = to_store ? (void*)(dst + i * fb) : src[i];
    const void* b = to_store ? src[i] : (const void*)(dst + i * fb);
    LOSS_TRY(cuda_check(h, cudaMemcpyAsync(a, b, fb, cudaMemcpyDeviceToDevice, h->stream), "state copy"));
  }
  return LOSS_OK;
}

static loss_status_t zero_state(loss_ctx* h, Shot& s) {
  const size_t fb = (size_t)s.total * s.esize;
  std::vector<void*> all = state_arrays(s, true);
  for (int i = 0; i < 8; ++i)
    if (s.tmp[i]) all.push_back(s.tmp[i]);
  for (int i = 0; i < 9; ++i)
    if (s.rdelta[i]) all.push_back(s.rdelta[i]);
  for (void* p : all)
    if (p) LOSS_TRY(cuda_check(h, cudaMemsetAsync(p, 0, fb, h->stream), "memset"));
  s.step = 0;
  s.staggered = false;
  s.rcv_steps = 0;
  return LOSS_OK;
}

template <typename T>
static PmlAxis<T> pml_tables(const Shot& s, int k, bool half) {
  return PmlAxis<T>{(const T*)s.pml_tab[k][0], s.pml_width, (int)s.n[k], half ? (const T*)s.pml_tab[k][1] : nullptr};
}

static int slot_of(int j) { return j == 1 ? 2 : (j == 2 ? 1 : 0); }  // paper direction x_j -> internal slot
static int sig_of(int i, int j) {
  if (i == j) return LOSS_FIELD_S11 + (i - 1);
  const int a = std::min(i, j), b = std::max(i, j);
  if (a == 1 && b == 2) return LOSS_FIELD_S12;
  if (a == 1 && b == 3) return LOSS_FIELD_S13;
  return LOSS_FIELD_S23;
}

// Built-in FP32 shape of the adjoint kernels (measured on the 193^3 gradient: 128 threads, chunks of 8, 4 % faster
// than the line kernels' defaults); a shape set with loss_set_tile / loss_set_launch takes precedence.
template <typename T>
static int adj_threads(const loss_ctx* h) {
  const int t = h->tile_threads[LOSS_KERNEL_ADJOINT];
  return (t <= 0 && sizeof(T) == 4 && h->lines_per_block[LOSS_KERNEL_ADJOINT] <= 0) ? 128 : t;
}
template <typename T>
static int adj_logc(const loss_ctx* h) {
  const int c = h->chunk_log2[LOSS_KERNEL_ADJOINT];
  return (c <= 0 && sizeof(T) == 4) ? 3 : c;
}

template <typename T>
static loss_status_t launch_term(loss_ctx* h, Shot& s, int slot, AdjArgs<T>& a) {
  LineGeom g;
  int logc, threads;
  LOSS_TRY(line_geom(h, s, slot, s.sz, s.sy, &g, &logc, &threads, 4, 0, h->lines_per_block[LOSS_KERNEL_ADJOINT],
                     adj_logc<T>(h), adj_threads<T>(h)));
  a.g = g;
  a.tb = Tables{s.W[slot], h->t32, h->t64};
  a.s3h = (T)(3.0 / s.h[slot]);
  a.s3hd = 3.0 / s.h[slot];
  a.minf = (T)(2.0 - std::sqrt(3.0));
  LaunchScope ls(h, LOSS_KERNEL_ADJOINT);
  return cuda_check(h, launch_adj<T>(a, logc, slot != 2, threads, h->stream), "adjoint kernel");
}

// Snapshot views: arrays of S_n (sn) and S_{n+1} (sn1), each of fb bytes, in state_arrays(s, false) order.
struct Snap {
  char* base;
  size_t fb;
  void* at(int i) const { return base + (size_t)i * fb; }
};

template <typename T>
static loss_status_t adjoint_step(loss_ctx* h, Shot& s, const Snap& sn, const Snap& sn1, int64_t row,
                                  const InjectJob<T>* jobs, int njobs, int64_t max_cnt) {
  const T dt = (T)s.d.dt;
  const bool el = s.d.physics == LOSS_ELASTIC;
  LOSS_TRY(cuda_check(h, launch_inject<T>(jobs, njobs, max_cnt, row, s.n_rcv, 0, h->stream), "inject"));
  // velocity sub-step terms
  const int ncomp = el ? 3 : 2;
  for (int ii = 0; ii < ncomp; ++ii) {
    const int i = el ? ii + 1 : (ii == 0 ? 1 : 3);  // velocity component
    const int vf = LOSS_FIELD_V1 + (i - 1);
    for (int j = 1; j <= 3; ++j) {
      if (!el && j != i) continue;  // acoustic: v_i changes with d_i sigma only
      if (!el && s.dim == 2 && j == 2) continue;
      const int slot = slot_of(j);
      AdjArgs<T> a{};
      a.mode = 1;
      a.sgn = el ? T(-1) : T(1);
      a.tau = dt;
      const int sf = el ? sig_of(i, j) : LOSS_FIELD_SIGMA;
      a.ffwd = (const T*)sn1.at(snap_field(s, sf));
      a.pml = s.pml_on ? 1 : 0;
      if (s.pml_on) {
        const int mi = el ? 9 + 3 * (i - 1) + (j - 1) : 2 * (slot == 0 ? 0 : 1);  // psi slot
        a.memf = (const T*)sn.at(snap_mem(s, mi));
        a.memb = (T*)s.lam_mem[mi];
        a.pa = pml_tables<T>(s, slot, true);
      }
      a.in3 = (const T*)s.lam[vf];
      a.rv = s.rv[i - 1] ? (const T*)s.rv[i - 1] : nullptr;
      a.c2 = s.b_const ? nullptr : (const T*)s.model[el ? 2 : 1];
      a.c2s = (T)s.b0;
      a.cw2 = T(1);
      a.g2 = s.grad[2];
      a.gw2 = T(1);
      a.out = (T*)s.lam[sf];
      LOSS_TRY(launch_term<T>(h, s, slot, a));
    }
  }
  LOSS_TRY(cuda_check(h, launch_inject<T>(jobs, njobs, max_cnt, row, s.n_rcv, 1, h->stream), "inject"));
  // stress sub-step terms
  for (int ii = 0; ii < ncomp; ++ii) {
    const int i = el ? ii + 1 : (ii == 0 ? 1 : 3);
    const int vf = LOSS_FIELD_V1 + (i - 1);
    for (int j = 1; j <= 3; ++j) {
      if (!el && j != i) continue;
      const int slot = slot_of(j);
      AdjArgs<T> a{};
      a.mode = 2;
      a.sgn = el ? T(-1) : T(1);
      a.tau = dt;
      a.ffwd = (const T*)sn.at(snap_field(s, vf));
      a.pml = s.pml_on ? 1 : 0;
      if (s.pml_on) {
        const int mi = el ? 3 * (i - 1) + (j - 1) : 2 * (slot == 0 ? 0 : 1) + 1;  // phi slot
        a.memf = (const T*)sn.at(snap_mem(s, mi));
        a.memb = (T*)s.lam_mem[mi];
        a.pa = pml_tables<T>(s, slot, false);
      }
      if (el) {
        if (i == j) {
          for (int k = 0; k < 3; ++k) a.in[k] = (const T*)s.lam[LOSS_FIELD_S11 + k];
          a.c1 = s.lam_const ? nullptr : (const T*)s.model[0];
          a.c1s = (T)s.lam0;
          a.g1 = s.grad[0];
          a.cw2 = T(2);
          a.gw2 = T(2);
        } else {
          a.c1s = T(0);
          a.cw2 = T(1);
          a.gw2 = T(1);
        }
        a.in3 = (const T*)s.lam[sig_of(i, j)];
        a.c2 = s.mu_const ? nullptr : (const T*)s.model[1];
        a.c2s = (T)s.mu0;
        a.g2 = s.grad[1];
      } else {
        a.in3 = (const T*)s.lam[LOSS_FIELD_SIGMA];
        a.c2 = (const T*)s.model[0];  // kappa (always an array)
        a.cw2 = T(1);
        a.gw2 = T(1);
        a.g2 = s.grad[0];
      }
      a.out = (T*)s.lam[vf];
      LOSS_TRY(launch_term<T>(h, s, slot, a));
    }
  }
  return LOSS_OK;
}

template <typename T>
static loss_status_t gradient_t(loss_ctx* h, Shot& s, const double* d_obs_host, int64_t C, int64_t n_steps,
                                double* misfit, std::vector<double> grads_out[3]) {
  const size_t fb = (size_t)s.total * s.esize;
  const size_t gb = (size_t)s.total * sizeof(double);
  const bool el = s.d.physics == LOSS_ELASTIC;
  // adjoint workspace
  for (int f = 0; f < LOSS_NUM_FIELDS; ++f)
    if (field_used(s, f) && !s.lam[f]) LOSS_TRY(dev_alloc(h, fb, &s.lam[f]));
  const int nmem = s.pml_on ? (el ? 18 : 4) : 0;
  for (int i = 0; i < nmem; ++i)
    if (!s.lam_mem[i]) LOSS_TRY(dev_alloc(h, fb, &s.lam_mem[i]));
  for (int i = 0; i < 3; ++i) {
    const bool want = !s.rcv[LOSS_FIELD_V1 + i].empty();
    if (want && !s.rv[i]) LOSS_TRY(dev_alloc(h, fb, &s.rv[i]));
    if (!want && s.rv[i]) {
      dev_free(h, s.rv[i]);
      s.rv[i] = nullptr;
    }
  }
  for (int i = 0; i < 3; ++i)
    if (!s.grad[i]) LOSS_TRY(dev_alloc(h, gb, (void**)&s.grad[i]));
  auto zero_adjoint = [&]() -> loss_status_t {
    for (int f = 0; f < LOSS_NUM_FIELDS; ++f)
      if (s.lam[f]) LOSS_TRY(cuda_check(h, cudaMemsetAsync(s.lam[f], 0, fb, h->stream), "memset"));
    for (int i = 0; i < nmem; ++i) LOSS_TRY(cuda_check(h, cudaMemsetAsync(s.lam_mem[i], 0, fb, h->stream), "memset"));
    for (int i = 0; i < 3; ++i) {
      if (s.rv[i]) LOSS_TRY(cuda_check(h, cudaMemsetAsync(s.rv[i], 0, fb, h->stream), "memset"));
      LOSS_TRY(cuda_check(h, cudaMemsetAsync(s.grad[i], 0, gb, h->stream), "memset"));
    }
    return LOSS_OK;
  };
  LOSS_TRY(zero_adjoint());

  // forward run from rest with checkpoints every C steps and one at the end
  LOSS_TRY(zero_state(h, s));
  LOSS_TRY(ensure_trace_capacity(h, s, n_steps));
  const std::vector<void*> full = state_arrays(s, true);
  const std::vector<void*> part = state_arrays(s, false);
  const int64_t K = (n_steps + C - 1) / C;
  void* ck = nullptr;
  void* sg = nullptr;
  struct Free {
    loss_ctx* h;
    void** a;
    void** b;
    ~Free() {
      dev_free(h, *a);
      dev_free(h, *b);
    }
  } fr{h, &ck, &sg};
  const size_t ck_bytes = full.size() * fb;
  LOSS_TRY(dev_alloc(h, (size_t)(K + 1) * ck_bytes, &ck));
  LOSS_TRY(dev_alloc(h, (size_t)(C + 1) * part.size() * fb, &sg));
  for (int64_t n = 0; n < n_steps; ++n) {
    if (n % C == 0) {
      LOSS_TRY(stagger_shot(h, s));
      LOSS_TRY(copy_arrays(h, full, (char*)ck + (size_t)(n / C) * ck_bytes, fb, true));
    }
    LOSS_TRY(step_shot(h, s));
  }
  LOSS_TRY(copy_arrays(h, full, (char*)ck + (size_t)K * ck_bytes, fb, true));
  // residual and misfit
  const int64_t nr = s.n_rcv;
  std::vector<char> tr((size_t)n_steps * nr * s.esize);
  LOSS_TRY(cuda_check(h, cudaMemcpyAsync(tr.data(), s.traces, tr.size(), cudaMemcpyDeviceToHost, h->stream),
                      "copy traces"));
  LOSS_TRY(cuda_check(h, cudaStreamSynchronize(h->stream), "sync"));
  std::vector<double> res((size_t)n_steps * nr);
  double J = 0.0;
  for (size_t i = 0; i < res.size(); ++i) {
    const double v = s.esize == 8 ? ((const double*)tr.data())[i] : (double)((const float*)tr.data())[i];
    res[i] = v - d_obs_host[i];
    J += 0.5 * res[i] * res[i];
  }
  *misfit = J;
  double* dres = nullptr;
  void* djobs = nullptr;
  struct Free2 {
    loss_ctx* h;
    double** a;
    void** b;
    ~Free2() {
      dev_free(h, *a);
      dev_free(h, *b);
    }
  } fr2{h, &dres, &djobs};
  LOSS_TRY(dev_alloc(h, res.size() * sizeof(double), (void**)&dres));
  LOSS_TRY(cuda_check(h, cudaMemcpyAsync(dres, res.data(), res.size() * sizeof(double), cudaMemcpyHostToDevice,
                                         h->stream), "copy residual"));
  std::vector<InjectJob<T>> jobs;
  int64_t max_cnt = 0;
  for (int f = 0; f < LOSS_NUM_FIELDS; ++f) {
    const int64_t off = s.rcv_offsets[f], cnt = s.rcv_offsets[f + 1] - off;
    if (cnt == 0) continue;
    InjectJob<T> j{};
    j.lam = (T*)s.lam[f];
    j.rv = is_velocity(f) ? (T*)s.rv[f - LOSS_FIELD_V1] : nullptr;
    j.idx = s.rcv_idx + off;
    j.r = dres + off;
    j.cnt = cnt;
    jobs.push_back(j);
    max_cnt = std::max(max_cnt, cnt);
  }
  LOSS_TRY(dev_alloc(h, std::max<size_t>(jobs.size(), 1) * sizeof(InjectJob<T>), &djobs));
  if (!jobs.empty())
    LOSS_TRY(cuda_check(h, cudaMemcpyAsync(djobs, jobs.data(), jobs.size() * sizeof(InjectJob<T>),
                                           cudaMemcpyHostToDevice, h->stream), "copy jobs"));
  LOSS_TRY(cuda_check(h, cudaStreamSynchronize(h->stream), "sync"));

  // backward, segment by segment
  const int64_t nrcv_saved = s.n_rcv;
  const int64_t rsteps_saved = s.rcv_steps;
  for (int64_t k = K - 1; k >= 0; --k) {
    const int64_t c0 = k * C, c1 = std::min(n_steps, c0 + C);
    LOSS_TRY(copy_arrays(h, full, (char*)ck + (size_t)k * ck_bytes, fb, false));
    s.step = c0;
    s.staggered = true;
    s.n_rcv = 0;  // no trace recording while recomputing
    loss_status_t st = copy_arrays(h, part, (char*)sg, fb, true);
    for (int64_t n = c0; n < c1 && st == LOSS_OK; ++n) {
      st = step_shot(h, s);
      if (st == LOSS_OK) st = copy_arrays(h, part, (char*)sg + (size_t)(n + 1 - c0) * part.size() * fb, fb, true);
    }
    s.n_rcv = nrcv_saved;
    LOSS_TRY(st);
    for (int64_t n = c1 - 1; n >= c0; --n) {
      const Snap sn{(char*)sg + (size_t)(n - c0) * part.size() * fb, fb};
      const Snap sn1{(char*)sg + (size_t)(n + 1 - c0) * part.size() * fb, fb};
      LOSS_TRY(adjoint_step<T>(h, s, sn, sn1, n, (const InjectJob<T>*)djobs, (int)jobs.size(), max_cnt));
    }
  }
  // leave the shot at the end of the forward run
  LOSS_TRY(copy_arrays(h, full, (char*)ck + (size_t)K * ck_bytes, fb, false));
  s.step = n_steps;
  s.staggered = true;
  s.rcv_steps = rsteps_saved;
  // gradients of the model coefficients, dense, FP64
  const int nk = 3;
  for (int i = 0; i < nk; ++i) {
    grads_out[i].assign((size_t)s.dense, 0.0);
    const size_t w = (size_t)s.len[2] * sizeof(double);
    LOSS_TRY(cuda_check(h, cudaMemcpy2DAsync(grads_out[i].data(), w, s.grad[i], (size_t)s.px * sizeof(double), w,
                                             (size_t)(s.len[0] * s.len[1]), cudaMemcpyDeviceToHost, h->stream),
                        "copy gradient"));
  }
  LOSS_TRY(cuda_check(h, cudaStreamSynchronize(h->stream), "sync"));
  return LOSS_OK;
}

loss_status_t run_gradient(loss_ctx* h, Shot& s, const double* d_obs, int32_t checkpoint_every, int64_t n_steps,
                           double* misfit, double* g_vp, double* g_vs, double* g_rho, int32_t mem) {
  if (n_steps < 1) return err(h, LOSS_E_ARG, "n_steps must be >= 1");
  if (checkpoint_every < 0) return err(h, LOSS_E_ARG, "checkpoint_every must be >= 0");
  if (!s.has_model || s.h_rho.empty()) return err(h, LOSS_E_STATE, "loss_set_model must precede loss_gradient");
  if (s.n_rcv == 0) return err(h, LOSS_E_STATE, "the shot has no receivers");
  if (!(s.d.physics == LOSS_ELASTIC || (s.d.physics == LOSS_ACOUSTIC && s.dim == 2)))
    return err(h, LOSS_E_UNSUPPORTED, "gradients are built for 2-D acoustic and 3-D elastic grids");
  if (s.src_on && (s.src_kinds & kForceMask))
    return err(h, LOSS_E_UNSUPPORTED, "gradients with a body-force source are not built");
  if (!d_obs || !misfit || !g_vp || !g_rho || (s.d.physics == LOSS_ELASTIC && !g_vs))
    return err(h, LOSS_E_ARG, "null argument");
  if (mem != LOSS_MEM_HOST && mem != LOSS_MEM_DEVICE) return err(h, LOSS_E_ARG, "bad mem");
  const int64_t C = checkpoint_every > 0 ? checkpoint_every : (int64_t)std::ceil(std::sqrt((double)n_steps));
  const size_t nobs = (size_t)n_steps * s.n_rcv;
  std::vector<double> obs;
  const double* ho = d_obs;
  if (mem == LOSS_MEM_DEVICE) {
    obs.resize(nobs);
    LOSS_TRY(cuda_check(h, cudaMemcpy(obs.data(), d_obs, nobs * sizeof(double), cudaMemcpyDeviceToHost), "copy d_obs"));
    ho = obs.data();
  }
  std::vector<double> gk[3];
  if (s.esize == 8) LOSS_TRY(gradient_t<double>(h, s, ho, C, n_steps, misfit, gk));
  else LOSS_TRY(gradient_t<float>(h, s, ho, C, n_steps, misfit, gk));
  // chain rule (FP64, dense): kappa = rho vp^2 | lambda = rho (vp^2 - 2 vs^2), mu = rho vs^2; b = 1 / rho
  const size_t N = (size_t)s.dense;
  std::vector<double> ovp(N), ovs(s.d.physics == LOSS_ELASTIC ? N : 0), orho(N);
  for (size_t i = 0; i < N; ++i) {
    const double vp = s.h_vp[i], rho = s.h_rho[i];
    if (s.d.physics == LOSS_ELASTIC) {
      const double vs = s.h_vs[i];
      ovp[i] = gk[0][i] * 2.0 * rho * vp;
      ovs[i] = gk[0][i] * (-4.0 * rho * vs) + gk[1][i] * 2.0 * rho * vs;
      orho[i] = gk[0][i] * (vp * vp - 2.0 * vs * vs) + gk[1][i] * vs * vs - gk[2][i] / (rho * rho);
    } else {
      ovp[i] = gk[0][i] * 2.0 * rho * vp;
      orho[i] = gk[0][i] * vp * vp - gk[2][i] / (rho * rho);
    }
  }
  const cudaMemcpyKind kind = mem == LOSS_MEM_HOST ? cudaMemcpyHostToHost : cudaMemcpyHostToDevice;
  LOSS_TRY(cuda_check(h, cudaMemcpy(g_vp, ovp.data(), N * sizeof(double), kind), "copy g_vp"));
  LOSS_TRY(cuda_check(h, cudaMemcpy(g_rho, orho.data(), N * sizeof(double), kind), "copy g_rho"));
  if (s.d.physics == LOSS_ELASTIC)
    LOSS_TRY(cuda_check(h, cudaMemcpy(g_vs, ovs.data(), N * sizeof(double), kind), "copy g_vs"));
  return LOSS_OK;
}

// Stand-alone D^T along internal slot k of dense arrays (DEVICE pointers).
template <typename T>
static loss_status_t derivative_adjoint_t(loss_ctx* h, Shot& s, int k, const T* g, T* out) {
  if (s.nu_tab[k]) return run_nu_derivative_adjoint<T>(h, s, k, g, out);  // an axis with knots
  const int64_t sy = s.len[2], sz = s.len[2] * s.len[1];
  LineGeom geo;
  int logc, threads;
  LOSS_TRY(line_geom(h, s, k, sz, sy, &geo, &logc, &threads, 4, 0, h->lines_per_block[LOSS_KERNEL_ADJOINT],
                     adj_logc<T>(h), adj_threads<T>(h)));
  AdjArgs<T> a{};
  a.g = geo;
  a.tb = Tables{s.W[k], h->t32, h->t64};
  a.s3h = (T)(3.0 / s.h[k]);
  a.s3hd = 3.0 / s.h[k];
  a.minf = (T)(2.0 - std::sqrt(3.0));
  a.mode = 0;
  a.in3 = g;
  a.out = out;
  LOSS_TRY(cuda_check(h, cudaMemsetAsync(out, 0, (size_t)s.dense * sizeof(T), h->stream), "memset"));
  LaunchScope ls(h, LOSS_KERNEL_ADJOINT);
  return cuda_check(h, launch_adj<T>(a, logc, k != 2, threads, h->stream), "adjoint kernel");
}

loss_status_t run_derivative_adjoint(loss_ctx* h, Shot& s, int k, const void* g, void* out, int mem) {
  const size_t fb = (size_t)s.dense * s.esize;
  void *dg = (void*)g, *dout = out;
  std::vector<void*> tmp;
  if (mem == LOSS_MEM_HOST) {
    LOSS_TRY(dev_alloc(h, fb, &dg));
    tmp.push_back(dg);
    LOSS_TRY(dev_alloc(h, fb, &dout));
    tmp.push_back(dout);
    LOSS_TRY(cuda_check(h, cudaMemcpyAsync(dg, g, fb, cudaMemcpyHostToDevice, h->stream), "copy g"));
  }
  loss_status_t st = s.esize == 8 ? derivative_adjoint_t<double>(h, s, k, (const double*)dg, (double*)dout)
                                  : derivative_adjoint_t<float>(h, s, k, (const float*)dg, (float*)dout);
  if (st == LOSS_OK && mem == LOSS_MEM_HOST) {
    st = cuda_check(h, cudaMemcpyAsync(out, dout, fb, cudaMemcpyDeviceToHost, h->stream), "copy out");
    if (st == LOSS_OK) st = cuda_check(h, cudaStreamSynchronize(h->stream), "sync");
  }
  for (void* p : tmp) dev_free(h, p);
  return st;
}

}  // namespace lossk
