// Time-stepping schedule (paper Sec. 3.3): Strang splitting "half A, full B, half A" with the velocity
// sub-step A and the stress sub-step B.  Between steps the velocities are kept half a step ahead (staggered),
// which merges the trailing half A of one step with the leading half A of the next; the state is brought back
// to the integer time level (v_n = v_{n+1/2} + dt/2 b grad sigma_n) whenever velocities are read.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "loss_fir.cuh"
#include "loss_host.h"

namespace lossk {

#define LOSS_TRY(expr)              \
  do {                              \
    loss_status_t st_ = (expr);     \
    if (st_ != LOSS_OK) return st_; \
  } while (0)

static double ricker(double t, double f0, double t0) {
  const double a = (M_PI * f0 * (t - t0)) * (M_PI * f0 * (t - t0));
  return (1.0 - 2.0 * a) * std::exp(-a);
}

// ---------------------------------------------------------------------------------------------------------------
// 2-D acoustic.
template <typename T>
static PmlAxis<T> pml_axis(const Shot& s, int k, double tau) {
  const int v = (tau == s.d.dt) ? 0 : (tau > 0 ? 1 : 2);
  // half-step table for the receiver corrections of full velocity sub-steps
  const T* th = (v == 0) ? (const T*)s.pml_tab[k][1] : nullptr;
  return PmlAxis<T>{(const T*)s.pml_tab[k][v], s.pml_width, (int)s.n[k], th};
}

// Receiver corrections are needed when velocities are recorded inside absorbing layers.
static loss_status_t ensure_rdelta(loss_ctx* h, Shot& s) {
  bool vel = false;
  for (int f = 0; f < 3; ++f) vel = vel || !s.rcv[f].empty();
  if (!s.pml_on || !vel || s.rdelta[0]) return LOSS_OK;
  const size_t fb = (size_t)s.total * s.esize;
  for (int i = 0; i < 9; ++i) {
    LOSS_TRY(dev_alloc(h, fb, &s.rdelta[i]));
    LOSS_TRY(cuda_check(h, cudaMemsetAsync(s.rdelta[i], 0, fb, h->stream), "memset"));
  }
  return LOSS_OK;
}

// Correction array of velocity component i (0..2) and derivative direction j (0 = x, 1 = y, 2 = z).
template <typename T>
static T* rdelta(const Shot& s, int i, int j, double tau) {
  return (tau == s.d.dt && s.rdelta[0]) ? (T*)s.rdelta[3 * i + j] : nullptr;
}

template <typename T>
static AcXArgs<T> ac_x_args(loss_ctx* h, Shot& s, const LineGeom& g, int do_B, double acoef, double src_amp) {
  AcXArgs<T> a{};
  a.g = g;
  a.tb = Tables{s.W[2], h->t32, h->t64};
  a.sigma = (T*)s.field[LOSS_FIELD_SIGMA];
  a.v1 = (T*)s.field[LOSS_FIELD_V1];
  a.kappa = (const T*)s.model[0];
  a.b = s.b_const ? nullptr : (const T*)s.model[1];
  a.b0 = (T)s.b0;
  a.tmp = (const T*)s.tmp[0];
  a.csig = (T*)s.comp[LOSS_FIELD_SIGMA];
  a.cv1 = (T*)s.comp[LOSS_FIELD_V1];
  a.dt = (T)s.d.dt;
  a.acoef = (T)acoef;
  a.s3h = (T)(3.0 / s.h[2]);
  a.dt_lo = lo_part<T>(s.d.dt);
  a.acoef_lo = lo_part<T>(acoef);
  a.s3h_lo = lo_part<T>(3.0 / s.h[2]);
  a.b0_lo = lo_part<T>(s.b0);
  a.sc = (T)(-acoef * s.b0 * (3.0 / s.h[2]));
  a.sc_lo = lo_part<T>(-acoef * s.b0 * (3.0 / s.h[2]));
  a.minf = (T)(2.0 - std::sqrt(3.0));
  a.do_B = do_B;
  a.src.on = (do_B && s.src_on && src_amp != 0.0) ? 1 : 0;
  a.src.zs = (int)s.src_idx[0];
  a.src.ys = 0;
  a.src.xs = (int)s.src_idx[2];
  a.src.amp = src_amp;
  for (int i = 0; i < 25; ++i) a.src.g[i] = s.src_g[i];
  a.pml = s.pml_on ? 1 : 0;
  if (s.pml_on) {
    a.xA = pml_axis<T>(s, 2, acoef);
    a.xB = pml_axis<T>(s, 2, s.d.dt);
    a.zB = pml_axis<T>(s, 0, s.d.dt);
    a.psix = (T*)s.psi[2];
    a.phix = (T*)s.phi[2];
    a.phiz = (T*)s.phi[0];
    a.dlt = rdelta<T>(s, 0, 0, acoef);
  }
  return a;
}

template <typename T, bool K>
static loss_status_t ac_x(loss_ctx* h, Shot& s, int do_B, double acoef, double src_amp) {
  LineGeom g;
  int logc, threads;
  LOSS_TRY(line_geom(h, s, 2, s.sz, s.sy, &g, &logc, &threads, 3, 4, h->lines_per_block[LOSS_KERNEL_ACOUSTIC_X],
                     h->chunk_log2[LOSS_KERNEL_ACOUSTIC_X], h->tile_threads[LOSS_KERNEL_ACOUSTIC_X]));
  const AcXArgs<T> a = ac_x_args<T>(h, s, g, do_B, acoef, src_amp);
  LaunchScope ls(h, LOSS_KERNEL_ACOUSTIC_X);
  return cuda_check(h, launch_ac_x<T, K>(a, logc, threads, h->stream), "acoustic x kernel");
}

template <typename T>
static AcZArgs<T> ac_z_args(loss_ctx* h, Shot& s, const LineGeom& g, double acoef, int do_tmp) {
  AcZArgs<T> a{};
  a.g = g;
  a.tb = Tables{s.W[0], h->t32, h->t64};
  a.sigma = (const T*)s.field[LOSS_FIELD_SIGMA];
  a.v3 = (T*)s.field[LOSS_FIELD_V3];
  a.b = s.b_const ? nullptr : (const T*)s.model[1];
  a.b0 = (T)s.b0;
  a.tmp = (T*)s.tmp[0];
  a.cv3 = (T*)s.comp[LOSS_FIELD_V3];
  a.acoef = (T)acoef;
  a.s3h = (T)(3.0 / s.h[0]);
  a.acoef_lo = lo_part<T>(acoef);
  a.s3h_lo = lo_part<T>(3.0 / s.h[0]);
  a.b0_lo = lo_part<T>(s.b0);
  a.sc = (T)(-acoef * s.b0 * (3.0 / s.h[0]));
  a.sc_lo = lo_part<T>(-acoef * s.b0 * (3.0 / s.h[0]));
  a.minf = (T)(2.0 - std::sqrt(3.0));
  a.do_tmp = do_tmp;
  a.pml = s.pml_on ? 1 : 0;
  if (s.pml_on) {
    a.zA = pml_axis<T>(s, 0, acoef);
    a.psiz = (T*)s.psi[0];
    a.dlt = rdelta<T>(s, 2, 2, acoef);
  }
  return a;
}

template <typename T, bool K>
static loss_status_t ac_z(loss_ctx* h, Shot& s, double acoef, int do_tmp) {
  LineGeom g;
  int logc, threads;
  LOSS_TRY(line_geom(h, s, 0, s.sz, s.sy, &g, &logc, &threads, 2, 0, h->lines_per_block[LOSS_KERNEL_ACOUSTIC_Z],
                     h->chunk_log2[LOSS_KERNEL_ACOUSTIC_Z], h->tile_threads[LOSS_KERNEL_ACOUSTIC_Z]));
  const AcZArgs<T> a = ac_z_args<T>(h, s, g, acoef, do_tmp);
  LaunchScope ls(h, LOSS_KERNEL_ACOUSTIC_Z);
  return cuda_check(h, launch_ac_z<T, K>(a, logc, threads, h->stream), "acoustic z kernel");
}

// ---------------------------------------------------------------------------------------------------------------
// FP32 tiles in the truncated-convolution form (loss_kernels_tiled.cu): four launches per step.
static bool tiled_ok(const loss_ctx* h, const Shot& s) {
  if (!h->tiled || s.esize != 4 || s.dim != 2 || s.d.physics != LOSS_ACOUSTIC) return false;
  const int Mz = (int)(s.n[0] / s.p[0]);
  return Mz <= 512 && std::max(s.d.n_nb, FirLen<float>::K) <= 64;
}

// z tiles: 32 columns x one patch, C = 2^zlogc positions per thread (a warp row); x rows: C = 8.
static TileGeom tile_geom(const Shot& s, int k, int* threads, int zlogc = 4) {
  TileGeom t{};
  t.n = (int)s.n[k];
  t.p = s.p[k];
  t.M = t.n / t.p;
  t.n_nb = s.d.n_nb;
  t.px = s.px;
  t.W = s.W[k];
  const FirConst fc = fir_const(t.M);
  t.s3h = (float)(3.0 / s.h[k]);
  t.s3h_lo = lo_part<float>(3.0 / s.h[k]);
  t.r = (float)fc.r;
  t.a = (float)fc.a;
  t.rho = (float)fc.rho;
  t.inv = (float)fc.inv;
  t.Wd = s.Wd[k];
  t.Rd = std::max(s.d.n_nb, FirLen<float>::K);
  t.pw = s.pml_on ? s.pml_width : 0;
  t.H = t.Rd;
  if (k == 0) {
    t.ncross = (int)s.len[2];
    t.ntl = (t.ncross + 31) / 32;
    t.R = 32;
    const int C = 1 << zlogc;
    *threads = 32 * ((t.M + C - 1) / C);
  } else {
    t.ncross = (int)s.len[0];
    t.ntl = t.ncross;
    t.R = 1;
    *threads = (((t.n + 7) / 8 + 31) / 32) * 32;
  }
  return t;
}

// Junction-correction weights of axis slot k in device memory (FP32 truncated-convolution kernels).
static loss_status_t ensure_delta_weights(loss_ctx* h, Shot& s, int k) {
  if (s.Wd[k]) return LOSS_OK;
  const std::vector<double> D = fir_delta_weights((int)s.n[k], s.p[k], s.d.n_nb, FirLen<float>::K);
  void* p = nullptr;
  LOSS_TRY(dev_alloc(h, D.size() * sizeof(double), &p));
  LOSS_TRY(cuda_check(h, cudaMemcpyAsync(p, D.data(), D.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream),
                      "copy junction weights"));
  LOSS_TRY(cuda_check(h, cudaStreamSynchronize(h->stream), "sync"));
  s.Wd[k] = (double*)p;
  return LOSS_OK;
}

// The pipelined x kernel takes rows of at most 4097 points (blocks of 256 threads up to 2049, of 512 above) in at
// most 64 patches whose length is a multiple of 8, with the staged rows within shared memory.
static bool xp_ok(const loss_ctx* h, const Shot& s, const TileGeom& t) {
  return h->tiled != LOSS_KERNELS_CONVOLUTION_ITEMS && s.n[2] <= 4096 && s.p[2] <= 64 && (s.n[2] / s.p[2]) % 8 == 0 &&
         xp_smem(t, s.kahan) + 2048 <= (size_t)h->smem_optin;
}

// x part of the FP32 step (sub-step B and the x part of A, or the latter alone): the pipelined row kernel when a
// row fits its shared-memory stages, else the (row, patch) item kernels, two launches.
template <bool K>
static loss_status_t xpart(loss_ctx* h, Shot& s, int do_B, double acoef, double amp) {
  int threads;
  TileGeom t = tile_geom(s, 2, &threads);
  LOSS_TRY(ensure_delta_weights(h, s, 2));
  t.Wd = s.Wd[2];
  t.ncross = (int)s.len[0];
  const AcXArgs<float> a = ac_x_args<float>(h, s, LineGeom{}, do_B, acoef, amp);
  LaunchScope ls(h, LOSS_KERNEL_ACOUSTIC_X);
  if (xp_ok(h, s, t)) {
    const unsigned mm = (unsigned)((((uint64_t)1 << 32) + (uint64_t)t.M - 1) / (uint64_t)t.M);
    return cuda_check(h, launch_xp<K>(a, t, mm, h->dflag, h->wait_polls, h->num_sms, h->stream), "acoustic x kernel");
  }
  if (xt_smem(t) > (size_t)h->smem_optin) {
    h->err = "x patch does not fit in shared memory";
    return LOSS_E_UNSUPPORTED;
  }
  return cuda_check(h, launch_xt<K>(a, t, h->stream), "acoustic x item kernels");
}

bool conv_z_used(const loss_ctx* h) {
  for (const Shot& s : h->shots)
    if (tiled_ok(h, s)) return true;
  return false;
}

// log2 of the z tile chunk of Z1 (mode 1) or Z2 (mode 2): the tuned value, else 16 positions.
static int zchunk_log2(const loss_ctx* h, int mode) {
  const int c = h->chunk_log2[mode == 1 ? LOSS_KERNEL_ACOUSTIC_Z : LOSS_KERNEL_ACOUSTIC_Z2];
  return c == 3 ? 3 : 4;
}

template <bool K>
static loss_status_t tz(loss_ctx* h, Shot& s, int mode, double acoef) {
  LOSS_TRY(ensure_delta_weights(h, s, 0));
  int threads;
  const int lc = zchunk_log2(h, mode);
  const TileGeom t = tile_geom(s, 0, &threads, lc);
  const AcZArgs<float> a = ac_z_args<float>(h, s, LineGeom{}, acoef, 0);
  LaunchScope ls(h, mode == 1 ? LOSS_KERNEL_ACOUSTIC_Z : LOSS_KERNEL_ACOUSTIC_Z2);
  return cuda_check(h, launch_tz<K>(a, t, mode, threads, lc, h->stream), "acoustic z tile kernel");
}

template <typename T>
static loss_status_t gather_fields(loss_ctx* h, Shot& s, bool velocities, int mode, cudaStream_t st = nullptr) {
  if (s.n_rcv == 0) return LOSS_OK;
  if (!st) st = h->stream;
  T* row = (T*)s.traces + (size_t)s.rcv_steps * s.n_rcv;
  for (int f = 0; f < LOSS_NUM_FIELDS; ++f) {
    const int64_t off = s.rcv_offsets[f], cnt = s.rcv_offsets[f + 1] - off;
    if (cnt == 0 || is_velocity(f) != velocities) continue;
    LaunchScope ls(h, LOSS_KERNEL_GATHER);
    const T* d[3] = {nullptr, nullptr, nullptr};
    if (mode == 1 && s.rdelta[0])
      for (int j = 0; j < 3; ++j) d[j] = (const T*)s.rdelta[3 * f + j];
    LOSS_TRY(cuda_check(h, launch_gather<T>((const T*)s.field[f], s.rcv_idx + off, cnt, row + off, mode, d[0], d[1],
                                            d[2], st),
                        "receiver gather"));
  }
  return LOSS_OK;
}

// Pressure-source increment of step n (applied in sub-step B at t_n + dt/2), or 0.
static double pressure_amp(const Shot& s, int64_t n) {
  if (!(s.src_on && (s.src_kinds & LOSS_SRC_PRESSURE))) return 0.0;
  const double dt = s.d.dt;
  return dt * s.src_norm * ricker((double)n * dt + 0.5 * dt, s.src_f0, s.src_t0);
}

// The staggered start: half velocity sub-step, then d_z v3 for the first B.
template <typename T, bool K>
static loss_status_t acoustic2d_start(loss_ctx* h, Shot& s) {
  const double dt = s.d.dt;
  if (sizeof(T) == 4 && tiled_ok(h, s)) {
    LOSS_TRY(xpart<K>(h, s, 0, 0.5 * dt, 0.0));
    LOSS_TRY(tz<K>(h, s, 1, 0.5 * dt));
    return tz<K>(h, s, 2, 0.0);
  }
  LOSS_TRY((ac_x<T, K>(h, s, 0, 0.5 * dt, 0.0)));
  return ac_z<T, K>(h, s, 0.5 * dt, 1);
}

// The pressure receivers of a step read sigma, which is final once the x kernel has run: their gather runs on the
// handle's side stream, overlapping the z kernels, and the main stream waits for it at the end of the step (the next
// step's x kernel rewrites sigma).  With per-launch profiling on, everything stays on the main stream.
static loss_status_t side_gather_begin(loss_ctx* h, bool* on) {
  *on = !h->prof && !h->capturing;
  if (!*on) return LOSS_OK;
  if (!h->side) {
    LOSS_TRY(cuda_check(h, cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking), "side stream"));
    LOSS_TRY(cuda_check(h, cudaEventCreateWithFlags(&h->ev_x, cudaEventDisableTiming), "event"));
    LOSS_TRY(cuda_check(h, cudaEventCreateWithFlags(&h->ev_g, cudaEventDisableTiming), "event"));
  }
  LOSS_TRY(cuda_check(h, cudaEventRecord(h->ev_x, h->stream), "record"));
  return cuda_check(h, cudaStreamWaitEvent(h->side, h->ev_x, 0), "wait");
}

template <typename T, bool K>
static loss_status_t acoustic2d_step(loss_ctx* h, Shot& s) {
  const double dt = s.d.dt;
  LOSS_TRY(ensure_rdelta(h, s));
  if (!s.staggered) {
    LOSS_TRY((acoustic2d_start<T, K>(h, s)));
    s.staggered = true;
  }
  LOSS_TRY(gather_fields<T>(h, s, true, 0));  // v at t_{n+1/2}
  const bool conv = sizeof(T) == 4 && tiled_ok(h, s);
  if (conv) LOSS_TRY(xpart<K>(h, s, 1, dt, pressure_amp(s, s.step)));
  else LOSS_TRY((ac_x<T, K>(h, s, 1, dt, pressure_amp(s, s.step))));
  bool side = false;
  if (s.n_rcv) {
    LOSS_TRY(side_gather_begin(h, &side));
    LOSS_TRY(gather_fields<T>(h, s, false, 0, side ? h->side : h->stream));  // sigma_{n+1}
    if (side) LOSS_TRY(cuda_check(h, cudaEventRecord(h->ev_g, h->side), "record"));
  }
  if (conv) {
    LOSS_TRY(tz<K>(h, s, 1, dt));
    LOSS_TRY(tz<K>(h, s, 2, 0.0));
  } else {
    LOSS_TRY((ac_z<T, K>(h, s, dt, 1)));
  }
  LOSS_TRY(gather_fields<T>(h, s, true, 1));   // (v_{n+1/2} + v_{n+3/2}) / 2 = v_{n+1}
  if (side) LOSS_TRY(cuda_check(h, cudaStreamWaitEvent(h->stream, h->ev_g, 0), "wait"));
  if (s.n_rcv) ++s.rcv_steps;
  ++s.step;
  return LOSS_OK;
}

template <typename T, bool K>
static loss_status_t acoustic2d_unstagger(loss_ctx* h, Shot& s) {
  const double dt = s.d.dt;
  if (sizeof(T) == 4 && tiled_ok(h, s)) {
    LOSS_TRY(xpart<K>(h, s, 0, -0.5 * dt, 0.0));
    LOSS_TRY(tz<K>(h, s, 1, -0.5 * dt));
    s.staggered = false;
    return LOSS_OK;
  }
  LOSS_TRY((ac_x<T, K>(h, s, 0, -0.5 * dt, 0.0)));
  LOSS_TRY((ac_z<T, K>(h, s, -0.5 * dt, 0)));
  s.staggered = false;
  return LOSS_OK;
}


// ---------------------------------------------------------------------------------------------------------------
// 3-D elastic: five line passes per step (loss_kernels_elastic.cu).
enum { EL_BX = 0, EL_BY = 1, EL_BZ = 2, EL_AX = 3, EL_AY = 4 };

// Arguments of an elastic pass along axis slot k that do not depend on its launch shape.
template <typename T>
static ElArgs<T> el_args(const loss_ctx* h, Shot& s, int k, int pass_src, int do_B, int do_A, double acoef,
                         double amp) {
  ElArgs<T> a{};
  a.tb = Tables{s.W[k], h->t32, h->t64};
  int srcf[3];
  switch (pass_src) {
    case 0: srcf[0] = LOSS_FIELD_V1, srcf[1] = LOSS_FIELD_V2, srcf[2] = LOSS_FIELD_V3; break;
    case 1: srcf[0] = LOSS_FIELD_S13, srcf[1] = LOSS_FIELD_S23, srcf[2] = LOSS_FIELD_S33; break;
    case 2: srcf[0] = LOSS_FIELD_S11, srcf[1] = LOSS_FIELD_S12, srcf[2] = LOSS_FIELD_S13; break;
    default: srcf[0] = LOSS_FIELD_S12, srcf[1] = LOSS_FIELD_S22, srcf[2] = LOSS_FIELD_S23; break;
  }
  for (int i = 0; i < 3; ++i) a.src[i] = (const T*)s.field[srcf[i]];
  for (int f = 0; f < 9; ++f) {
    a.fld[f] = (T*)s.field[f];
    a.cmp[f] = (T*)s.comp[f];
  }
  for (int i = 0; i < 8; ++i) a.tmp[i] = (T*)s.tmp[i];
  a.lam = s.lam_const ? nullptr : (const T*)s.model[0];
  a.mu = s.mu_const ? nullptr : (const T*)s.model[1];
  a.b = s.b_const ? nullptr : (const T*)s.model[2];
  a.lam0 = (T)s.lam0;
  a.mu0 = (T)s.mu0;
  a.b0 = (T)s.b0;
  a.dt = (T)s.d.dt;
  a.acoef = (T)acoef;
  a.s3h = (T)(3.0 / s.h[k]);
  a.dt_lo = lo_part<T>(s.d.dt);
  a.acoef_lo = lo_part<T>(acoef);
  a.s3h_lo = lo_part<T>(3.0 / s.h[k]);
  a.lam0_lo = lo_part<T>(s.lam0);
  a.mu0_lo = lo_part<T>(s.mu0);
  a.b0_lo = lo_part<T>(s.b0);
  a.minf = (T)(2.0 - std::sqrt(3.0));
  a.do_B = do_B;
  a.do_A = do_A;
  a.pml = s.pml_on ? 1 : 0;
  if (s.pml_on) {
    a.pB = pml_axis<T>(s, k, s.d.dt);
    a.pA = pml_axis<T>(s, k, acoef);
    // derivative direction j (1 = x, 2 = y, 3 = z) of this pass
    const int j = (k == 2) ? 1 : (k == 1 ? 2 : 3);
    for (int i = 0; i < 3; ++i) a.memB[i] = (T*)s.pmem[3 * i + (j - 1)];  // d_j v_i
    // velocity sub-step terms d_j sigma_ij, equation i = 1..3
    for (int i = 0; i < 3; ++i) a.memA[i] = (T*)s.pmem[9 + 3 * i + (j - 1)];
    for (int i = 0; i < 3; ++i) a.dlt[i] = do_A ? rdelta<T>(s, i, j - 1, acoef) : nullptr;
  }
  a.srcp.on = amp != 0.0 ? 1 : 0;
  a.srcp.zs = (int)s.src_idx[0];
  a.srcp.ys = (int)s.src_idx[1];
  a.srcp.xs = (int)s.src_idx[2];
  a.srcp.amp = amp;
  for (int i = 0; i < 25; ++i) a.srcp.g[i] = s.src_g[i];
  a.src_explosive = (s.src_kinds & LOSS_SRC_EXPLOSIVE) ? 1 : 0;
  a.src_shear = (s.src_kinds & LOSS_SRC_SHEAR_XZ) ? 1 : 0;
  a.force_mask = force_components(s.src_kinds);
  return a;
}

// The FP32 y / z tile passes: the convolution family (loss_set_kernels), patches of at most 256 positions (8-position
// chunks up to M = 64, at most 8 warps; 16-position chunks above, at most 16 warps) and tiles within shared memory.
static int elt_logc(const Shot& s, int k) { return (s.n[k] / s.p[k]) <= 64 ? 3 : 4; }
static ElTile elt_geom(const Shot& s, int k) {
  ElTile g{};
  int threads;
  g.t = tile_geom(s, k, &threads);
  g.t.px = (k == 1) ? s.sy : s.sz;
  g.t.Wd = s.Wd[k];
  g.ostride = (k == 1) ? s.sz : s.sy;
  g.nouter = (int)((k == 1) ? s.len[0] : s.len[1]);
  g.nx = (int)s.len[2];
  g.ncg = (g.nx + 31) / 32;
  return g;
}
static bool elt_ok(const loss_ctx* h, const Shot& s) {
  if (s.esize != 4 || !h->tiled || s.dim != 3) return false;
  for (int k = 0; k < 2; ++k) {
    const int M = (int)(s.n[k] / s.p[k]);
    if (M > 256 || std::max(s.d.n_nb, FirLen<float>::K) > 64) return false;
    if (elt_smem(elt_geom(s, k), elt_logc(s, k)) + 8192 > (size_t)h->smem_optin) return false;
  }
  return true;
}

template <bool K>
static loss_status_t elt_pass(loss_ctx* h, Shot& s, int pass, double acoef, double amp) {
  const int k = (pass == ET_BY || pass == ET_AY) ? 1 : 0;
  LOSS_TRY(ensure_delta_weights(h, s, k));
  const int src = (pass == ET_BY || pass == ET_BZ) ? 0 : (pass == ET_AZ ? 1 : 3);
  const int do_B = (pass == ET_BY || pass == ET_BZ) ? 1 : 0;
  const ElArgs<float> a = el_args<float>(h, s, k, src, do_B, 1 - do_B, acoef, amp);
  const ElTile g = elt_geom(s, k);
  LaunchScope ls(h, k == 1 ? LOSS_KERNEL_ELASTIC_Y : LOSS_KERNEL_ELASTIC_Z);
  return cuda_check(h, launch_elt<K>(a, g, pass, elt_logc(s, k), h->stream), "elastic tile kernel");
}

template <typename T, bool K>
static loss_status_t el_pass(loss_ctx* h, Shot& s, int pass, int do_B, int do_A, double acoef, double amp) {
  // internal axis slot of the pass: x = 2, y = 1, z = 0
  const int k = (pass == EL_BX || pass == EL_AX) ? 2 : ((pass == EL_BY || pass == EL_AY) ? 1 : 0);
  LineGeom g;
  int logc, threads;
  const int kid = (k == 2) ? LOSS_KERNEL_ELASTIC_X : (k == 1 ? LOSS_KERNEL_ELASTIC_Y : LOSS_KERNEL_ELASTIC_Z);
  // Built-in FP32 shapes of the elastic passes (what the autotuner picks on the 257^3 and 193^3 grids): chunks of
  // 8 unknowns on every axis, 128 threads per x block and 256 per y / z block.
  int want_threads = h->tile_threads[kid], want_logc = h->chunk_log2[kid];
  if (sizeof(T) == 4 && h->lines_per_block[kid] <= 0) {
    if (want_threads <= 0) want_threads = k == 2 ? 128 : 256;
    if (want_logc <= 0) want_logc = 3;
  }
  LOSS_TRY(line_geom(h, s, k, s.sz, s.sy, &g, &logc, &threads, 6, 0, h->lines_per_block[kid], want_logc,
                     want_threads));
  int src;
  switch (pass) {
    case EL_BX:
    case EL_BY: src = 0; break;
    case EL_BZ: src = do_B ? 0 : 1; break;
    case EL_AX: src = 2; break;
    default: src = 3; break;
  }
  ElArgs<T> a = el_args<T>(h, s, k, src, do_B, do_A, acoef, amp);
  a.g = g;
  LaunchScope ls(h, kid);
  return cuda_check(h, launch_el<T, K>(a, pass, logc, threads, h->stream), "elastic kernel");
}

// Velocity sub-step of length tau on the current stresses (three passes); force_t = time of the body force.
template <typename T, bool K>
static loss_status_t elastic_A(loss_ctx* h, Shot& s, double tau, double force_t) {
  double famp = 0.0;
  if (s.src_on && (s.src_kinds & kForceMask)) famp = tau * s.src_norm * ricker(force_t, s.src_f0, s.src_t0);
  if (sizeof(T) == 4 && elt_ok(h, s)) {
    LOSS_TRY((elt_pass<K>(h, s, ET_AZ, tau, 0.0)));
    LOSS_TRY((el_pass<T, K>(h, s, EL_AX, 0, 1, tau, 0.0)));
    return elt_pass<K>(h, s, ET_AY, tau, famp);
  }
  LOSS_TRY((el_pass<T, K>(h, s, EL_BZ, 0, 1, tau, 0.0)));
  LOSS_TRY((el_pass<T, K>(h, s, EL_AX, 0, 1, tau, 0.0)));
  return el_pass<T, K>(h, s, EL_AY, 0, 1, tau, famp);
}

template <typename T, bool K>
static loss_status_t elastic3d_step(loss_ctx* h, Shot& s) {
  const double dt = s.d.dt;
  LOSS_TRY(ensure_rdelta(h, s));
  const double tn = (double)s.step * dt;
  if (!s.staggered) {
    LOSS_TRY((elastic_A<T, K>(h, s, 0.5 * dt, tn)));
    s.staggered = true;
  }
  LOSS_TRY(gather_fields<T>(h, s, true, 0));
  double amp = 0.0;
  if (s.src_on && (s.src_kinds & (LOSS_SRC_EXPLOSIVE | LOSS_SRC_SHEAR_XZ)))
    amp = dt * s.src_norm * ricker(tn + 0.5 * dt, s.src_f0, s.src_t0);
  double famp = 0.0;
  if (s.src_on && (s.src_kinds & kForceMask)) famp = dt * s.src_norm * ricker(tn + dt, s.src_f0, s.src_t0);
  if (sizeof(T) == 4 && elt_ok(h, s)) {
    LOSS_TRY((el_pass<T, K>(h, s, EL_BX, 1, 0, dt, 0.0)));
    LOSS_TRY((elt_pass<K>(h, s, ET_BY, dt, 0.0)));
    LOSS_TRY((elt_pass<K>(h, s, ET_BZ, dt, amp)));
    LOSS_TRY((elt_pass<K>(h, s, ET_AZ, dt, 0.0)));
    LOSS_TRY((el_pass<T, K>(h, s, EL_AX, 0, 1, dt, 0.0)));
    LOSS_TRY((elt_pass<K>(h, s, ET_AY, dt, famp)));
  } else {
    LOSS_TRY((el_pass<T, K>(h, s, EL_BX, 1, 0, dt, 0.0)));
    LOSS_TRY((el_pass<T, K>(h, s, EL_BY, 1, 0, dt, 0.0)));
    LOSS_TRY((el_pass<T, K>(h, s, EL_BZ, 1, 1, dt, amp)));
    LOSS_TRY((el_pass<T, K>(h, s, EL_AX, 0, 1, dt, 0.0)));
    LOSS_TRY((el_pass<T, K>(h, s, EL_AY, 0, 1, dt, famp)));
  }
  LOSS_TRY(gather_fields<T>(h, s, true, 1));
  LOSS_TRY(gather_fields<T>(h, s, false, 0));
  if (s.n_rcv) ++s.rcv_steps;
  ++s.step;
  return LOSS_OK;
}

template <typename T, bool K>
static loss_status_t elastic3d_unstagger(loss_ctx* h, Shot& s) {
  LOSS_TRY((elastic_A<T, K>(h, s, -0.5 * s.d.dt, (double)s.step * s.d.dt)));
  s.staggered = false;
  return LOSS_OK;
}

// ---------------------------------------------------------------------------------------------------------------
// Batched schedule for handles of 2-D acoustic shots: each step is one persistent launch of the X kernel and one
// of the Z kernel over the tiles of all shots, plus one launch per receiver phase and a clock tick.  Everything
// that changes from step to step (source amplitude, trace row) is read from device memory, so a step's launches
// have the same arguments every step: k steps are captured once in a CUDA graph and replayed.  Arithmetic is that
// of the per-shot schedule, so both give the same fields and traces.

static bool conv_batch_ok(const loss_ctx* h);

bool batch_eligible(const loss_ctx* h) {
  if (h->shots.empty()) return false;
  if (!(h->graph_steps > 0 || (h->batched && h->shots.size() > 1))) return false;
  const Shot& s0 = h->shots[0];
  for (const Shot& s : h->shots)
    if (s.d.physics != LOSS_ACOUSTIC || s.dim != 2 || s.esize != s0.esize || s.kahan != s0.kahan ||
        any_nonuniform(s))
      return false;
  // without the batched convolution kernels the batch runs the line kernels, which hold whole rows: shots with
  // rows the whole-row kernels do not take stay on the per-shot schedule (the (row, patch) item kernels)
  if (s0.esize == 4 && !conv_batch_ok(h))
    for (const Shot& s : h->shots)
      if (s.n[2] > 2048) return false;
  return true;
}

void batch_release(loss_ctx* h) {
  if (h->batch.gexec) cudaGraphExecDestroy(h->batch.gexec);
  h->batch.gexec = nullptr;
  h->batch.gsig.clear();
}

void batch_destroy(loss_ctx* h) {
  batch_release(h);
  if (h->batch.cap_stream) cudaStreamDestroy(h->batch.cap_stream);
  h->batch.cap_stream = nullptr;
}

// Per-step pressure amplitudes of steps 0 .. upto-1 in device memory (rebuilt when the source changed).
static loss_status_t ensure_amp(loss_ctx* h, Shot& s, int64_t upto) {
  const double sig[5] = {s.d.dt, s.src_norm, s.src_f0, s.src_t0, (double)(s.src_on ? s.src_kinds : 0u)};
  bool same = s.amp_tab != nullptr;
  for (int i = 0; i < 5 && same; ++i) same = sig[i] == s.amp_sig[i];
  if (same && upto <= s.amp_cap) return LOSS_OK;
  const int64_t cap = std::max<int64_t>(std::max<int64_t>(upto, same ? 2 * s.amp_cap : 0), 1024);
  std::vector<double> a((size_t)cap);
  for (int64_t n = 0; n < cap; ++n) a[n] = pressure_amp(s, n);
  void* p = nullptr;
  LOSS_TRY(dev_alloc(h, (size_t)cap * sizeof(double), &p));
  LOSS_TRY(cuda_check(h, cudaMemcpyAsync(p, a.data(), (size_t)cap * sizeof(double), cudaMemcpyHostToDevice, h->stream),
                      "upload source amplitudes"));
  LOSS_TRY(cuda_check(h, cudaStreamSynchronize(h->stream), "sync"));
  if (s.amp_tab) dev_free(h, s.amp_tab);
  s.amp_tab = (double*)p;
  s.amp_cap = cap;
  for (int i = 0; i < 5; ++i) s.amp_sig[i] = sig[i];
  return LOSS_OK;
}

// Geometry of every shot for one batched kernel, with one block size for all: the largest per-shot default
// block (or the loss_set_tile target), each shot taking the widest bundle that fits in it.
static loss_status_t batch_geoms(loss_ctx* h, int k, int kid, int nbuf, int nstage, std::vector<LineGeom>& gs,
                                 int* logc, int* threads, size_t* smem) {
  int target = h->tile_threads[kid];
  if (target <= 0 && h->lines_per_block[kid] <= 0) {
    for (Shot& s : h->shots) {
      LineGeom g;
      int lc, t;
      LOSS_TRY(line_geom(h, s, k, s.sz, s.sy, &g, &lc, &t, nbuf, nstage, 0, h->chunk_log2[kid]));
      target = std::max(target, t);
    }
  }
  if (target > kBatchThreads) target = kBatchThreads;
  gs.resize(h->shots.size());
  *logc = -1;
  *threads = 0;
  *smem = 0;
  for (size_t i = 0; i < h->shots.size(); ++i) {
    Shot& s = h->shots[i];
    int lc, t;
    LOSS_TRY(line_geom(h, s, k, s.sz, s.sy, &gs[i], &lc, &t, nbuf, nstage, h->lines_per_block[kid], h->chunk_log2[kid],
                       target));
    if (*logc >= 0 && lc != *logc) {
      h->err = "batched shots need one chunk length";
      return LOSS_E_UNSUPPORTED;
    }
    if (t > kBatchThreads) {
      h->err = "batched launches hold at most " + std::to_string(kBatchThreads) + " threads per block";
      return LOSS_E_UNSUPPORTED;
    }
    *logc = lc;
    *threads = std::max(*threads, t);
    *smem = std::max(*smem, smem_bytes(gs[i], nbuf, nstage, s.esize));
  }
  return LOSS_OK;
}

// Upload one device table when its contents changed (reallocating when it grew).
static loss_status_t upload_table(loss_ctx* h, int which, const std::vector<unsigned char>& bytes, void** dptr) {
  BatchState& B = h->batch;
  if (bytes.size() > B.cap_bytes[which] || !*dptr) {
    if (*dptr) dev_free(h, *dptr);
    *dptr = nullptr;
    LOSS_TRY(dev_alloc(h, std::max<size_t>(bytes.size(), 64), dptr));
    B.cap_bytes[which] = std::max<size_t>(bytes.size(), 64);
    B.host[which].clear();
  }
  if (bytes == B.host[which]) return LOSS_OK;
  if (!bytes.empty())
    LOSS_TRY(cuda_check(h, cudaMemcpyAsync(*dptr, bytes.data(), bytes.size(), cudaMemcpyHostToDevice, h->stream),
                        "upload batch tables"));
  LOSS_TRY(cuda_check(h, cudaStreamSynchronize(h->stream), "sync"));
  B.host[which] = bytes;
  return LOSS_OK;
}

template <class V>
static std::vector<unsigned char> as_bytes(const std::vector<V>& v) {
  const unsigned char* p = reinterpret_cast<const unsigned char*>(v.data());
  return std::vector<unsigned char>(p, p + v.size() * sizeof(V));
}

template <typename T, bool K>
static loss_status_t batch_launch_step(loss_ctx* h) {
  BatchState& B = h->batch;
  const int S = (int)h->shots.size();
  const GatherJob<T>* jobs = (const GatherJob<T>*)B.jobs;
  if (B.npre) {
    LaunchScope ls(h, LOSS_KERNEL_GATHER);
    LOSS_TRY(cuda_check(h, launch_gather_batch<T>(jobs, B.npre, B.pre_max, h->stream), "batched receiver gather"));
  }
  if constexpr (sizeof(T) == 4) {
    if (B.conv) {
      const int* unit0 = B.tile0;
      const int* bunit = unit0 + S + 1;
      const int* bshot = bunit + B.xpgrid + 1;
      const int* zt0 = bshot + B.xpgrid;
      {
        LaunchScope ls(h, LOSS_KERNEL_ACOUSTIC_X);
        LOSS_TRY(cuda_check(h, launch_xp_batch<K>((const XpShot*)B.xptab, unit0, bunit, bshot, B.xl, B.xpthreads,
                                                  B.xpgrid, h->dflag, h->wait_polls, h->stream),
                            "batched acoustic x kernel"));
      }
      for (int mode = 1; mode <= 2; ++mode) {
        LaunchScope ls(h, mode == 1 ? LOSS_KERNEL_ACOUSTIC_Z : LOSS_KERNEL_ACOUSTIC_Z2);
        LOSS_TRY(cuda_check(h, launch_tz_batch<K>((const TzShot*)B.tztab + (mode - 1) * S, zt0, S, B.tztiles, mode,
                                                  B.tzthreads[mode - 1], B.tzlogc[mode - 1], B.tzsmem[mode - 1],
                                                  B.tzgrid[mode - 1], h->stream),
                            "batched acoustic z tile kernel"));
      }
      if (B.npost) {
        LaunchScope ls(h, LOSS_KERNEL_GATHER);
        LOSS_TRY(cuda_check(h, launch_gather_batch<T>(jobs + B.npre, B.npost, B.post_max, h->stream),
                            "batched receiver gather"));
      }
      LaunchScope ls(h, LOSS_KERNEL_CLOCK);
      return cuda_check(h, launch_tick(B.clk, S, h->stream), "clock tick");
    }
  }
  {
    LaunchScope ls(h, LOSS_KERNEL_ACOUSTIC_X);
    LOSS_TRY(cuda_check(h, launch_ac_x_batch<T, K>((const AcXArgs<T>*)B.xtab, B.tile0, S, B.xtiles, B.xlogc,
                                                   B.xthreads, B.xsmem, B.xgrid, h->stream),
                        "batched acoustic x kernel"));
  }
  {
    LaunchScope ls(h, LOSS_KERNEL_ACOUSTIC_Z);
    LOSS_TRY(cuda_check(h, launch_ac_z_batch<T, K>((const AcZArgs<T>*)B.ztab, B.tile0 + S + 1, S, B.ztiles, B.zlogc,
                                                   B.zthreads, B.zsmem, B.zgrid, h->stream),
                        "batched acoustic z kernel"));
  }
  if (B.npost) {
    LaunchScope ls(h, LOSS_KERNEL_GATHER);
    LOSS_TRY(cuda_check(h, launch_gather_batch<T>(jobs + B.npre, B.npost, B.post_max, h->stream),
                        "batched receiver gather"));
  }
  LaunchScope ls(h, LOSS_KERNEL_CLOCK);
  return cuda_check(h, launch_tick(B.clk, S, h->stream), "clock tick");
}

template <typename T, bool K>
static loss_status_t capture_graph(loss_ctx* h, int64_t k) {
  BatchState& B = h->batch;
  batch_release(h);
  int64_t snap[LOSS_NUM_KERNELS];
  for (int i = 0; i < LOSS_NUM_KERNELS; ++i) snap[i] = h->launches[i];
  if (!B.cap_stream)
    LOSS_TRY(cuda_check(h, cudaStreamCreateWithFlags(&B.cap_stream, cudaStreamNonBlocking), "create capture stream"));
  // Capturing records the launches without running them, so the captured stream needs no ordering with the
  // handle's stream; the replays are issued on the handle's stream.
  cudaStream_t own = h->stream;
  LOSS_TRY(cuda_check(h, cudaStreamBeginCapture(B.cap_stream, cudaStreamCaptureModeThreadLocal),
                      "begin graph capture"));
  h->stream = B.cap_stream;
  h->capturing = true;
  loss_status_t st = LOSS_OK;
  for (int64_t i = 0; i < k && st == LOSS_OK; ++i) st = batch_launch_step<T, K>(h);
  h->capturing = false;
  h->stream = own;
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(B.cap_stream, &graph);
  for (int i = 0; i < LOSS_NUM_KERNELS; ++i) {
    B.graph_launches[i] = h->launches[i] - snap[i];
    h->launches[i] = snap[i];
  }
  if (st != LOSS_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return st != LOSS_OK ? st : cuda_check(h, e, "end graph capture");
  }
  const cudaError_t ei = cudaGraphInstantiate(&B.gexec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    B.gexec = nullptr;
    return cuda_check(h, ei, "instantiate graph");
  }
  B.graph_k = k;
  return LOSS_OK;
}

// Every shot takes the FP32 truncated-convolution kernels (z tiles of at most 512 threads and the pipelined x
// kernel), and their batched x layout fits shared memory.
static bool conv_batch_ok(const loss_ctx* h) {
  std::vector<TileGeom> ts;
  int threads = 32;
  for (const Shot& s : h->shots) {
    if (!tiled_ok(h, s)) return false;
    for (int mode = 1; mode <= 2; ++mode) {  // batched z blocks hold at most 512 threads
      int zt;
      tile_geom(s, 0, &zt, zchunk_log2(h, mode));
      if (zt > 512) return false;
    }
    int thr;
    TileGeom t = tile_geom(s, 2, &thr);
    if (s.n[2] > 2048 || !xp_ok(h, s, t)) return false;  // the batched x kernel takes blocks of at most 256 threads
    ts.push_back(t);
    threads = std::max(threads, thr);
  }
  while (threads & (threads - 1)) threads += 32;
  std::vector<int> rs;
  for (const TileGeom& t : ts) rs.push_back(xp_rows_per_unit(t.n, threads));
  return !ts.empty() &&
         (size_t)xp_batch_layout(ts, rs, h->shots[0].kahan).total * 4 + 2048 <= (size_t)h->smem_optin;
}

// Descriptors, work ranges and launch shapes of the batched convolution kernels (the shots are staggered and their
// amplitude tables exist).  The x blocks take whole units of rows in about equal numbers of points.
template <bool K>
static loss_status_t conv_tables(loss_ctx* h) {
  BatchState& B = h->batch;
  const int S = (int)h->shots.size();
  std::vector<XpShot> xs(S);
  std::vector<TzShot> zs(2 * S);
  std::vector<TileGeom> txs(S);
  std::vector<int> unit0(S + 1, 0), zt0(S + 1, 0), rs(S);
  int xthreads = 32, zthreads[2] = {32, 32};
  const int zlc[2] = {zchunk_log2(h, 1), zchunk_log2(h, 2)};
  size_t zsm[2] = {0, 0};
  int64_t ptot = 0;
  for (int i = 0; i < S; ++i) {
    int thr;
    tile_geom(h->shots[i], 2, &thr);
    xthreads = std::max(xthreads, thr);
  }
  while (xthreads & (xthreads - 1)) xthreads += 32;  // a power of two of warps, so that short rows form groups
  for (int i = 0; i < S; ++i) {
    Shot& s = h->shots[i];
    LOSS_TRY(ensure_delta_weights(h, s, 0));
    LOSS_TRY(ensure_delta_weights(h, s, 2));
    int thr;
    TileGeom tx = tile_geom(s, 2, &thr);
    tx.ncross = (int)s.len[0];
    XpShot& x = xs[i];
    x.a = ac_x_args<float>(h, s, LineGeom{}, 1, s.d.dt, 0.0);
    x.a.src.on = (s.src_on && (s.src_kinds & LOSS_SRC_PRESSURE)) ? 1 : 0;
    x.a.src.amp_tab = s.amp_tab;
    x.a.src.clk = B.clk + i;
    x.t = tx;
    x.mmagic = (unsigned)((((uint64_t)1 << 32) + (uint64_t)tx.M - 1) / (uint64_t)tx.M);
    rs[i] = xp_rows_per_unit(tx.n, xthreads);
    x.R = rs[i];
    x.unit0 = unit0[i];
    x.pad = 0;
    unit0[i + 1] = unit0[i] + (tx.ncross + rs[i] - 1) / rs[i];
    ptot += (int64_t)(tx.n + 1) * tx.ncross;
    txs[i] = tx;
    for (int m = 0; m < 2; ++m) {
      const TileGeom tz = tile_geom(s, 0, &thr, zlc[m]);
      zs[m * S + i] = TzShot{ac_z_args<float>(h, s, LineGeom{}, m == 0 ? s.d.dt : 0.0, 0), tz, thr >> 5, 0};
      zthreads[m] = std::max(zthreads[m], thr);
      zsm[m] = std::max(zsm[m], tile_smem_z(tz, m + 1, zlc[m]));
      if (m == 0) zt0[i + 1] = zt0[i] + tz.ntl * tz.p;
    }
  }
  B.xl = xp_batch_layout(txs, rs, K);
  B.xpthreads = xthreads;
  int per = 0;
  LOSS_TRY(cuda_check(h, xp_batch_per_sm<K>(B.xl, xthreads, &per), "batched x kernel shape"));
  if (per < 1) {
    h->err = "batched x kernel does not fit an SM";
    return LOSS_E_UNSUPPORTED;
  }
  const int G = (int)std::min<int64_t>(unit0[S], (int64_t)per * h->num_sms);
  // block b starts at the first unit whose preceding points reach b * ptot / G
  std::vector<int> brow(G + 1, unit0[S]), bshot(G, S - 1);
  {
    int b = 0, u = 0;
    int64_t before = 0;
    for (int i = 0; i < S && b < G; ++i)
      for (int w = 0; w < unit0[i + 1] - unit0[i] && b < G; ++w, ++u) {
        while (b < G && before >= (ptot * b + G - 1) / G) {
          brow[b] = u;
          bshot[b] = i;
          ++b;
        }
        before += (int64_t)(txs[i].n + 1) * std::min(rs[i], txs[i].ncross - w * rs[i]);
      }
  }
  B.xpgrid = G;
  B.tztiles = zt0[S];
  for (int m = 0; m < 2; ++m) {
    B.tzsmem[m] = zsm[m];
    B.tzthreads[m] = zthreads[m];
    B.tzlogc[m] = zlc[m];
    LOSS_TRY(cuda_check(h, tz_batch_per_sm<K>(m + 1, zthreads[m], zlc[m], zsm[m], &per), "batched z kernel shape"));
    if (per < 1) {
      h->err = "batched z kernel does not fit an SM";
      return LOSS_E_UNSUPPORTED;
    }
    B.tzgrid[m] = std::min(B.tztiles, per * h->num_sms);
  }
  std::vector<int> ints = unit0;
  ints.insert(ints.end(), brow.begin(), brow.end());
  ints.insert(ints.end(), bshot.begin(), bshot.end());
  ints.insert(ints.end(), zt0.begin(), zt0.end());
  LOSS_TRY(upload_table(h, 4, as_bytes(xs), &B.xptab));
  LOSS_TRY(upload_table(h, 5, as_bytes(zs), &B.tztab));
  void* t0p = B.tile0;
  LOSS_TRY(upload_table(h, 2, as_bytes(ints), &t0p));
  B.tile0 = (int*)t0p;
  return LOSS_OK;
}

template <typename T, bool K>
static loss_status_t step_batched_t(loss_ctx* h, int64_t n) {
  BatchState& B = h->batch;
  const int S = (int)h->shots.size();
  B.conv = false;
  if constexpr (sizeof(T) == 4) B.conv = conv_batch_ok(h);
  // per-shot preparation: receiver corrections, staggered start (that of the per-shot schedule of the same
  // kernels), source amplitudes
  for (Shot& s : h->shots) {
    LOSS_TRY(ensure_rdelta(h, s));
    if (!s.staggered) {
      if (B.conv) {
        LOSS_TRY((acoustic2d_start<T, K>(h, s)));
      } else {
        LOSS_TRY((ac_x<T, K>(h, s, 0, 0.5 * s.d.dt, 0.0)));
        LOSS_TRY((ac_z<T, K>(h, s, 0.5 * s.d.dt, 1)));
      }
      s.staggered = true;
    }
    LOSS_TRY(ensure_amp(h, s, s.step + n));
  }
  // launch shapes and descriptors
  std::vector<LineGeom> gx, gz;
  if (!B.conv) {
    LOSS_TRY(batch_geoms(h, 2, LOSS_KERNEL_ACOUSTIC_X, 3, 4, gx, &B.xlogc, &B.xthreads, &B.xsmem));
    LOSS_TRY(batch_geoms(h, 0, LOSS_KERNEL_ACOUSTIC_Z, 2, 0, gz, &B.zlogc, &B.zthreads, &B.zsmem));
  }
  if (B.clk_cap < S) {
    if (B.clk) dev_free(h, B.clk);
    void* p = nullptr;
    LOSS_TRY(dev_alloc(h, (size_t)S * sizeof(StepClock), &p));
    B.clk = (StepClock*)p;
    B.clk_cap = S;
    B.clk_host.clear();
  }
  std::vector<AcXArgs<T>> xa(S);
  std::vector<AcZArgs<T>> za(S);
  std::vector<int> t0(2 * (S + 1), 0);
  std::vector<GatherJob<T>> pre, post;
  int64_t pre_max = 0, post_max = 0;
  for (int i = 0; i < S; ++i) {
    Shot& s = h->shots[i];
    if (!B.conv) {
      xa[i] = ac_x_args<T>(h, s, gx[i], 1, s.d.dt, 0.0);
      xa[i].src.on = (s.src_on && (s.src_kinds & LOSS_SRC_PRESSURE)) ? 1 : 0;
      xa[i].src.amp_tab = s.amp_tab;
      xa[i].src.clk = B.clk + i;
      za[i] = ac_z_args<T>(h, s, gz[i], s.d.dt, 1);
      t0[i + 1] = t0[i] + gx[i].nbundles;
      t0[S + 1 + i + 1] = t0[S + 1 + i] + gz[i].nbundles;
    }
    for (int f = 0; f < LOSS_NUM_FIELDS; ++f) {
      if (s.n_rcv == 0) break;
      const int64_t off = s.rcv_offsets[f], cnt = s.rcv_offsets[f + 1] - off;
      if (cnt == 0) continue;
      GatherJob<T> j{};
      j.f = (const T*)s.field[f];
      j.idx = s.rcv_idx + off;
      j.cnt = cnt;
      j.trace = (T*)s.traces;
      j.n_rcv = s.n_rcv;
      j.off = off;
      j.clk = B.clk + i;
      if (is_velocity(f)) {
        j.mode = 0;
        pre.push_back(j);
        pre_max = std::max(pre_max, cnt);
        j.mode = 1;
        if (s.rdelta[0])
          for (int d = 0; d < 3; ++d) j.d[d] = (const T*)s.rdelta[3 * f + d];
      } else {
        j.mode = 0;
      }
      post.push_back(j);
      post_max = std::max(post_max, cnt);
    }
  }
  B.xtiles = t0[S];
  B.ztiles = t0[2 * S + 1];
  B.npre = (int)pre.size();
  B.npost = (int)post.size();
  B.pre_max = pre_max;
  B.post_max = post_max;
  std::vector<GatherJob<T>> jobs = pre;
  jobs.insert(jobs.end(), post.begin(), post.end());
  if (B.conv) {
    if constexpr (sizeof(T) == 4) LOSS_TRY(conv_tables<K>(h));
  } else {
    LOSS_TRY(upload_table(h, 0, as_bytes(xa), &B.xtab));
    LOSS_TRY(upload_table(h, 1, as_bytes(za), &B.ztab));
    void* t0p = B.tile0;
    LOSS_TRY(upload_table(h, 2, as_bytes(t0), &t0p));
    B.tile0 = (int*)t0p;
  }
  LOSS_TRY(upload_table(h, 3, as_bytes(jobs), &B.jobs));
  // device clocks: set from the host counters unless they already hold them
  std::vector<StepClock> ck(S);
  for (int i = 0; i < S; ++i)
    ck[i] = StepClock{h->shots[i].step, h->shots[i].rcv_steps, h->shots[i].n_rcv ? 1 : 0, 0};
  std::vector<unsigned char> ckb = as_bytes(ck);
  if (ckb != B.clk_host) {
    LOSS_TRY(cuda_check(h, cudaMemcpyAsync(B.clk, ckb.data(), ckb.size(), cudaMemcpyHostToDevice, h->stream),
                        "upload clocks"));
    LOSS_TRY(cuda_check(h, cudaStreamSynchronize(h->stream), "sync"));
  }
  if (!B.conv) {
    LOSS_TRY(cuda_check(h, batch_grid_ac_x<T, K>(B.xlogc, B.xthreads, B.xsmem, B.xtiles, h->num_sms, &B.xgrid),
                        "batched x kernel shape"));
    LOSS_TRY(cuda_check(h, batch_grid_ac_z<T, K>(B.zlogc, B.zthreads, B.zsmem, B.ztiles, h->num_sms, &B.zgrid),
                        "batched z kernel shape"));
  }
  // launches
  int64_t done = 0;
  const int64_t k = h->graph_steps;
  if (k > 0 && n >= k) {
    const std::vector<int64_t> sig = {B.xthreads, (int64_t)B.xsmem, B.xlogc, B.xtiles, B.xgrid, B.zthreads,
                                      (int64_t)B.zsmem, B.zlogc, B.ztiles, B.zgrid, B.npre, B.npost, B.pre_max,
                                      B.post_max, (int64_t)(intptr_t)B.xtab, (int64_t)(intptr_t)B.ztab,
                                      (int64_t)(intptr_t)B.tile0, (int64_t)(intptr_t)B.jobs,
                                      (int64_t)(intptr_t)B.clk, S, (int64_t)sizeof(T), K ? 1 : 0, k, B.conv ? 1 : 0,
                                      (int64_t)(intptr_t)B.xptab, (int64_t)(intptr_t)B.tztab, B.xpgrid, B.xpthreads,
                                      B.xl.total, B.tzthreads[0], B.tzthreads[1], B.tzlogc[0], B.tzlogc[1],
                                      B.tztiles, B.tzgrid[0], B.tzgrid[1],
                                      (int64_t)B.tzsmem[0], (int64_t)B.tzsmem[1], (int64_t)h->wait_polls};
    if (!B.gexec || sig != B.gsig) {
      LOSS_TRY((capture_graph<T, K>(h, k)));
      B.gsig = sig;
    }
    for (; n - done >= k; done += k) {
      LOSS_TRY(cuda_check(h, cudaGraphLaunch(B.gexec, h->stream), "graph launch"));
      for (int i = 0; i < LOSS_NUM_KERNELS; ++i) h->launches[i] += B.graph_launches[i];
    }
  }
  for (; done < n; ++done) LOSS_TRY((batch_launch_step<T, K>(h)));
  for (int i = 0; i < S; ++i) {
    Shot& s = h->shots[i];
    s.step += n;
    if (s.n_rcv) s.rcv_steps += n;
    ck[i] = StepClock{s.step, s.rcv_steps, s.n_rcv ? 1 : 0, 0};
  }
  B.clk_host = as_bytes(ck);
  return LOSS_OK;
}

loss_status_t step_batched(loss_ctx* h, int64_t n) {
  if (n <= 0) return LOSS_OK;
  const Shot& s = h->shots[0];
  if (s.esize == 8) return step_batched_t<double, false>(h, n);
  if (s.kahan) return step_batched_t<float, true>(h, n);
  return step_batched_t<float, false>(h, n);
}

loss_status_t step_shot(loss_ctx* h, Shot& s) {
  if (any_nonuniform(s)) {
    LOSS_TRY(nu_step(h, s));
    // receivers at the integer time level (the non-uniform step keeps no staggered velocities)
    if (s.esize == 8) {
      LOSS_TRY(gather_fields<double>(h, s, true, 0));
      LOSS_TRY(gather_fields<double>(h, s, false, 0));
    } else {
      LOSS_TRY(gather_fields<float>(h, s, true, 0));
      LOSS_TRY(gather_fields<float>(h, s, false, 0));
    }
    if (s.n_rcv) ++s.rcv_steps;
    ++s.step;
    return LOSS_OK;
  }
  if (s.d.physics == LOSS_ACOUSTIC && s.dim == 2) {
    if (s.esize == 8) return acoustic2d_step<double, false>(h, s);
    if (s.kahan) return acoustic2d_step<float, true>(h, s);
    return acoustic2d_step<float, false>(h, s);
  }
  if (s.d.physics == LOSS_ELASTIC) {
    if (s.esize == 8) return elastic3d_step<double, false>(h, s);
    if (s.kahan) return elastic3d_step<float, true>(h, s);
    return elastic3d_step<float, false>(h, s);
  }
  h->err = "time stepping of this physics/dimension is not built";
  return LOSS_E_UNSUPPORTED;
}

// The staggered start (half velocity sub-step) on its own.
loss_status_t stagger_shot(loss_ctx* h, Shot& s) {
  if (s.staggered) return LOSS_OK;
  LOSS_TRY(ensure_rdelta(h, s));
  const double dt = s.d.dt;
  if (s.d.physics == LOSS_ACOUSTIC && s.dim == 2) {
    if (s.esize == 8) LOSS_TRY((acoustic2d_start<double, false>(h, s)));
    else if (s.kahan) LOSS_TRY((acoustic2d_start<float, true>(h, s)));
    else LOSS_TRY((acoustic2d_start<float, false>(h, s)));
  } else if (s.d.physics == LOSS_ELASTIC) {
    const double tn = (double)s.step * dt;
    if (s.esize == 8) LOSS_TRY((elastic_A<double, false>(h, s, 0.5 * dt, tn)));
    else if (s.kahan) LOSS_TRY((elastic_A<float, true>(h, s, 0.5 * dt, tn)));
    else LOSS_TRY((elastic_A<float, false>(h, s, 0.5 * dt, tn)));
  } else {
    h->err = "time stepping of this physics/dimension is not built";
    return LOSS_E_UNSUPPORTED;
  }
  s.staggered = true;
  return LOSS_OK;
}

loss_status_t unstagger(loss_ctx* h, Shot& s) {
  if (!s.staggered) return LOSS_OK;
  if (s.d.physics == LOSS_ACOUSTIC && s.dim == 2) {
    if (s.esize == 8) return acoustic2d_unstagger<double, false>(h, s);
    if (s.kahan) return acoustic2d_unstagger<float, true>(h, s);
    return acoustic2d_unstagger<float, false>(h, s);
  }
  if (s.d.physics == LOSS_ELASTIC) {
    if (s.esize == 8) return elastic3d_unstagger<double, false>(h, s);
    if (s.kahan) return elastic3d_unstagger<float, true>(h, s);
    return elastic3d_unstagger<float, false>(h, s);
  }
  return LOSS_E_UNSUPPORTED;
}

}  // namespace lossk
