// Time-stepping schedule (paper Sec. 3.3): Strang splitting "half A, full B, half A" with the velocity
// sub-step A and the stress sub-step B.  Between steps the velocities are kept half a step ahead (staggered),
// which merges the trailing half A of one step with the leading half A of the next; the state is brought back
// to the integer time level (v_n = v_{n+1/2} + dt/2 b grad sigma_n) whenever velocities are read.
#include <cmath>

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

template <typename T, bool K>
static loss_status_t ac_x(loss_ctx* h, Shot& s, int do_B, double acoef, double src_amp) {
  LineGeom g;
  int logc, threads;
  LOSS_TRY(line_geom(h, s, 2, s.sz, s.sy, &g, &logc, &threads, 3, 4, h->lines_per_block[LOSS_KERNEL_ACOUSTIC_X],
                     h->chunk_log2[LOSS_KERNEL_ACOUSTIC_X]));
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
  LaunchScope ls(h, LOSS_KERNEL_ACOUSTIC_X);
  return cuda_check(h, launch_ac_x<T, K>(a, logc, threads, h->stream), "acoustic x kernel");
}

template <typename T, bool K>
static loss_status_t ac_z(loss_ctx* h, Shot& s, double acoef, int do_tmp) {
  LineGeom g;
  int logc, threads;
  LOSS_TRY(line_geom(h, s, 0, s.sz, s.sy, &g, &logc, &threads, 2, 0, h->lines_per_block[LOSS_KERNEL_ACOUSTIC_Z],
                     h->chunk_log2[LOSS_KERNEL_ACOUSTIC_Z]));
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
  a.minf = (T)(2.0 - std::sqrt(3.0));
  a.do_tmp = do_tmp;
  a.pml = s.pml_on ? 1 : 0;
  if (s.pml_on) {
    a.zA = pml_axis<T>(s, 0, acoef);
    a.psiz = (T*)s.psi[0];
    a.dlt = rdelta<T>(s, 2, 2, acoef);
  }
  LaunchScope ls(h, LOSS_KERNEL_ACOUSTIC_Z);
  return cuda_check(h, launch_ac_z<T, K>(a, logc, threads, h->stream), "acoustic z kernel");
}

template <typename T>
static loss_status_t gather_fields(loss_ctx* h, Shot& s, bool velocities, int mode) {
  if (s.n_rcv == 0) return LOSS_OK;
  T* row = (T*)s.traces + (size_t)s.rcv_steps * s.n_rcv;
  for (int f = 0; f < LOSS_NUM_FIELDS; ++f) {
    const int64_t off = s.rcv_offsets[f], cnt = s.rcv_offsets[f + 1] - off;
    if (cnt == 0 || is_velocity(f) != velocities) continue;
    LaunchScope ls(h, LOSS_KERNEL_GATHER);
    const T* d[3] = {nullptr, nullptr, nullptr};
    if (mode == 1 && s.rdelta[0])
      for (int j = 0; j < 3; ++j) d[j] = (const T*)s.rdelta[3 * f + j];
    LOSS_TRY(cuda_check(h, launch_gather<T>((const T*)s.field[f], s.rcv_idx + off, cnt, row + off, mode, d[0], d[1],
                                            d[2], h->stream),
                        "receiver gather"));
  }
  return LOSS_OK;
}

template <typename T, bool K>
static loss_status_t acoustic2d_step(loss_ctx* h, Shot& s) {
  const double dt = s.d.dt;
  LOSS_TRY(ensure_rdelta(h, s));
  if (!s.staggered) {
    LOSS_TRY((ac_x<T, K>(h, s, 0, 0.5 * dt, 0.0)));
    LOSS_TRY((ac_z<T, K>(h, s, 0.5 * dt, 1)));
    s.staggered = true;
  }
  LOSS_TRY(gather_fields<T>(h, s, true, 0));  // v at t_{n+1/2}
  double amp = 0.0;
  if (s.src_on && (s.src_kinds & LOSS_SRC_PRESSURE))
    amp = dt * s.src_norm * ricker((double)s.step * dt + 0.5 * dt, s.src_f0, s.src_t0);
  LOSS_TRY((ac_x<T, K>(h, s, 1, dt, amp)));
  LOSS_TRY((ac_z<T, K>(h, s, dt, 1)));
  LOSS_TRY(gather_fields<T>(h, s, true, 1));   // (v_{n+1/2} + v_{n+3/2}) / 2 = v_{n+1}
  LOSS_TRY(gather_fields<T>(h, s, false, 0));  // sigma_{n+1}
  if (s.n_rcv) ++s.rcv_steps;
  ++s.step;
  return LOSS_OK;
}

template <typename T, bool K>
static loss_status_t acoustic2d_unstagger(loss_ctx* h, Shot& s) {
  const double dt = s.d.dt;
  LOSS_TRY((ac_x<T, K>(h, s, 0, -0.5 * dt, 0.0)));
  LOSS_TRY((ac_z<T, K>(h, s, -0.5 * dt, 0)));
  s.staggered = false;
  return LOSS_OK;
}


// ---------------------------------------------------------------------------------------------------------------
// 3-D elastic: five line passes per step (loss_kernels_elastic.cu).
enum { EL_BX = 0, EL_BY = 1, EL_BZ = 2, EL_AX = 3, EL_AY = 4 };

template <typename T, bool K>
static loss_status_t el_pass(loss_ctx* h, Shot& s, int pass, int do_B, int do_A, double acoef, double amp) {
  // internal axis slot of the pass: x = 2, y = 1, z = 0
  const int k = (pass == EL_BX || pass == EL_AX) ? 2 : ((pass == EL_BY || pass == EL_AY) ? 1 : 0);
  LineGeom g;
  int logc, threads;
  const int kid = (k == 2) ? LOSS_KERNEL_ELASTIC_X : (k == 1 ? LOSS_KERNEL_ELASTIC_Y : LOSS_KERNEL_ELASTIC_Z);
  LOSS_TRY(line_geom(h, s, k, s.sz, s.sy, &g, &logc, &threads, 6, 0, h->lines_per_block[kid], h->chunk_log2[kid]));
  ElArgs<T> a{};
  a.g = g;
  a.tb = Tables{s.W[k], h->t32, h->t64};
  int srcf[3];
  switch (pass) {
    case EL_BX:
    case EL_BY: srcf[0] = LOSS_FIELD_V1, srcf[1] = LOSS_FIELD_V2, srcf[2] = LOSS_FIELD_V3; break;
    case EL_BZ:
      if (do_B) srcf[0] = LOSS_FIELD_V1, srcf[1] = LOSS_FIELD_V2, srcf[2] = LOSS_FIELD_V3;
      else srcf[0] = LOSS_FIELD_S13, srcf[1] = LOSS_FIELD_S23, srcf[2] = LOSS_FIELD_S33;
      break;
    case EL_AX: srcf[0] = LOSS_FIELD_S11, srcf[1] = LOSS_FIELD_S12, srcf[2] = LOSS_FIELD_S13; break;
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
  LaunchScope ls(h, kid);
  return cuda_check(h, launch_el<T, K>(a, pass, logc, threads, h->stream), "elastic kernel");
}

// Velocity sub-step of length tau on the current stresses (three passes); force_t = time of the body force.
template <typename T, bool K>
static loss_status_t elastic_A(loss_ctx* h, Shot& s, double tau, double force_t) {
  double famp = 0.0;
  if (s.src_on && (s.src_kinds & LOSS_SRC_FORCE_Z)) famp = tau * s.src_norm * ricker(force_t, s.src_f0, s.src_t0);
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
  if (s.src_on && (s.src_kinds & LOSS_SRC_FORCE_Z)) famp = dt * s.src_norm * ricker(tn + dt, s.src_f0, s.src_t0);
  LOSS_TRY((el_pass<T, K>(h, s, EL_BX, 1, 0, dt, 0.0)));
  LOSS_TRY((el_pass<T, K>(h, s, EL_BY, 1, 0, dt, 0.0)));
  LOSS_TRY((el_pass<T, K>(h, s, EL_BZ, 1, 1, dt, amp)));
  LOSS_TRY((el_pass<T, K>(h, s, EL_AX, 0, 1, dt, 0.0)));
  LOSS_TRY((el_pass<T, K>(h, s, EL_AY, 0, 1, dt, famp)));
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

loss_status_t step_shot(loss_ctx* h, Shot& s) {
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
