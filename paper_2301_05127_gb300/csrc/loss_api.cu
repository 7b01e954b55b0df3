// Host runtime behind include/loss.h: handle and memory management, PMBC weight tables, launch geometry,
// and the time-stepping schedule.  Every entry point is extern "C", returns a status and never throws.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <new>
#include <string>
#include <vector>

#include "../../include/loss.h"
#include "loss_host.h"

namespace lossk {

// ----------------------------------------------------------------------------------------------------------------
// PMBC weights.  With the natural end rows of Eq. (spline_cofficient_eq), (c_{-1} - 2 c_0 + c_1)/h^2 = 0 and the
// collocation row at x_0 give c_0 = f_0 and c_{-1} = 2 c_0 - c_1 (likewise c_N = f_N, c_{N+1} = 2 c_N - c_{N-1}),
// so the interior coefficients solve the (N-1)x(N-1) system T c = f - (f_0/6) e_1 - (f_N/6) e_{N-1} with
// T = tridiag(1, 4, 1)/6.  Row k of b = A^{-1} restricted to the data columns is then z_k (T z_k = e_k, T is
// symmetric) on the interior columns and -z_k[1]/6, -z_k[N-1]/6 on columns 0 and N.  The PMBC weights of
// junction lM are (b_{lM+1, .} - b_{lM-1, .}) / (2h) (Eq. PMBC_coeffcients, end closures of Sec. 3.2); they
// are stored multiplied by h/3 because the kernels solve for e = d h / 3.
static std::vector<double> coef_row(int n, int k) {
  std::vector<double> row(n + 1, 0.0);
  if (k == 0 || k == n) {
    row[k] = 1.0;
    return row;
  }
  // Solve tridiag(1,4,1) z = 6 e_k on unknowns 1..n-1 (Thomas, exact factors).
  const int m = n - 1;
  std::vector<double> u(m + 1), y(m + 1), z(m + 2, 0.0);
  for (int i = 1; i <= m; ++i) {
    const double rhs = (i == k) ? 6.0 : 0.0;
    if (i == 1) {
      u[i] = 4.0;
      y[i] = rhs;
    } else {
      u[i] = 4.0 - 1.0 / u[i - 1];
      y[i] = rhs - y[i - 1] / u[i - 1];
    }
  }
  for (int i = m; i >= 1; --i) z[i] = (y[i] - (i < m ? z[i + 1] : 0.0)) / u[i];
  for (int i = 1; i <= m; ++i) row[i] = z[i];
  row[0] = -z[1] / 6.0;
  row[n] = -z[m] / 6.0;
  return row;
}

// Row of the coefficient index k in -1..n+1.
static std::vector<double> coef_row_ext(int n, int k) {
  if (k == -1 || k == n + 1) {
    const int e = (k == -1) ? 0 : n;
    std::vector<double> r = coef_row(n, (k == -1) ? 1 : n - 1);
    for (double& v : r) v = -v;
    r[e] += 2.0;
    return r;
  }
  return coef_row(n, k);
}

std::vector<double> pmbc_weights_scaled(int n, int p, int n_nb) {
  const int M = n / p;
  const int wl = 2 * n_nb + 1;
  std::vector<double> W((size_t)(p + 1) * wl, 0.0);
  for (int j = 0; j <= p; ++j) {
    const int c = j * M;
    const std::vector<double> rp = coef_row_ext(n, c + 1);
    const std::vector<double> rm = coef_row_ext(n, c - 1);
    const int mlo = (j == 0) ? 0 : -n_nb;
    const int mhi = (j == p) ? 0 : n_nb;
    for (int m = mlo; m <= mhi; ++m) {
      const int col = c + m;
      if (col < 0 || col > n) continue;
      // (b_{c+1,col} - b_{c-1,col}) / (2h) * (h/3)
      W[(size_t)j * wl + (m + n_nb)] = (rp[col] - rm[col]) / 6.0;
    }
  }
  return W;
}

// Junction-correction weights of the truncated-convolution form (loss_fir.cuh): D_j = phi_j - eF_j as weights on
// the field at positions jM + m, |m| <= R = max(n_nb, K): the PMBC weights (scaled by h/3) minus the weights of
// eF_j = a sum_{k=1..K} r^{k-1} (f_{c+k} - f_{c-k}) with the line continued by odd reflection beyond its ends
// (f_{-q} = 2 f_0 - f_q, f_{n+q} = 2 f_n - f_{n-q}, q clamped to the line).  Formed in FP64; away from the
// physical ends the two weight sets agree to O(r^K), so the FP32 sum of D f carries no cancellation.
std::vector<double> fir_delta_weights(int n, int p, int n_nb, int K) {
  const std::vector<double> W = pmbc_weights_scaled(n, p, n_nb);
  const int M = n / p;
  const int R = std::max(n_nb, K);
  const int wl = 2 * R + 1;
  const double r = std::sqrt(3.0) - 2.0;
  const double a = (1.0 - r * r) / (2.0 * std::sqrt(3.0));
  std::vector<double> D((size_t)(p + 1) * wl, 0.0);
  for (int j = 0; j <= p; ++j) {
    const int c = j * M;
    double* Dj = D.data() + (size_t)j * wl + R;  // Dj[m], m = -R..R
    for (int m = -n_nb; m <= n_nb; ++m)
      if (c + m >= 0 && c + m <= n) Dj[m] += W[(size_t)j * (2 * n_nb + 1) + (m + n_nb)];
    auto add = [&](int pos, double w) {
      if (pos >= 0 && pos <= n) {
        Dj[pos - c] += w;
      } else if (pos < 0) {
        const int q = std::min(-pos, n);
        Dj[0 - c] += 2.0 * w;
        Dj[q - c] -= w;
      } else {
        const int q = std::max(n - (pos - n), 0);
        Dj[n - c] += 2.0 * w;
        Dj[q - c] -= w;
      }
    };
    double rk = 1.0;
    for (int k = 1; k <= K; ++k) {
      add(c + k, -a * rk);
      add(c - k, a * rk);
      rk *= r;
    }
  }
  return D;
}

void thomas_tables(std::vector<double>& t64, std::vector<float>& t32) {
  t64.assign(kTableLen, 0.0);
  t32.assign(kTableLen, 0.0f);
  t64[0] = 1.0;
  double u = 4.0;
  for (int j = 1; j < kTableLen; ++j) {
    t64[j] = 1.0 / u;
    u = 4.0 - t64[j];
  }
  for (int j = 0; j < kTableLen; ++j) t32[j] = (float)t64[j];
}

// ----------------------------------------------------------------------------------------------------------------
// Error plumbing.
#define LOSS_TRY(expr)                      \
  do {                                      \
    loss_status_t st_ = (expr);             \
    if (st_ != LOSS_OK) return st_;         \
  } while (0)

static loss_status_t fail(loss_ctx* h, loss_status_t st, const std::string& msg) {
  if (h) {
    h->err = msg;
    if (st == LOSS_E_CUDA || st == LOSS_E_TIMEOUT) h->sticky = st;
  }
  return st;
}

loss_status_t cuda_check(loss_ctx* h, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return LOSS_OK;
  return fail(h, LOSS_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

static loss_status_t guard(loss_ctx* h) {
  if (!h) return LOSS_E_ARG;
  if (h->sticky != LOSS_OK) return h->sticky;
  return LOSS_OK;
}

// ----------------------------------------------------------------------------------------------------------------
// Device memory.
loss_status_t dev_alloc(loss_ctx* h, size_t bytes, void** out) {
  *out = nullptr;
  if (bytes == 0) return LOSS_OK;
  void* p = nullptr;
  if (h->has_alloc) {
    p = h->alloc.alloc(h->alloc.ctx, bytes, (void*)h->stream);
    if (!p) return fail(h, LOSS_E_NOMEM, "allocator callback failed for " + std::to_string(bytes) + " bytes");
  } else {
    cudaError_t e = cudaMallocAsync(&p, bytes, h->stream);
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      return fail(h, LOSS_E_NOMEM, "cudaMallocAsync failed for " + std::to_string(bytes) + " bytes");
    }
    LOSS_TRY(cuda_check(h, e, "cudaMallocAsync"));
  }
  h->owned.push_back(p);
  *out = p;
  return LOSS_OK;
}

void dev_free(loss_ctx* h, void* p) {
  if (!p) return;
  auto it = std::find(h->owned.begin(), h->owned.end(), p);
  if (it != h->owned.end()) h->owned.erase(it);
  if (h->has_alloc)
    h->alloc.free(h->alloc.ctx, p, (void*)h->stream);
  else
    cudaFreeAsync(p, h->stream);
}

static loss_status_t dev_zero_alloc(loss_ctx* h, size_t bytes, void** out) {
  LOSS_TRY(dev_alloc(h, bytes, out));
  if (bytes) LOSS_TRY(cuda_check(h, cudaMemsetAsync(*out, 0, bytes, h->stream), "cudaMemsetAsync"));
  return LOSS_OK;
}

// ----------------------------------------------------------------------------------------------------------------
// Geometry.
static int axis_slot(const Shot& s, int axis) {
  // public axis index -> internal slot (0 = z, 1 = y, 2 = x)
  if (s.dim == 3) return axis;
  return axis == 0 ? 0 : 2;
}

// Build the launch geometry of lines along internal slot `k` for an array with strides (sz, sy, 1).
// nbuf padded line buffers and nstage dense row-staging buffers (X flavour) per block; want_L > 0 requests a
// bundle width (lines per block); otherwise want_threads > 0 requests the widest power-of-two bundle whose chunks
// fit in that many threads.
loss_status_t line_geom(loss_ctx* h, const Shot& s, int k, int64_t sz, int64_t sy, LineGeom* g, int* logc,
                        int* threads, int nbuf, int nstage, int want_L, int want_logc, int want_threads) {
  const int n = (int)s.n[k];
  const int p = s.p[k];
  const int M = n / p;
  LineGeom G{};
  G.n = n;
  G.p = p;
  G.M = M;
  // Chunk length: 8 for FP32 lines along x (more threads per line, shorter serial chains), else 16 (the
  // Thomas factors reach their limit to double rounding within 16 positions).
  *logc = (k == 2 && s.esize == 4) ? 3 : 4;
  if (want_logc >= 3 && want_logc <= 4 && !(s.esize == 8 && want_logc == 3)) *logc = want_logc;
  const int C = 1 << *logc;
  G.NC = (M - 1 + C - 1) / C;
  G.n_nb = s.d.n_nb;
  G.mmagic = (unsigned)((((uint64_t)1 << 32) + (uint64_t)M - 1) / (uint64_t)M);
  const int per_line = p * G.NC;
  const size_t es = s.esize;
  const size_t smax = (size_t)h->smem_optin - 4096;  // headroom for the kernels' static shared memory
  if (want_L <= 0 && want_threads > 0) {
    want_L = 1;
    while (want_L < 32 && 2 * want_L * per_line <= want_threads) want_L *= 2;
  }
  const int np_pad = (n + (n >> *logc)) + 1;  // padpos(n) + 1
  const int vec = (int)(16 / es);
  G.spitch = ((n + 1 + vec - 1) / vec) * vec;
  if (k == 2) {
    // X flavour: rows of the flattened (z, y) index.
    int L = 1;
    while (L < 32 && 2 * L * per_line <= 256) L *= 2;
    if (want_L > 0 && want_L <= 32 && want_L * per_line <= (es == 8 ? 512 : 1024)) L = want_L;
    while (true) {
      int pitch = np_pad;
      const int want = per_line % 32;
      if (per_line < 32) {
        while ((pitch & 31) != want) ++pitch;
      }
      G.L = L;
      G.pitch = pitch;
      G.buf = L * pitch;
      G.stage = nstage ? L * G.spitch : 0;
      if (smem_bytes(G, nbuf, nstage, es) <= smax || L == 1) break;
      L = std::max(1, L / 2);
    }
    G.ny1 = (int)s.len[1];
    G.sz = sz;
    G.sy = sy;
    G.nrows = s.len[0] * s.len[1];
    G.nbundles = (int)((G.nrows + G.L - 1) / G.L);
    G.pstride = 1;
  } else {
    // S flavour: bundles of neighbouring x lines (nstage must be 0).
    int L = (want_L > 0 && want_L <= 32) ? want_L : (es == 8 ? 4 : 8);
    while (L > 1) {
      G.L = L;
      G.pitch = L;
      G.buf = np_pad * L;
      G.stage = 0;
      if (smem_bytes(G, nbuf, 0, es) <= smax && L * per_line <= (es == 8 ? 512 : 1024)) break;
      L /= 2;
    }
    G.L = L;
    G.pitch = L;
    G.buf = np_pad * L;
    G.stage = 0;
    G.nx1 = (int)s.len[2];
    G.nxb = (G.nx1 + L - 1) / L;
    if (k == 0) {
      G.so = sy;  // outer = y
      G.pstride = sz;
      G.nbundles = (int)(s.len[1] * G.nxb);
    } else {
      G.so = sz;  // outer = z
      G.pstride = sy;
      G.nbundles = (int)(s.len[0] * G.nxb);
    }
  }
  if (smem_bytes(G, nbuf, nstage, es) > smax)
    return fail(h, LOSS_E_UNSUPPORTED,
                "grid line of " + std::to_string(n + 1) + " points does not fit in shared memory");
  const int work = G.L * per_line;
  const int max_threads = (es == 8) ? 512 : 1024;
  if (work > max_threads)
    return fail(h, LOSS_E_UNSUPPORTED, "grid line of " + std::to_string(n + 1) + " points needs more than 1024 chunks");
  *threads = ((work + 31) / 32) * 32;
  *g = G;
  return LOSS_OK;
}

// ----------------------------------------------------------------------------------------------------------------
// Source profile: g[o] = exp(-o^2/8), o = -12..12, amplitude normalised by the in-grid sum and the cell volume.
static void source_setup(Shot& s) {
  for (int o = -12; o <= 12; ++o) s.src_g[o + 12] = std::exp(-(double)o * o / 8.0);
  double sum = 1.0, cell = 1.0;
  const int slots[3] = {0, 1, 2};
  for (int a = 0; a < 3; ++a) {
    const int k = slots[a];
    if (s.dim == 2 && k == 1) continue;
    double ax = 0.0;
    for (int o = -12; o <= 12; ++o) {
      const int64_t q = s.src_idx[k] + o;
      if (q >= 0 && q <= s.n[k]) ax += s.src_g[o + 12];
    }
    sum *= ax;
    cell *= s.h[k];
  }
  s.src_norm = s.src_amp / (sum * cell);
}


// ----------------------------------------------------------------------------------------------------------------
// Shot setup.
loss_status_t validate(const loss_grid_desc_t& d, std::string* why) {
  if (d.dim != 2 && d.dim != 3) return *why = "dim must be 2 or 3", LOSS_E_SHAPE;
  if (d.physics != LOSS_ACOUSTIC && d.physics != LOSS_ELASTIC) return *why = "unknown physics", LOSS_E_ARG;
  if (d.precision != LOSS_FP64 && d.precision != LOSS_FP32 && d.precision != LOSS_FP32_KAHAN)
    return *why = "unknown precision", LOSS_E_ARG;
  if (d.physics == LOSS_ELASTIC && d.dim != 3) return *why = "elastic grids must be 3-D", LOSS_E_SHAPE;
  if (d.n_nb < 1) return *why = "n_nb must be >= 1", LOSS_E_SHAPE;
  if (!(d.dt > 0.0)) return *why = "dt must be > 0", LOSS_E_SHAPE;
  const int axes[3] = {0, d.dim == 3 ? 1 : -1, d.dim == 3 ? 2 : 1};
  for (int a = 0; a < 3; ++a) {
    const int i = axes[a];
    if (i < 0) continue;
    if (d.n[i] < 2 || d.p[i] < 1 || d.n[i] % d.p[i] != 0)
      return *why = "axis " + std::to_string(i) + ": n must be >= 2 and a multiple of p", LOSS_E_SHAPE;
    const int64_t M = d.n[i] / d.p[i];
    if (M < 2 || d.n_nb > M) return *why = "axis " + std::to_string(i) + ": need M >= 2 and n_nb <= M", LOSS_E_SHAPE;
    if (!(d.h[i] > 0.0)) return *why = "h must be > 0", LOSS_E_SHAPE;
    if (d.n[i] > (1 << 20)) return *why = "axis too long", LOSS_E_SHAPE;
  }
  return LOSS_OK;
}

void shot_geometry(Shot& s) {
  const loss_grid_desc_t& d = s.d;
  s.dim = d.dim;
  // internal slots: 0 = z, 1 = y, 2 = x
  if (d.dim == 3) {
    for (int a = 0; a < 3; ++a) {
      s.n[a] = d.n[a];
      s.p[a] = d.p[a];
      s.h[a] = d.h[a];
    }
  } else {
    s.n[0] = d.n[0];
    s.p[0] = d.p[0];
    s.h[0] = d.h[0];
    s.n[1] = 0;
    s.p[1] = 1;
    s.h[1] = 1.0;
    s.n[2] = d.n[1];
    s.p[2] = d.p[1];
    s.h[2] = d.h[1];
  }
  for (int a = 0; a < 3; ++a) s.len[a] = s.n[a] + 1;
  s.esize = d.precision == LOSS_FP64 ? 8 : 4;
  s.kahan = d.precision == LOSS_FP32_KAHAN;
  s.px = ((s.len[2] + 31) / 32) * 32;
  s.sy = s.px;
  s.sz = s.px * s.len[1];
  s.total = s.sz * s.len[0];
  s.dense = s.len[0] * s.len[1] * s.len[2];
}

static loss_status_t setup_shot(loss_ctx* h, Shot& s) {
  const loss_grid_desc_t& d = s.d;
  shot_geometry(s);
  const size_t fb = (size_t)s.total * s.esize;
  s.nfields = d.physics == LOSS_ELASTIC ? 9 : 4;  // acoustic uses V1, V2 (3-D), V3, SIGMA(=3)
  for (int f = 0; f < LOSS_NUM_FIELDS; ++f) {
    if (!field_used(s, f)) continue;
    LOSS_TRY(dev_zero_alloc(h, fb, &s.field[f]));
    if (s.kahan) LOSS_TRY(dev_zero_alloc(h, fb, &s.comp[f]));
  }
  const int nmodel = d.physics == LOSS_ELASTIC ? 3 : 2;
  for (int m = 0; m < nmodel; ++m) LOSS_TRY(dev_zero_alloc(h, fb, &s.model[m]));
  const int ntmp = d.physics == LOSS_ELASTIC ? 8 : 1;
  for (int i = 0; i < ntmp; ++i) LOSS_TRY(dev_zero_alloc(h, fb, &s.tmp[i]));
  // PMBC tables per used axis.
  for (int k = 0; k < 3; ++k) {
    if (s.dim == 2 && k == 1) continue;
    std::vector<double> W = pmbc_weights_scaled((int)s.n[k], s.p[k], d.n_nb);
    LOSS_TRY(dev_alloc(h, W.size() * sizeof(double), (void**)&s.W[k]));
    LOSS_TRY(cuda_check(h, cudaMemcpyAsync(s.W[k], W.data(), W.size() * sizeof(double), cudaMemcpyHostToDevice,
                                           h->stream), "copy W"));
    LOSS_TRY(cuda_check(h, cudaStreamSynchronize(h->stream), "sync"));
  }
  return LOSS_OK;
}

bool field_used(const Shot& s, int f) {
  if (s.d.physics == LOSS_ELASTIC) return f >= 0 && f < 9;
  if (f == LOSS_FIELD_SIGMA || f == LOSS_FIELD_V1 || f == LOSS_FIELD_V3) return true;
  return f == LOSS_FIELD_V2 && s.dim == 3;
}

// ----------------------------------------------------------------------------------------------------------------
// Copies between dense caller arrays and the padded device layout.
static loss_status_t copy_in(loss_ctx* h, const Shot& s, void* dst, const void* src, int mem) {
  const size_t w = (size_t)s.len[2] * s.esize;
  return cuda_check(h, cudaMemcpy2DAsync(dst, (size_t)s.px * s.esize, src, w, w, (size_t)(s.len[0] * s.len[1]),
                                         mem == LOSS_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                         h->stream),
                    "copy in");
}

// Device address of a pinned host array that kernels may read and write directly, or null (pageable memory).
static void* mapped_host(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// Host upload of a field: the pitch kernel reads a mapped pinned host array directly and spreads it into the
// padded rows; pageable arrays take the 2-D copy.
static loss_status_t upload_field(loss_ctx* h, const Shot& s, void* dst, const void* src, int mem) {
  if (mem != LOSS_MEM_HOST) return copy_in(h, s, dst, src, mem);
  const void* msrc = mapped_host(src);
  if (msrc)
    return cuda_check(h, launch_pitch_in(msrc, dst, s.len[0] * s.len[1], s.len[2], s.px, s.esize, h->num_sms,
                                         h->stream), "pitch kernel");
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, src) != cudaSuccess) {
    cudaGetLastError();
    return copy_in(h, s, dst, src, mem);
  }
  if (at.type != cudaMemoryTypeHost) return copy_in(h, s, dst, src, mem);
  const size_t bytes = (size_t)s.dense * s.esize;
  if (h->stage_bytes < bytes) {
    if (h->stage) dev_free(h, h->stage);
    h->stage = nullptr;
    h->stage_bytes = 0;
    LOSS_TRY(dev_alloc(h, bytes, &h->stage));
    h->stage_bytes = bytes;
  }
  LOSS_TRY(cuda_check(h, cudaMemcpyAsync(h->stage, src, bytes, cudaMemcpyHostToDevice, h->stream), "copy in"));
  return cuda_check(h, launch_pitch_in(h->stage, dst, s.len[0] * s.len[1], s.len[2], s.px, s.esize, h->num_sms,
                                       h->stream), "pitch kernel");
}

static loss_status_t copy_out(loss_ctx* h, const Shot& s, void* dst, const void* src, int mem) {
  if (mem == LOSS_MEM_HOST) {
    void* mdst = mapped_host(dst);
    if (mdst)
      return cuda_check(h, launch_pitch_out(src, mdst, s.len[0] * s.len[1], s.len[2], s.px, s.esize, h->num_sms,
                                            h->stream), "pitch kernel");
  }
  const size_t w = (size_t)s.len[2] * s.esize;
  return cuda_check(h, cudaMemcpy2DAsync(dst, w, src, (size_t)s.px * s.esize, w, (size_t)(s.len[0] * s.len[1]),
                                         mem == LOSS_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                                         h->stream),
                    "copy out");
}

static void drop_events(loss_ctx* h) {
  for (auto& e : h->events) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  h->events.clear();
}

}  // namespace lossk

using namespace lossk;

// ----------------------------------------------------------------------------------------------------------------
// C ABI.
extern "C" {

const char* loss_version(void) { return "loss-gb300 0.1 (sm_103a)"; }

const char* loss_status_str(loss_status_t st) {
  switch (st) {
    case LOSS_OK: return "LOSS_OK";
    case LOSS_E_ARG: return "LOSS_E_ARG";
    case LOSS_E_SHAPE: return "LOSS_E_SHAPE";
    case LOSS_E_NOMEM: return "LOSS_E_NOMEM";
    case LOSS_E_CUDA: return "LOSS_E_CUDA";
    case LOSS_E_STATE: return "LOSS_E_STATE";
    case LOSS_E_TIMEOUT: return "LOSS_E_TIMEOUT";
    case LOSS_E_NUMERIC: return "LOSS_E_NUMERIC";
    case LOSS_E_UNSUPPORTED: return "LOSS_E_UNSUPPORTED";
  }
  return "LOSS_E_UNKNOWN";
}

const char* loss_last_error(loss_handle_t h) { return h ? h->err.c_str() : "null handle"; }

loss_status_t loss_create_grid(const loss_grid_desc_t* descs, int32_t n_shots, const loss_allocator_t* alloc,
                               void* cuda_stream, loss_handle_t* out) {
  if (!out) return LOSS_E_ARG;
  *out = nullptr;
  if (!descs || n_shots < 1) return LOSS_E_ARG;
  if (alloc && (!alloc->alloc || !alloc->free)) return LOSS_E_ARG;
  for (int i = 0; i < n_shots; ++i) {
    std::string why;
    loss_status_t st = validate(descs[i], &why);
    if (st != LOSS_OK) return st;
  }
  loss_ctx* h = new (std::nothrow) loss_ctx();
  if (!h) return LOSS_E_NOMEM;
  h->stream = (cudaStream_t)cuda_stream;
  if (alloc) {
    h->alloc = *alloc;
    h->has_alloc = true;
  }
  auto bail = [&](loss_status_t st) {
    loss_destroy(h);
    return st;
  };
  if (cudaGetDevice(&h->device) != cudaSuccess) return bail(LOSS_E_CUDA);
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device) != cudaSuccess)
    return bail(LOSS_E_CUDA);
  h->smem_optin = v;
  cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  // Thomas factor tables.
  std::vector<double> t64;
  std::vector<float> t32;
  thomas_tables(t64, t32);
  if (dev_alloc(h, kTableLen * sizeof(double), (void**)&h->t64) != LOSS_OK) return bail(LOSS_E_NOMEM);
  if (dev_alloc(h, kTableLen * sizeof(float), (void**)&h->t32) != LOSS_OK) return bail(LOSS_E_NOMEM);
  if (cudaMemcpyAsync(h->t64, t64.data(), kTableLen * sizeof(double), cudaMemcpyHostToDevice, h->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(h->t32, t32.data(), kTableLen * sizeof(float), cudaMemcpyHostToDevice, h->stream) !=
          cudaSuccess)
    return bail(LOSS_E_CUDA);
  if (dev_alloc(h, 2 * sizeof(int), (void**)&h->dflag) != LOSS_OK ||
      cudaMemsetAsync(h->dflag, 0, 2 * sizeof(int), h->stream) != cudaSuccess)
    return bail(LOSS_E_NOMEM);
  h->nflag = h->dflag + 1;
  h->shots.resize(n_shots);
  for (int i = 0; i < n_shots; ++i) {
    h->shots[i].d = descs[i];
    loss_status_t st = setup_shot(h, h->shots[i]);
    if (st != LOSS_OK) return bail(st);
  }
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return bail(LOSS_E_CUDA);
  *out = h;
  return LOSS_OK;
}

loss_status_t loss_destroy(loss_handle_t h) {
  if (!h) return LOSS_OK;
  cudaStreamSynchronize(h->stream);
  if (h->side) cudaStreamSynchronize(h->side);
  drop_events(h);
  batch_destroy(h);
  if (h->ev_x) cudaEventDestroy(h->ev_x);
  if (h->ev_g) cudaEventDestroy(h->ev_g);
  if (h->side) cudaStreamDestroy(h->side);
  std::vector<void*> owned = h->owned;
  for (void* p : owned) dev_free(h, p);
  cudaStreamSynchronize(h->stream);
  delete h;
  return LOSS_OK;
}

loss_status_t loss_set_launch(loss_handle_t h, int32_t kernel, int32_t lines_per_block, int32_t chunk_log2) {
  LOSS_TRY(guard(h));
  if (chunk_log2 != 0 && chunk_log2 != 3 && chunk_log2 != 4) return fail(h, LOSS_E_ARG, "chunk_log2 must be 0, 3 or 4");
  if (kernel < 0 || kernel >= LOSS_NUM_KERNELS) return fail(h, LOSS_E_ARG, "kernel id out of range");
  if (lines_per_block < 0 || lines_per_block > 32 || (lines_per_block & (lines_per_block - 1)))
    return fail(h, LOSS_E_ARG, "lines_per_block must be 0 or a power of two <= 32");
  h->lines_per_block[kernel] = lines_per_block;
  h->chunk_log2[kernel] = chunk_log2;
  return LOSS_OK;
}

loss_status_t loss_set_tile(loss_handle_t h, int32_t kernel, int32_t threads_per_block, int32_t chunk_log2) {
  LOSS_TRY(guard(h));
  if (chunk_log2 != 0 && chunk_log2 != 3 && chunk_log2 != 4) return fail(h, LOSS_E_ARG, "chunk_log2 must be 0, 3 or 4");
  if (kernel < 0 || kernel >= LOSS_NUM_KERNELS) return fail(h, LOSS_E_ARG, "kernel id out of range");
  if (threads_per_block != 0 && (threads_per_block < 32 || threads_per_block > 1024))
    return fail(h, LOSS_E_ARG, "threads_per_block must be 0 or in 32..1024");
  h->tile_threads[kernel] = threads_per_block;
  h->chunk_log2[kernel] = chunk_log2;
  return LOSS_OK;
}

loss_status_t loss_set_kernels(loss_handle_t h, int32_t family) {
  LOSS_TRY(guard(h));
  if (family != LOSS_KERNELS_LINE && family != LOSS_KERNELS_CONVOLUTION && family != LOSS_KERNELS_CONVOLUTION_ITEMS)
    return fail(h, LOSS_E_ARG, "unknown kernel family");
  for (const Shot& s : h->shots)
    if (s.staggered) return fail(h, LOSS_E_STATE, "choose the kernel family before the first step");
  h->tiled = family;
  return LOSS_OK;
}

loss_status_t loss_set_schedule(loss_handle_t h, int32_t batched, int32_t graph_steps) {
  LOSS_TRY(guard(h));
  if (graph_steps < 0) return fail(h, LOSS_E_ARG, "graph_steps must be >= 0");
  h->batched = batched != 0;
  h->graph_steps = graph_steps;
  if (graph_steps == 0) batch_release(h);
  return LOSS_OK;
}

loss_status_t loss_autotune(loss_handle_t h, int32_t steps, loss_tune_entry_t* out, int32_t cap, int32_t* n_out) {
  LOSS_TRY(guard(h));
  if (steps < 1) return fail(h, LOSS_E_ARG, "steps must be >= 1");
  if (n_out) *n_out = 0;
  bool ac = false, el = false, fp64 = false;
  for (const Shot& s : h->shots) {
    if (!s.has_model) return fail(h, LOSS_E_STATE, "loss_set_model must be called for every shot before tuning");
    ac = ac || s.d.physics == LOSS_ACOUSTIC;
    el = el || s.d.physics == LOSS_ELASTIC;
    fp64 = fp64 || s.esize == 8;
  }
  std::vector<int> kids;
  if (ac) kids.insert(kids.end(), {LOSS_KERNEL_ACOUSTIC_X, LOSS_KERNEL_ACOUSTIC_Z});
  if (ac && conv_z_used(h)) kids.push_back(LOSS_KERNEL_ACOUSTIC_Z2);  // the convolution z tiles: Z1 and Z2
  if (el) kids.insert(kids.end(), {LOSS_KERNEL_ELASTIC_X, LOSS_KERNEL_ELASTIC_Y, LOSS_KERNEL_ELASTIC_Z});
  // candidates: (threads, chunk_log2)
  std::vector<std::pair<int, int>> cand;
  for (int lc : {3, 4}) {
    if (fp64 && lc == 3) continue;
    for (int t : {128, 256, 512, 1024})
      if (!(fp64 && t > 512)) cand.push_back({t, lc});
  }
  // scratch copy: same grids, models, layers, source and schedule; zero fields
  std::vector<loss_grid_desc_t> descs;
  for (const Shot& s : h->shots) descs.push_back(s.d);
  loss_handle_t t = nullptr;
  LOSS_TRY(loss_create_grid(descs.data(), (int32_t)descs.size(), h->has_alloc ? &h->alloc : nullptr,
                            (void*)h->stream, &t));
  struct Drop {
    loss_handle_t t;
    ~Drop() { loss_destroy(t); }
  } drop{t};
  auto relay = [&](loss_status_t st) {
    if (st != LOSS_OK) h->err = "autotune: " + t->err;
    return st;
  };
  for (size_t i = 0; i < h->shots.size(); ++i) {
    const Shot& a = h->shots[i];
    Shot& b = t->shots[i];
    for (int m = 0; m < 3; ++m)
      if (a.model[m] && b.model[m])
        LOSS_TRY(cuda_check(h, cudaMemcpyAsync(b.model[m], a.model[m], (size_t)a.total * a.esize,
                                               cudaMemcpyDeviceToDevice, h->stream), "copy model"));
    b.has_model = true;
    b.vmax = a.vmax;
    b.b_const = a.b_const;
    b.b0 = a.b0;
    b.lam_const = a.lam_const;
    b.mu_const = a.mu_const;
    b.lam0 = a.lam0;
    b.mu0 = a.mu0;
    if (a.pml_on) LOSS_TRY(relay(loss_set_pml(t, (int32_t)i, a.pml_width, a.pml_R, a.pml_kmax, a.pml_f0)));
    b.src_on = a.src_on;
    b.src_kinds = a.src_kinds;
    for (int k = 0; k < 3; ++k) b.src_idx[k] = a.src_idx[k];
    b.src_amp = a.src_amp;
    b.src_f0 = a.src_f0;
    b.src_t0 = a.src_t0;
    b.src_norm = a.src_norm;
    for (int k = 0; k < 25; ++k) b.src_g[k] = a.src_g[k];
  }
  t->batched = h->batched;
  t->tiled = h->tiled;
  t->graph_steps = 0;  // plain launches, so that every kernel can be timed
  for (int k = 0; k < LOSS_NUM_KERNELS; ++k) {
    t->tile_threads[k] = h->tile_threads[k];
    t->chunk_log2[k] = h->chunk_log2[k];
  }
  const double inf = 1e300;
  std::vector<double> best(kids.size(), inf);
  std::vector<int> best_c(kids.size(), -1);
  for (size_t c = 0; c < cand.size(); ++c) {
    for (int kid : kids) {
      t->lines_per_block[kid] = 0;
      t->tile_threads[kid] = cand[c].first;
      t->chunk_log2[kid] = cand[c].second;
    }
    loss_status_t st = loss_step(t, 1);
    if (st == LOSS_E_UNSUPPORTED) continue;  // a shape that does not fit this grid
    LOSS_TRY(relay(st));
    LOSS_TRY(relay(loss_profile(t, 1)));
    LOSS_TRY(relay(loss_step(t, steps)));
    for (size_t f = 0; f < kids.size(); ++f) {
      double ms = 0.0;
      int64_t nl = 0;
      LOSS_TRY(relay(loss_profile_read(t, kids[f], &ms, &nl)));
      const double per_step = nl ? ms / steps : inf;
      if (per_step < best[f]) best[f] = per_step, best_c[f] = (int)c;
    }
    LOSS_TRY(relay(loss_profile(t, 0)));
  }
  int32_t n = 0;
  for (size_t f = 0; f < kids.size(); ++f) {
    if (best_c[f] < 0) continue;
    h->lines_per_block[kids[f]] = 0;
    h->tile_threads[kids[f]] = cand[best_c[f]].first;
    h->chunk_log2[kids[f]] = cand[best_c[f]].second;
    if (out && n < cap) out[n] = loss_tune_entry_t{kids[f], cand[best_c[f]].first, cand[best_c[f]].second, best[f]};
    ++n;
  }
  if (n_out) *n_out = n;
  return LOSS_OK;
}

loss_status_t loss_profile(loss_handle_t h, int32_t enable) {
  LOSS_TRY(guard(h));
  LOSS_TRY(cuda_check(h, cudaStreamSynchronize(h->stream), "sync"));
  drop_events(h);
  for (auto& c : h->launches) c = 0;
  h->prof = enable != 0;
  return LOSS_OK;
}

loss_status_t loss_profile_read(loss_handle_t h, int32_t kernel, double* total_ms, int64_t* launches) {
  LOSS_TRY(guard(h));
  if (kernel < -1 || kernel >= LOSS_NUM_KERNELS) return fail(h, LOSS_E_ARG, "kernel id out of range");
  LOSS_TRY(cuda_check(h, cudaStreamSynchronize(h->stream), "sync"));
  double ms = 0.0;
  for (auto& e : h->events) {
    if (kernel >= 0 && e.kernel != kernel) continue;
    float t = 0.0f;
    LOSS_TRY(cuda_check(h, cudaEventElapsedTime(&t, e.a, e.b), "cudaEventElapsedTime"));
    ms += t;
  }
  int64_t n = 0;
  for (int k = 0; k < LOSS_NUM_KERNELS; ++k)
    if (kernel < 0 || k == kernel) n += h->launches[k];
  if (total_ms) *total_ms = ms;
  if (launches) *launches = n;
  return LOSS_OK;
}

loss_status_t loss_sync(loss_handle_t h) {
  LOSS_TRY(guard(h));
  LOSS_TRY(cuda_check(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize"));
  int flag[2] = {0, 0};
  if (h->dflag)
    LOSS_TRY(cuda_check(h, cudaMemcpy(flag, h->dflag, 2 * sizeof(int), cudaMemcpyDeviceToHost), "read flags"));
  if (flag[0]) return fail(h, LOSS_E_TIMEOUT, "a kernel gave up waiting for its staged data");
  if (flag[1]) {
    LOSS_TRY(cuda_check(h, cudaMemsetAsync(h->nflag, 0, sizeof(int), h->stream), "clear flag"));
    LOSS_TRY(cuda_check(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize"));
    const int shot = (flag[1] - 1) / LOSS_NUM_FIELDS, field = (flag[1] - 1) % LOSS_NUM_FIELDS;
    return fail(h, LOSS_E_NUMERIC,
                "non-finite value in shot " + std::to_string(shot) + ", field " + std::to_string(field));
  }
  return LOSS_OK;
}

loss_status_t loss_set_wait_limit(loss_handle_t h, int64_t polls) {
  LOSS_TRY(guard(h));
  h->wait_polls = polls < 0 ? (1u << 24) : (unsigned)std::min<int64_t>(polls, 0xffffffffLL);
  return LOSS_OK;
}

loss_status_t loss_set_watchdog(loss_handle_t h, int64_t every_steps) {
  LOSS_TRY(guard(h));
  if (every_steps < 0) return fail(h, LOSS_E_ARG, "every_steps must be >= 0");
  h->watch_every = every_steps;
  h->watch_count = 0;
  return LOSS_OK;
}

// One watchdog pass over every field of every shot (loss_set_watchdog).
static loss_status_t watch_fields(loss_ctx* h) {
  for (size_t i = 0; i < h->shots.size(); ++i) {
    Shot& s = h->shots[i];
    for (int f = 0; f < LOSS_NUM_FIELDS; ++f) {
      if (!field_used(s, f)) continue;
      LaunchScope ls(h, LOSS_KERNEL_WATCH);
      LOSS_TRY(cuda_check(h, launch_finite(s.field[f], s.total, s.esize, h->nflag, 1 + (int)i * LOSS_NUM_FIELDS + f,
                                           h->num_sms, h->stream), "watchdog"));
    }
  }
  return LOSS_OK;
}

static loss_status_t get_shot(loss_ctx* h, int32_t shot, Shot** s) {
  LOSS_TRY(guard(h));
  if (shot < 0 || shot >= (int)h->shots.size()) return fail(h, LOSS_E_ARG, "shot index out of range");
  *s = &h->shots[shot];
  return LOSS_OK;
}

// SplitMix64 output function for input z (Steele, Lea and Flood, OOPSLA 2014): a bijective 64-bit mix.
static inline uint64_t splitmix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

// x rounded to one of its two FP32 neighbours with probabilities that make the result unbiased.
static float round_unbiased(double x, uint64_t key) {
  const float f = (float)x;
  const double d = (double)f;
  if (d == x || !std::isfinite(f) || !std::isfinite(x)) return f;
  const float g = std::nextafter(f, d < x ? std::numeric_limits<float>::infinity()
                                          : -std::numeric_limits<float>::infinity());
  const double lo = std::min(d, (double)g), hi = std::max(d, (double)g);
  const double up = (x - lo) / (hi - lo);
  const double u = (double)(splitmix64(key) >> 11) * 0x1.0p-53;
  return (float)(u < up ? hi : lo);
}

loss_status_t loss_round_fp32_unbiased(const double* x, float* out, int64_t n, uint64_t key0) {
  if (n < 0 || (n > 0 && (!x || !out))) return LOSS_E_ARG;
  for (int64_t i = 0; i < n; ++i) out[i] = round_unbiased(x[i], key0 + (uint64_t)i);
  return LOSS_OK;
}

loss_status_t loss_set_model(loss_handle_t h, int32_t shot, const double* vp, const double* vs, const double* rho,
                             int32_t mem) {
  Shot* s;
  LOSS_TRY(get_shot(h, shot, &s));
  const bool el = s->d.physics == LOSS_ELASTIC;
  if (!vp || !rho || (el && !vs)) return fail(h, LOSS_E_ARG, "missing model array");
  if (mem != LOSS_MEM_HOST && mem != LOSS_MEM_DEVICE) return fail(h, LOSS_E_ARG, "bad mem");
  const int64_t N = s->dense;
  std::vector<double> hvp, hvs, hrho;
  const double *pvp = vp, *pvs = vs, *prho = rho;
  if (mem == LOSS_MEM_DEVICE) {
    hvp.resize(N);
    hrho.resize(N);
    LOSS_TRY(cuda_check(h, cudaMemcpy(hvp.data(), vp, N * 8, cudaMemcpyDeviceToHost), "copy vp"));
    LOSS_TRY(cuda_check(h, cudaMemcpy(hrho.data(), rho, N * 8, cudaMemcpyDeviceToHost), "copy rho"));
    pvp = hvp.data();
    prho = hrho.data();
    if (el) {
      hvs.resize(N);
      LOSS_TRY(cuda_check(h, cudaMemcpy(hvs.data(), vs, N * 8, cudaMemcpyDeviceToHost), "copy vs"));
      pvs = hvs.data();
    }
  }
  const int nm = el ? 3 : 2;
  std::vector<double> md[3];
  for (int m = 0; m < nm; ++m) md[m].resize(N);
  for (int64_t i = 0; i < N; ++i) {
    const double r = prho[i];
    if (!(r > 0.0) || !std::isfinite(pvp[i])) return fail(h, LOSS_E_ARG, "rho must be > 0 and vp finite");
    if (el) {
      md[0][i] = r * (pvp[i] * pvp[i] - 2.0 * pvs[i] * pvs[i]);  // lambda
      md[1][i] = r * pvs[i] * pvs[i];                            // mu
      md[2][i] = 1.0 / r;                                        // b
    } else {
      md[0][i] = r * pvp[i] * pvp[i];  // kappa
      md[1][i] = 1.0 / r;              // b
    }
  }
  s->h_vp.assign(pvp, pvp + N);
  s->h_rho.assign(prho, prho + N);
  if (el) s->h_vs.assign(pvs, pvs + N);
  else s->h_vs.clear();
  s->vmax = 0.0;
  for (int64_t i = 0; i < N; ++i) s->vmax = std::max(s->vmax, std::fabs(pvp[i]));
  s->b_const = true;
  for (int64_t i = 1; i < N && s->b_const; ++i) s->b_const = prho[i] == prho[0];
  s->b0 = 1.0 / prho[0];
  if (el) {
    s->lam_const = s->mu_const = true;
    for (int64_t i = 1; i < N && s->lam_const; ++i) s->lam_const = md[0][i] == md[0][0];
    for (int64_t i = 1; i < N && s->mu_const; ++i) s->mu_const = md[1][i] == md[1][0];
    s->lam0 = md[0][0];
    s->mu0 = md[1][0];
  }
  for (int m = 0; m < nm; ++m) {
    if (s->esize == 8) {
      LOSS_TRY(copy_in(h, *s, s->model[m], md[m].data(), LOSS_MEM_HOST));
    } else {
      std::vector<float> f(N);
      // unbiased rounding: a layer of constant kappa (or lambda, mu) would otherwise carry one common relative
      // error of up to 2^-24, a systematic wave-speed bias whose phase error grows with the travel time
      for (int64_t i = 0; i < N; ++i) f[i] = round_unbiased(md[m][i], 3 * (uint64_t)i + (uint64_t)m);
      LOSS_TRY(copy_in(h, *s, s->model[m], f.data(), LOSS_MEM_HOST));
      LOSS_TRY(cuda_check(h, cudaStreamSynchronize(h->stream), "sync"));
    }
  }
  LOSS_TRY(cuda_check(h, cudaStreamSynchronize(h->stream), "sync"));
  s->has_model = true;
  return LOSS_OK;
}

loss_status_t loss_set_source(loss_handle_t h, int32_t shot, const int64_t idx[3], uint32_t kind_mask, double amp,
                              double f0, double t0) {
  Shot* s;
  LOSS_TRY(get_shot(h, shot, &s));
  if (kind_mask == 0) {
    s->src_on = false;
    return LOSS_OK;
  }
  if (!idx) return fail(h, LOSS_E_ARG, "null source index");
  const uint32_t allowed = s->d.physics == LOSS_ELASTIC
                               ? (LOSS_SRC_EXPLOSIVE | LOSS_SRC_SHEAR_XZ | kForceMask)
                               : LOSS_SRC_PRESSURE;
  if (kind_mask & ~allowed) return fail(h, LOSS_E_ARG, "source kind not valid for this physics");
  int64_t c[3];
  if (s->dim == 3) {
    c[0] = idx[0];
    c[1] = idx[1];
    c[2] = idx[2];
  } else {
    c[0] = idx[0];
    c[1] = 0;
    c[2] = idx[2];
  }
  for (int k = 0; k < 3; ++k)
    if (c[k] < 0 || c[k] > s->n[k]) return fail(h, LOSS_E_ARG, "source index outside the grid");
  for (int k = 0; k < 3; ++k) s->src_idx[k] = c[k];
  s->src_kinds = kind_mask;
  s->src_amp = amp;
  s->src_f0 = f0;
  s->src_t0 = t0;
  s->src_on = true;
  source_setup(*s);
  return LOSS_OK;
}

// Layer profile of axis slot k at position i: damping d and normalised depth r (paper Sec. 3.3, d = d0 r^2).  On
// an axis with knots of its own the depth is the physical distance into the layer over the layer's thickness,
// each end with its own thickness and d0; equally spaced knots give the same values as the point count.
static void pml_profile(const Shot& s, int k, std::vector<double>& d, std::vector<double>& r) {
  const int n = (int)s.n[k];
  const int W = s.pml_width;
  d.assign(n + 1, 0.0);
  r.assign(n + 1, 0.0);
  if (s.coords[k].empty()) {
    const double L = W * s.h[k];
    const double d0 = -3.0 * s.vmax * std::log(s.pml_R) / (2.0 * L);
    for (int i = 0; i <= n; ++i) {
      r[i] = std::max(std::max((double)(W - i), (double)(i - (n - W))), 0.0) / W;
      d[i] = d0 * r[i] * r[i];
    }
    return;
  }
  const std::vector<double>& x = s.coords[k];
  for (int side = 0; side < 2; ++side) {
    const int lo = side == 0 ? 0 : n - W, hi = side == 0 ? W : n;
    const double inner = side == 0 ? x[W] : x[n - W];
    const double L = std::fabs(inner - (side == 0 ? x[0] : x[n]));
    const double d0 = -3.0 * s.vmax * std::log(s.pml_R) / (2.0 * L);
    for (int i = lo; i <= hi; ++i) {
      const double rr = std::fabs(x[i] - inner) / L;
      r[i] = std::max(r[i], rr);
      d[i] = std::max(d[i], d0 * rr * rr);
    }
  }
}

static void pml_table(const Shot& s, int k, double tau, std::vector<double>& tab) {
  const int n = (int)s.n[k];
  tab.assign((size_t)4 * (n + 1), 0.0);
  std::vector<double> dd, rr;
  pml_profile(s, k, dd, rr);
  for (int i = 0; i <= n; ++i) {
    const double r = rr[i];
    const double d = dd[i], kk = 1.0 + (s.pml_kmax - 1.0) * r, al = M_PI * s.pml_f0 * (1.0 - r);
    double E = 1.0, cp = 0.0, c1 = 0.0, c2 = tau;
    if (d > 0.0) {
      const double beta = d / kk + al;
      E = std::exp(-beta * tau);
      cp = (d / (kk * kk)) * (1.0 - E) / beta;
      c1 = 1.0 / beta;
      c2 = tau * al / (d + al * kk);
    }
    tab[i] = E;
    tab[(n + 1) + i] = cp;
    tab[2 * (n + 1) + i] = c1;
    tab[3 * (n + 1) + i] = c2;
  }
}

static loss_status_t rebuild_receivers(loss_ctx* h, Shot& s) {
  if (s.rcv_steps > 0) return fail(h, LOSS_E_STATE, "read the recorded traces (loss_record) before changing receivers");
  std::vector<int64_t> all;
  s.rcv_offsets.clear();
  for (int f = 0; f < LOSS_NUM_FIELDS; ++f) {
    s.rcv_offsets.push_back((int64_t)all.size());
    for (int64_t q : s.rcv[f]) {
      const int64_t x = q % s.len[2];
      const int64_t r = q / s.len[2];
      all.push_back(r * s.px + x);  // rows (z, y) are contiguous in the padded layout with pitch px
    }
  }
  s.rcv_offsets.push_back((int64_t)all.size());
  s.n_rcv = (int64_t)all.size();
  if (s.rcv_idx) dev_free(h, s.rcv_idx);
  s.rcv_idx = nullptr;
  if (!all.empty()) {
    LOSS_TRY(dev_alloc(h, all.size() * sizeof(int64_t), (void**)&s.rcv_idx));
    LOSS_TRY(cuda_check(h, cudaMemcpyAsync(s.rcv_idx, all.data(), all.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                                           h->stream), "copy receivers"));
    LOSS_TRY(cuda_check(h, cudaStreamSynchronize(h->stream), "sync"));
  }
  return LOSS_OK;
}

loss_status_t loss_set_pml(loss_handle_t h, int32_t shot, int32_t width, double R, double k_max, double f0) {
  Shot* s;
  LOSS_TRY(get_shot(h, shot, &s));
  if (width < 0 || !(R > 0.0 && R < 1.0) || !(k_max > 0.0) || !(f0 > 0.0))
    return fail(h, LOSS_E_ARG, "bad PML parameters");
  for (int k = 0; k < 3; ++k)
    if (!(s->dim == 2 && k == 1) && 2 * (int64_t)width > s->n[k]) return fail(h, LOSS_E_ARG, "PML wider than half an axis");
  if (width > 0 && !s->has_model) return fail(h, LOSS_E_STATE, "loss_set_model must precede loss_set_pml");
  LOSS_TRY(unstagger(h, *s));
  s->pml_on = width > 0;
  s->pml_width = width;
  s->pml_R = R;
  s->pml_kmax = k_max;
  s->pml_f0 = f0;
  if (!s->pml_on) return LOSS_OK;
  LOSS_TRY(pml_upload_tables(h, *s));
  const size_t fb = (size_t)s->total * s->esize;
  for (int k = 0; k < 3; ++k) {
    if (s->dim == 2 && k == 1) continue;
    if (s->d.physics == LOSS_ELASTIC) continue;
    if (!s->psi[k]) LOSS_TRY(dev_zero_alloc(h, fb, &s->psi[k]));
    if (!s->phi[k]) LOSS_TRY(dev_zero_alloc(h, fb, &s->phi[k]));
    LOSS_TRY(cuda_check(h, cudaMemsetAsync(s->psi[k], 0, fb, h->stream), "memset"));
    LOSS_TRY(cuda_check(h, cudaMemsetAsync(s->phi[k], 0, fb, h->stream), "memset"));
  }
  if (s->d.physics == LOSS_ELASTIC)
    for (int i = 0; i < 18; ++i) {
      if (!s->pmem[i]) LOSS_TRY(dev_zero_alloc(h, fb, &s->pmem[i]));
      LOSS_TRY(cuda_check(h, cudaMemsetAsync(s->pmem[i], 0, fb, h->stream), "memset"));
    }
  return cuda_check(h, cudaStreamSynchronize(h->stream), "sync");
}

loss_status_t loss_set_receivers(loss_handle_t h, int32_t shot, int32_t field, const int64_t* flat_idx, int64_t n,
                                 int32_t mem) {
  Shot* s;
  LOSS_TRY(get_shot(h, shot, &s));
  if (!field_used(*s, field)) return fail(h, LOSS_E_ARG, "field not present on this grid");
  if (n < 0 || (n > 0 && !flat_idx)) return fail(h, LOSS_E_ARG, "bad receiver list");
  std::vector<int64_t> idx(n);
  if (n) {
    if (mem == LOSS_MEM_DEVICE)
      LOSS_TRY(cuda_check(h, cudaMemcpy(idx.data(), flat_idx, n * 8, cudaMemcpyDeviceToHost), "copy receivers"));
    else
      std::memcpy(idx.data(), flat_idx, n * 8);
  }
  for (int64_t q : idx)
    if (q < 0 || q >= s->dense) return fail(h, LOSS_E_ARG, "receiver index outside the grid");
  std::vector<int64_t> old = s->rcv[field];
  s->rcv[field] = idx;
  loss_status_t st = rebuild_receivers(h, *s);
  if (st != LOSS_OK) s->rcv[field] = old;
  return st;
}

loss_status_t loss_set_field(loss_handle_t h, int32_t shot, int32_t field, const void* src, int32_t mem) {
  Shot* s;
  LOSS_TRY(get_shot(h, shot, &s));
  if (!field_used(*s, field)) return fail(h, LOSS_E_ARG, "field not present on this grid");
  if (!src || (mem != LOSS_MEM_HOST && mem != LOSS_MEM_DEVICE)) return fail(h, LOSS_E_ARG, "bad source buffer");
  LOSS_TRY(unstagger(h, *s));
  LOSS_TRY(upload_field(h, *s, s->field[field], src, mem));
  if (s->kahan)
    LOSS_TRY(cuda_check(h, cudaMemsetAsync(s->comp[field], 0, (size_t)s->total * s->esize, h->stream), "memset"));
  if (mem == LOSS_MEM_HOST) LOSS_TRY(cuda_check(h, cudaStreamSynchronize(h->stream), "sync"));
  return LOSS_OK;
}

loss_status_t loss_get_field(loss_handle_t h, int32_t shot, int32_t field, void* dst, int32_t mem) {
  Shot* s;
  LOSS_TRY(get_shot(h, shot, &s));
  if (!field_used(*s, field)) return fail(h, LOSS_E_ARG, "field not present on this grid");
  if (!dst || (mem != LOSS_MEM_HOST && mem != LOSS_MEM_DEVICE)) return fail(h, LOSS_E_ARG, "bad destination");
  if (is_velocity(field)) LOSS_TRY(unstagger(h, *s));
  LOSS_TRY(copy_out(h, *s, dst, s->field[field], mem));
  if (mem == LOSS_MEM_HOST) LOSS_TRY(cuda_check(h, cudaStreamSynchronize(h->stream), "sync"));
  return LOSS_OK;
}

loss_status_t loss_get_step(loss_handle_t h, int32_t shot, int64_t* step) {
  Shot* s;
  LOSS_TRY(get_shot(h, shot, &s));
  if (!step) return fail(h, LOSS_E_ARG, "null step");
  *step = s->step;
  return LOSS_OK;
}

loss_status_t loss_step(loss_handle_t h, int64_t n_steps) {
  LOSS_TRY(guard(h));
  if (n_steps < 0) return fail(h, LOSS_E_ARG, "n_steps must be >= 0");
  for (Shot& s : h->shots) {
    if (!s.has_model) return fail(h, LOSS_E_STATE, "loss_set_model must be called for every shot before stepping");
  }
  for (Shot& s : h->shots) LOSS_TRY(ensure_trace_capacity(h, s, s.rcv_steps + n_steps));
  if (batch_eligible(h)) {
    LOSS_TRY(step_batched(h, n_steps));
  } else {
    for (int64_t k = 0; k < n_steps; ++k) {
      for (Shot& s : h->shots) LOSS_TRY(step_shot(h, s));
    }
  }
  if (h->watch_every > 0) {
    h->watch_count += n_steps;
    if (h->watch_count >= h->watch_every) {
      h->watch_count %= h->watch_every;
      LOSS_TRY(watch_fields(h));
    }
  }
  return LOSS_OK;
}

loss_status_t loss_record_count(loss_handle_t h, int32_t shot, int64_t* n_steps, int64_t* n_receivers) {
  Shot* s;
  LOSS_TRY(get_shot(h, shot, &s));
  if (n_steps) *n_steps = s->rcv_steps;
  if (n_receivers) *n_receivers = s->n_rcv;
  return LOSS_OK;
}

loss_status_t loss_record(loss_handle_t h, int32_t shot, void* out, int32_t mem) {
  Shot* s;
  LOSS_TRY(get_shot(h, shot, &s));
  const size_t bytes = (size_t)s->rcv_steps * s->n_rcv * s->esize;
  if (bytes) {
    if (!out) return fail(h, LOSS_E_ARG, "null output");
    LOSS_TRY(cuda_check(h, cudaMemcpyAsync(out, s->traces, bytes,
                                           mem == LOSS_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                                           h->stream), "copy traces"));
    LOSS_TRY(cuda_check(h, cudaStreamSynchronize(h->stream), "sync"));
  }
  s->rcv_steps = 0;
  return LOSS_OK;
}

loss_status_t loss_derivative(loss_handle_t h, int32_t shot, int32_t axis, const void* f, void* d1, void* d2,
                              int32_t mem) {
  Shot* s;
  LOSS_TRY(get_shot(h, shot, &s));
  if (axis < 0 || axis >= s->dim) return fail(h, LOSS_E_ARG, "axis out of range");
  if (!f || !d1 || (mem != LOSS_MEM_HOST && mem != LOSS_MEM_DEVICE)) return fail(h, LOSS_E_ARG, "bad buffers");
  return run_derivative(h, *s, axis_slot(*s, axis), f, d1, d2, nullptr, mem);
}

loss_status_t loss_set_coordinates(loss_handle_t h, int32_t shot, int32_t axis, const double* x) {
  Shot* s;
  LOSS_TRY(get_shot(h, shot, &s));
  if (axis < 0 || axis >= s->dim) return fail(h, LOSS_E_ARG, "axis out of range");
  LOSS_TRY(unstagger(h, *s));  // the fields go back to the integer time level before the operator changes
  return set_coordinates(h, *s, axis_slot(*s, axis), x);
}

loss_status_t loss_derivative_adjoint(loss_handle_t h, int32_t shot, int32_t axis, const void* g, void* out,
                                      int32_t mem) {
  Shot* s;
  LOSS_TRY(get_shot(h, shot, &s));
  if (axis < 0 || axis >= s->dim) return fail(h, LOSS_E_ARG, "axis out of range");
  if (!g || !out || (mem != LOSS_MEM_HOST && mem != LOSS_MEM_DEVICE)) return fail(h, LOSS_E_ARG, "bad buffers");
  return run_derivative_adjoint(h, *s, axis_slot(*s, axis), g, out, mem);
}

loss_status_t loss_gradient(loss_handle_t h, int32_t shot, const double* d_obs, int32_t checkpoint_every,
                            int64_t n_steps, double* misfit, double* g_vp, double* g_vs, double* g_rho, int32_t mem) {
  Shot* s;
  LOSS_TRY(get_shot(h, shot, &s));
  if (any_nonuniform(*s)) return fail(h, LOSS_E_UNSUPPORTED, "gradients on non-uniform grids are not built");
  return run_gradient(h, *s, d_obs, checkpoint_every, n_steps, misfit, g_vp, g_vs, g_rho, mem);
}

loss_status_t loss_pmbc_phi(loss_handle_t h, int32_t shot, int32_t axis, const void* f, double* phi, int32_t mem) {
  Shot* s;
  LOSS_TRY(get_shot(h, shot, &s));
  if (axis < 0 || axis >= s->dim) return fail(h, LOSS_E_ARG, "axis out of range");
  if (!f || !phi || (mem != LOSS_MEM_HOST && mem != LOSS_MEM_DEVICE)) return fail(h, LOSS_E_ARG, "bad buffers");
  return run_derivative(h, *s, axis_slot(*s, axis), f, nullptr, nullptr, phi, mem);
}

loss_status_t loss_get_state(loss_handle_t h, void* blob, size_t* bytes) {
  LOSS_TRY(guard(h));
  if (!bytes) return fail(h, LOSS_E_ARG, "null size");
  size_t need = sizeof(uint64_t) * 2;
  for (Shot& s : h->shots) {
    need += sizeof(int64_t);
    for (int f = 0; f < LOSS_NUM_FIELDS; ++f)
      if (field_used(s, f)) need += (size_t)s.dense * s.esize * (s.kahan ? 2 : 1);
    for (int k = 0; k < 3; ++k)
      if (s.psi[k]) need += 2 * (size_t)s.dense * s.esize;
    for (int i = 0; i < 18; ++i)
      if (s.pmem[i]) need += (size_t)s.dense * s.esize;
  }
  if (!blob) {
    *bytes = need;
    return LOSS_OK;
  }
  if (*bytes < need) return fail(h, LOSS_E_ARG, "state buffer too small");
  unsigned char* p = (unsigned char*)blob;
  const uint64_t magic = 0x4c4f535353544154ull, ns = h->shots.size();
  std::memcpy(p, &magic, 8);
  std::memcpy(p + 8, &ns, 8);
  p += 16;
  for (Shot& s : h->shots) {
    LOSS_TRY(unstagger(h, s));
    std::memcpy(p, &s.step, 8);
    p += 8;
    for (int f = 0; f < LOSS_NUM_FIELDS; ++f) {
      if (!field_used(s, f)) continue;
      LOSS_TRY(copy_out(h, s, p, s.field[f], LOSS_MEM_HOST));
      p += (size_t)s.dense * s.esize;
      if (s.kahan) {
        LOSS_TRY(copy_out(h, s, p, s.comp[f], LOSS_MEM_HOST));
        p += (size_t)s.dense * s.esize;
      }
    }
    for (int k = 0; k < 3; ++k) {
      if (!s.psi[k]) continue;
      LOSS_TRY(copy_out(h, s, p, s.psi[k], LOSS_MEM_HOST));
      p += (size_t)s.dense * s.esize;
      LOSS_TRY(copy_out(h, s, p, s.phi[k], LOSS_MEM_HOST));
      p += (size_t)s.dense * s.esize;
    }
    for (int i = 0; i < 18; ++i) {
      if (!s.pmem[i]) continue;
      LOSS_TRY(copy_out(h, s, p, s.pmem[i], LOSS_MEM_HOST));
      p += (size_t)s.dense * s.esize;
    }
  }
  LOSS_TRY(cuda_check(h, cudaStreamSynchronize(h->stream), "sync"));
  *bytes = need;
  return LOSS_OK;
}

loss_status_t loss_set_state(loss_handle_t h, const void* blob, size_t bytes) {
  LOSS_TRY(guard(h));
  size_t need = 0;
  LOSS_TRY(loss_get_state(h, nullptr, &need));
  if (!blob || bytes != need) return fail(h, LOSS_E_ARG, "state blob has the wrong size");
  const unsigned char* p = (const unsigned char*)blob;
  uint64_t magic, ns;
  std::memcpy(&magic, p, 8);
  std::memcpy(&ns, p + 8, 8);
  if (magic != 0x4c4f535353544154ull || ns != h->shots.size()) return fail(h, LOSS_E_ARG, "not a state blob of this grid");
  p += 16;
  for (Shot& s : h->shots) {
    std::memcpy(&s.step, p, 8);
    p += 8;
    s.staggered = false;
    for (int f = 0; f < LOSS_NUM_FIELDS; ++f) {
      if (!field_used(s, f)) continue;
      LOSS_TRY(copy_in(h, s, s.field[f], p, LOSS_MEM_HOST));
      p += (size_t)s.dense * s.esize;
      if (s.kahan) {
        LOSS_TRY(copy_in(h, s, s.comp[f], p, LOSS_MEM_HOST));
        p += (size_t)s.dense * s.esize;
      }
    }
    for (int k = 0; k < 3; ++k) {
      if (!s.psi[k]) continue;
      LOSS_TRY(copy_in(h, s, s.psi[k], p, LOSS_MEM_HOST));
      p += (size_t)s.dense * s.esize;
      LOSS_TRY(copy_in(h, s, s.phi[k], p, LOSS_MEM_HOST));
      p += (size_t)s.dense * s.esize;
    }
    for (int i = 0; i < 18; ++i) {
      if (!s.pmem[i]) continue;
      LOSS_TRY(copy_in(h, s, s.pmem[i], p, LOSS_MEM_HOST));
      p += (size_t)s.dense * s.esize;
    }
  }
  return cuda_check(h, cudaStreamSynchronize(h->stream), "sync");
}

}  // extern "C"

// ----------------------------------------------------------------------------------------------------------------
// Internal pieces used above.
namespace lossk {

// The layer coefficient tables of every axis slot for the sub-step lengths dt, dt/2 and -dt/2.
loss_status_t pml_upload_tables(loss_ctx* h, Shot& s) {
  const double taus[3] = {s.d.dt, 0.5 * s.d.dt, -0.5 * s.d.dt};
  for (int k = 0; k < 3; ++k) {
    if (s.dim == 2 && k == 1) continue;
    for (int v = 0; v < 3; ++v) {
      std::vector<double> tab;
      pml_table(s, k, taus[v], tab);
      if (!s.pml_tab[k][v]) LOSS_TRY(dev_alloc(h, tab.size() * s.esize, &s.pml_tab[k][v]));
      if (s.esize == 8) {
        LOSS_TRY(cuda_check(h, cudaMemcpy(s.pml_tab[k][v], tab.data(), tab.size() * 8, cudaMemcpyHostToDevice),
                            "copy pml"));
      } else {
        std::vector<float> f(tab.begin(), tab.end());
        LOSS_TRY(cuda_check(h, cudaMemcpy(s.pml_tab[k][v], f.data(), f.size() * 4, cudaMemcpyHostToDevice),
                            "copy pml"));
      }
    }
  }
  return LOSS_OK;
}


bool is_velocity(int f) { return f == LOSS_FIELD_V1 || f == LOSS_FIELD_V2 || f == LOSS_FIELD_V3; }

loss_status_t ensure_trace_capacity(loss_ctx* h, Shot& s, int64_t rows) {
  if (s.n_rcv == 0 || rows <= s.trace_cap) return LOSS_OK;
  // at least 256 steps of headroom, so that stepping one step at a time does not reallocate every few steps
  const int64_t cap = std::max<int64_t>(rows + 256, 2 * s.trace_cap);
  void* nt = nullptr;
  LOSS_TRY(dev_alloc(h, (size_t)cap * s.n_rcv * s.esize, &nt));
  if (s.traces && s.rcv_steps)
    LOSS_TRY(cuda_check(h, cudaMemcpyAsync(nt, s.traces, (size_t)s.rcv_steps * s.n_rcv * s.esize,
                                           cudaMemcpyDeviceToDevice, h->stream), "grow traces"));
  if (s.traces) dev_free(h, s.traces);
  s.traces = nt;
  s.trace_cap = cap;
  return LOSS_OK;
}

template <typename T>
static Tables tables_for(loss_ctx* h, const Shot& s, int k) {
  return Tables{s.W[k], h->t32, h->t64};
}

template <typename T>
static loss_status_t run_derivative_t(loss_ctx* h, Shot& s, int k, const T* f, T* d1, T* d2, double* phi) {
  if (s.nu_tab[k]) {
    if (d2 && !d1) return fail(h, LOSS_E_ARG, "second derivatives on knots need the first derivative's array");
    return run_nu_derivative<T>(h, s, k, f, d1, phi, d2);
  }
  const int64_t sy = s.len[2], sz = s.len[2] * s.len[1];
  LineGeom g;
  int logc, threads;
  LOSS_TRY(line_geom(h, s, k, sz, sy, &g, &logc, &threads, d2 ? 3 : 2, 0, h->lines_per_block[LOSS_KERNEL_DERIVATIVE],
                     h->chunk_log2[LOSS_KERNEL_DERIVATIVE], h->tile_threads[LOSS_KERNEL_DERIVATIVE]));
  DerivArgs<T> a{};
  a.g = g;
  a.tb = tables_for<T>(h, s, k);
  a.f = f;
  a.d1 = d1;
  a.d2 = d2;
  a.phi_out = phi;
  a.s1 = (T)(3.0 / s.h[k]);
  a.s1d = 3.0 / s.h[k];
  a.s2 = (T)(6.0 / (s.h[k] * s.h[k]));
  a.minf = (T)(2.0 - std::sqrt(3.0));
  a.lines_per_outer = (int)s.len[2];
  LaunchScope ls(h, LOSS_KERNEL_DERIVATIVE);
  return cuda_check(h, launch_deriv<T>(a, logc, k != 2, threads, h->stream), "derivative kernel");
}

loss_status_t run_derivative(loss_ctx* h, Shot& s, int k, const void* f, void* d1, void* d2, double* phi, int mem) {
  const size_t fb = (size_t)s.dense * s.esize;
  const int64_t lines = s.dense / s.len[k];
  const size_t pb = (size_t)lines * (s.p[k] + 1) * sizeof(double);
  void *df = (void*)f, *dd1 = d1, *dd2 = d2;
  double* dphi = phi;
  std::vector<void*> tmp;
  auto cleanup = [&]() {
    for (void* p : tmp) dev_free(h, p);
  };
  if (mem == LOSS_MEM_HOST) {
    LOSS_TRY(dev_alloc(h, fb, &df));
    tmp.push_back(df);
    LOSS_TRY(cuda_check(h, cudaMemcpyAsync(df, f, fb, cudaMemcpyHostToDevice, h->stream), "copy f"));
    if (d1) {
      LOSS_TRY(dev_alloc(h, fb, &dd1));
      tmp.push_back(dd1);
    }
    if (d2) {
      LOSS_TRY(dev_alloc(h, fb, &dd2));
      tmp.push_back(dd2);
    }
    if (phi) {
      LOSS_TRY(dev_alloc(h, pb, (void**)&dphi));
      tmp.push_back(dphi);
    }
  }
  loss_status_t st;
  if (s.esize == 8)
    st = run_derivative_t<double>(h, s, k, (const double*)df, (double*)dd1, (double*)dd2, dphi);
  else
    st = run_derivative_t<float>(h, s, k, (const float*)df, (float*)dd1, (float*)dd2, dphi);
  if (st == LOSS_OK && mem == LOSS_MEM_HOST) {
    if (d1) st = cuda_check(h, cudaMemcpyAsync(d1, dd1, fb, cudaMemcpyDeviceToHost, h->stream), "copy d1");
    if (st == LOSS_OK && d2) st = cuda_check(h, cudaMemcpyAsync(d2, dd2, fb, cudaMemcpyDeviceToHost, h->stream), "copy d2");
    if (st == LOSS_OK && phi) st = cuda_check(h, cudaMemcpyAsync(phi, dphi, pb, cudaMemcpyDeviceToHost, h->stream), "copy phi");
    if (st == LOSS_OK) st = cuda_check(h, cudaStreamSynchronize(h->stream), "sync");
  }
  cleanup();
  return st;
}

}  // namespace lossk
