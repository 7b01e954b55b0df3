// Host-side state of a LOSS handle and the internal functions shared by the host translation units.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/loss.h"
#include "loss_types.h"

namespace lossk {

constexpr int kTableLen = 64;
// Rounding error of v rounded to T, rounded to T (0 for double): the low part of a coefficient for mulc.
template <typename T>
inline T lo_part(double v) {
  return (T)(v - (double)(T)v);
}
// Body-force source kinds (f_1, f_2, f_3) and the component of each.
constexpr uint32_t kForceMask = LOSS_SRC_FORCE_X | LOSS_SRC_FORCE_Y | LOSS_SRC_FORCE_Z;
inline int force_components(uint32_t kinds) {
  return ((kinds & LOSS_SRC_FORCE_X) ? 1 : 0) | ((kinds & LOSS_SRC_FORCE_Y) ? 2 : 0) |
         ((kinds & LOSS_SRC_FORCE_Z) ? 4 : 0);
}

// One independent grid (shot).  Internal axis slots: 0 = z, 1 = y, 2 = x; 2-D grids have a y extent of 1.
// Device arrays use a padded layout: x pitch px (multiple of 32 elements), y stride sy = px, z stride sz.
struct Shot {
  loss_grid_desc_t d{};
  int dim = 0;
  int64_t n[3] = {0, 0, 0};
  int p[3] = {1, 1, 1};
  double h[3] = {1, 1, 1};
  int64_t len[3] = {1, 1, 1};
  int64_t px = 0, sy = 0, sz = 0, total = 0, dense = 0;
  size_t esize = 8;
  bool kahan = false;
  int nfields = 0;
  void* field[LOSS_NUM_FIELDS] = {};
  void* comp[LOSS_NUM_FIELDS] = {};
  void* model[3] = {};   // acoustic: kappa, b; elastic: lambda, mu, b
  void* tmp[8] = {};     // derivative temporaries (acoustic: tmp[0] = d_z v3)
  double* W[3] = {};     // PMBC weights per axis slot, scaled by h/3
  double* Wd[3] = {};     // junction-correction weights of the FP32 truncated-convolution kernels (on first use)
  void* nu_tab[3] = {};   // non-uniform axis slot (loss_set_coordinates): PMBC weights and elimination tables
  std::vector<double> coords[3];  // the knots loss_set_coordinates gave an axis slot (empty: equally spaced)
  bool has_model = false;
  double vmax = 0.0;
  bool b_const = false;  // density constant: buoyancy passed as a scalar, the b array is not read
  double b0 = 0.0;
  // source
  bool src_on = false;
  uint32_t src_kinds = 0;
  int64_t src_idx[3] = {0, 0, 0};
  double src_amp = 0, src_f0 = 0, src_t0 = 0, src_norm = 0;
  double src_g[25] = {};
  // receivers
  std::vector<int64_t> rcv[LOSS_NUM_FIELDS];
  std::vector<int64_t> rcv_offsets;
  int64_t* rcv_idx = nullptr;  // padded offsets, all fields concatenated
  int64_t n_rcv = 0;
  void* traces = nullptr;
  int64_t trace_cap = 0, rcv_steps = 0;
  // absorbing ADE-PML layer
  bool pml_on = false;
  int pml_width = 0;
  double pml_R = 1e-6, pml_kmax = 1.0, pml_f0 = 0.0;
  void* pml_tab[3][3] = {};  // [axis slot][0: tau = dt, 1: dt/2, 2: -dt/2], each [4][n+1] in working precision
  void* psi[3] = {};         // memory variables of the velocity sub-step, per derivative axis slot (acoustic)
  void* phi[3] = {};         // memory variables of the stress sub-step (acoustic)
  void* pmem[18] = {};       // elastic: 9 stress-sub-step terms d_j v_i at 3(i-1)+(j-1), then 9 velocity terms
  void* rdelta[9] = {};      // receiver corrections of velocity term (i, j) at 3(i-1)+(j-1), layers only
  bool lam_const = false, mu_const = false;
  double lam0 = 0.0, mu0 = 0.0;
  // time stepping
  int64_t step = 0;
  bool staggered = false;  // velocities hold v at t_step + dt/2 instead of t_step
  // model as given to loss_set_model (dense, FP64), for the chain rule of the misfit gradient
  std::vector<double> h_vp, h_vs, h_rho;
  // adjoint workspace (loss_gradient): adjoint fields, adjoint PML memory variables (same slots as psi/phi or
  // pmem), velocity residual arrays, FP64 gradients of (lambda or kappa, mu, b)
  void* lam[LOSS_NUM_FIELDS] = {};
  void* lam_mem[18] = {};
  void* rv[3] = {};
  double* grad[3] = {};
  // per-step source amplitudes for launches that read them from the device (batched / graph schedule)
  double* amp_tab = nullptr;
  int64_t amp_cap = 0;
  double amp_sig[5] = {};  // dt, norm, f0, t0, kinds the table was built for
};

// Device tables and launch shapes of the batched schedule (one persistent launch per kernel over all shots).
struct BatchState {
  void* xtab = nullptr;   // AcXArgs[n_shots]
  void* ztab = nullptr;   // AcZArgs[n_shots]
  int* tile0 = nullptr;   // [2][n_shots + 1]: first tile of each shot, X then Z
  void* jobs = nullptr;   // GatherJob[pre jobs + post jobs]
  StepClock* clk = nullptr;
  size_t cap_bytes[6] = {};  // allocated bytes of xtab, ztab, tile0, jobs, xptab, tztab
  int clk_cap = 0;
  std::vector<unsigned char> host[6];  // last uploaded contents of the same tables
  int xthreads = 0, zthreads = 0, xlogc = 0, zlogc = 0;
  size_t xsmem = 0, zsmem = 0;
  int xtiles = 0, ztiles = 0;
  int xgrid = 0, zgrid = 0;  // persistent grid sizes
  std::vector<unsigned char> clk_host;  // clocks the device holds after the last batched call
  int npre = 0, npost = 0;
  int64_t pre_max = 0, post_max = 0;
  // captured graph of graph_k batched steps and the launch signature it was captured for
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t cap_stream = nullptr;  // private stream the graph is captured on (the legacy default stream of the
                                      // handle cannot be captured); replays go to the handle's stream
  int64_t graph_k = 0;
  std::vector<int64_t> gsig;
  int64_t graph_launches[LOSS_NUM_KERNELS] = {};  // kernel launches in one replay
  // FP32 truncated-convolution form: x descriptors, z descriptors of Z1 then Z2; the int table in tile0's slot holds
  // unit0[n_shots + 1], bunit[xpgrid + 1], bshot[xpgrid], ztile0[n_shots + 1]
  bool conv = false;
  void* xptab = nullptr;  // XpShot[n_shots]
  void* tztab = nullptr;  // TzShot[2 n_shots]
  XpSmem xl{};
  int xpthreads = 0, xpgrid = 0, tztiles = 0;
  int tzthreads[2] = {0, 0}, tzlogc[2] = {4, 4}, tzgrid[2] = {0, 0};
  size_t tzsmem[2] = {0, 0};
};

}  // namespace lossk

struct loss_ctx {
  std::vector<lossk::Shot> shots;
  cudaStream_t stream = nullptr;
  loss_allocator_t alloc{};
  bool has_alloc = false;
  std::vector<void*> owned;
  std::string err;
  loss_status_t sticky = LOSS_OK;
  int device = 0;
  int smem_optin = 0;
  int num_sms = 0;
  double* t64 = nullptr;
  float* t32 = nullptr;
  int lines_per_block[LOSS_NUM_KERNELS] = {};  // 0 = built-in choice (loss_set_launch)
  int chunk_log2[LOSS_NUM_KERNELS] = {};
  int tile_threads[LOSS_NUM_KERNELS] = {};     // 0 = built-in choice (loss_set_tile)
  // schedule (loss_set_schedule)
  int batched = 1;       // several 2-D acoustic shots: one persistent launch per kernel over all of them
  int tiled = 1;         // LOSS_KERNELS_* family of the FP32 2-D acoustic shots stepped one at a time
  int* dflag = nullptr;  // device error flag of kernels with bounded waits (read by loss_sync)
  unsigned wait_polls = 1u << 24;  // poll limit of those waits (loss_set_wait_limit)
  // non-finite watchdog (loss_set_watchdog): every watch_every steps (0 = off) a check of every field sets nflag to
  // 1 + shot * LOSS_NUM_FIELDS + field of the first non-finite field found (read and cleared by loss_sync)
  int64_t watch_every = 0, watch_count = 0;
  int* nflag = nullptr;
  void* stage = nullptr;  // dense device staging buffer of pinned host uploads (loss_set_field)
  // side stream of the per-shot step's pressure / stress receiver gather, which then overlaps the z kernels:
  // ev_x marks the end of the x kernel (the stresses are final), ev_g the end of the gather
  cudaStream_t side = nullptr;
  cudaEvent_t ev_x = nullptr, ev_g = nullptr;
  size_t stage_bytes = 0;
  int graph_steps = 0;   // > 0: steps are replayed from a captured CUDA graph of this many steps
  bool capturing = false;
  lossk::BatchState batch;
  // launch accounting (loss_profile / loss_profile_read)
  int64_t launches[LOSS_NUM_KERNELS] = {};
  bool prof = false;
  struct Ev {
    int kernel;
    cudaEvent_t a, b;
  };
  std::vector<Ev> events;
};

namespace lossk {

// loss_api.cu
loss_status_t cuda_check(loss_ctx* h, cudaError_t e, const char* what);
loss_status_t dev_alloc(loss_ctx* h, size_t bytes, void** out);
void dev_free(loss_ctx* h, void* p);
loss_status_t line_geom(loss_ctx* h, const Shot& s, int k, int64_t sz, int64_t sy, LineGeom* g, int* logc, int* threads,
                        int nbuf, int nstage, int want_L, int want_logc, int want_threads = 0);
bool field_used(const Shot& s, int f);
void shot_geometry(Shot& s);
loss_status_t validate(const loss_grid_desc_t& d, std::string* why);
bool is_velocity(int f);
loss_status_t ensure_trace_capacity(loss_ctx* h, Shot& s, int64_t rows);
loss_status_t run_derivative(loss_ctx* h, Shot& s, int k, const void* f, void* d1, void* d2, double* phi, int mem);
// loss_nonuniform.cu
template <typename T>
loss_status_t run_nu_derivative(loss_ctx* h, Shot& s, int k, const T* f, T* d1, double* phi, T* d2 = nullptr);
template <typename T>
loss_status_t run_nu_derivative_adjoint(loss_ctx* h, Shot& s, int k, const T* g, T* out);
loss_status_t set_coordinates(loss_ctx* h, Shot& s, int k, const double* x);
loss_status_t nu_step(loss_ctx* h, Shot& s);  // one Strang step of a shot with non-uniform axes (2-D acoustic)
inline bool any_nonuniform(const Shot& s) { return s.nu_tab[0] || s.nu_tab[1] || s.nu_tab[2]; }
// loss_adjoint.cu
loss_status_t run_derivative_adjoint(loss_ctx* h, Shot& s, int k, const void* g, void* out, int mem);
loss_status_t run_gradient(loss_ctx* h, Shot& s, const double* d_obs, int32_t checkpoint_every, int64_t n_steps,
                           double* misfit, double* g_vp, double* g_vs, double* g_rho, int32_t mem);
std::vector<double> pmbc_weights_scaled(int n, int p, int n_nb);
std::vector<double> fir_delta_weights(int n, int p, int n_nb, int K);
void thomas_tables(std::vector<double>& t64, std::vector<float>& t32);

// Counts one launch of `kernel` and, when profiling is on, brackets it with CUDA events on the stream.
struct LaunchScope {
  loss_ctx* h;
  int kernel;
  cudaEvent_t a = nullptr, b = nullptr;
  LaunchScope(loss_ctx* hh, int k) : h(hh), kernel(k) {
    ++h->launches[k];
    if (h->prof && !h->capturing && cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess)
      cudaEventRecord(a, h->stream);
  }
  ~LaunchScope() {
    if (a && b) {
      cudaEventRecord(b, h->stream);
      h->events.push_back({kernel, a, b});
    }
  }
};

// loss_step.cu
loss_status_t step_shot(loss_ctx* h, Shot& s);
loss_status_t unstagger(loss_ctx* h, Shot& s);
loss_status_t stagger_shot(loss_ctx* h, Shot& s);
bool batch_eligible(const loss_ctx* h);
bool conv_z_used(const loss_ctx* h);  // some shot's FP32 step runs the convolution z tiles
loss_status_t step_batched(loss_ctx* h, int64_t n_steps);
void batch_release(loss_ctx* h);
void batch_destroy(loss_ctx* h);

// kernels
size_t smem_bytes(const LineGeom& g, int nbuf, int nstage, size_t esize);
template <typename T>
cudaError_t launch_deriv(const DerivArgs<T>& a, int logc, bool sflav, int threads, cudaStream_t st);
template <typename T, bool KAHAN>
cudaError_t launch_ac_x(const AcXArgs<T>& a, int logc, int threads, cudaStream_t st);
template <typename T, bool KAHAN>
cudaError_t launch_ac_z(const AcZArgs<T>& a, int logc, int threads, cudaStream_t st);
template <typename T, bool KAHAN>
cudaError_t launch_el(const ElArgs<T>& a, int pass, int logc, int threads, cudaStream_t st);
template <typename T>
cudaError_t launch_gather(const T* f, const int64_t* idx, int64_t n, T* out, int mode, const T* d0, const T* d1,
                          const T* d2, cudaStream_t st);
template <typename T, bool KAHAN>
cudaError_t batch_grid_ac_x(int logc, int threads, size_t smem, int ntiles, int num_sms, int* grid);
template <typename T, bool KAHAN>
cudaError_t batch_grid_ac_z(int logc, int threads, size_t smem, int ntiles, int num_sms, int* grid);
template <typename T, bool KAHAN>
cudaError_t launch_ac_x_batch(const AcXArgs<T>* tab, const int* tile0, int nshots, int ntiles, int logc, int threads,
                              size_t smem, int grid, cudaStream_t st);
template <typename T, bool KAHAN>
cudaError_t launch_ac_z_batch(const AcZArgs<T>* tab, const int* tile0, int nshots, int ntiles, int logc, int threads,
                              size_t smem, int grid, cudaStream_t st);
template <typename T>
cudaError_t launch_gather_batch(const GatherJob<T>* jobs, int njobs, int64_t max_cnt, cudaStream_t st);
cudaError_t launch_tick(StepClock* c, int n, cudaStream_t st);
// loss_api.cu: the absorbing-layer tables of every axis (after loss_set_pml or a change of knots)
loss_status_t pml_upload_tables(loss_ctx* h, Shot& s);
// loss_copy.cu: dst[r * pitch + c] = src[r * cols + c] on the device
cudaError_t launch_pitch_in(const void* src, void* dst, int64_t rows, int64_t cols, int64_t pitch, size_t esize,
                            int num_sms, cudaStream_t st);
cudaError_t launch_pitch_out(const void* src, void* dst, int64_t rows, int64_t cols, int64_t pitch, size_t esize,
                            int num_sms, cudaStream_t st);
// loss_watch.cu: sets *flag to code (if it is still 0) when one of the n values at f is not finite
cudaError_t launch_finite(const void* f, int64_t n, size_t esize, int* flag, int code, int num_sms, cudaStream_t st);
template <bool KAHAN>
cudaError_t launch_tz(const AcZArgs<float>& a, const TileGeom& t, int mode, int threads, int logc, cudaStream_t st);
template <bool KAHAN>
cudaError_t launch_xp(const AcXArgs<float>& a, const TileGeom& t, unsigned mmagic, int* err, unsigned polls,
                      int num_sms, cudaStream_t st);
size_t tile_smem_z(const TileGeom& t, int mode, int logc);
// loss_kernels_xtile.cu: the x part on (row, x patch) items, for rows the pipelined x kernel does not take
template <bool KAHAN>
cudaError_t launch_xt(const AcXArgs<float>& a, const TileGeom& t, cudaStream_t st);
size_t xt_smem(const TileGeom& t);
// loss_kernels_elastic.cu: elastic y / z tile passes (FP32)
size_t elt_smem(const ElTile& g, int logc);
template <bool KAHAN>
cudaError_t launch_elt(const ElArgs<float>& a, const ElTile& g, int pass, int logc, cudaStream_t st);
size_t xp_smem(const TileGeom& t, bool kahan);
int xp_rows_per_unit(int n, int threads);
XpSmem xp_batch_layout(const std::vector<TileGeom>& ts, const std::vector<int>& rs, bool kahan);
template <bool KAHAN>
cudaError_t launch_xp_batch(const XpShot* shots, const int* unit0, const int* bunit, const int* bshot,
                            const XpSmem& L, int threads, int grid, int* err, unsigned polls, cudaStream_t st);
template <bool KAHAN>
cudaError_t xp_batch_per_sm(const XpSmem& L, int threads, int* per_sm);
template <bool KAHAN>
cudaError_t launch_tz_batch(const TzShot* tab, const int* tile0, int nshots, int ntiles, int mode, int threads,
                            int logc, size_t smem, int grid, cudaStream_t st);
template <bool KAHAN>
cudaError_t tz_batch_per_sm(int mode, int threads, int logc, size_t smem, int* per_sm);
template <typename T>
cudaError_t launch_adj(const AdjArgs<T>& a, int logc, bool sflav, int threads, cudaStream_t st);
template <typename T>
cudaError_t launch_inject(const InjectJob<T>* jobs, int njobs, int64_t max_cnt, int64_t row, int64_t row_stride,
                          int phase, cudaStream_t st);

}  // namespace lossk
