// loss_derivative_noalloc: the stand-alone LOSS derivative for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs inside another framework's memory pool or
// allocator hooks, which owns every device allocation of the process, or under a memory budget that forbids new
// allocations after start-up.  loss_create_grid allocates (fields, tables), so such callers cannot use a handle.
// This entry point needs no handle: the caller passes device input and output arrays, and the only device memory
// the kernel reads besides them -- the PMBC weights of the axis and the Thomas factors -- lives in the file-scope
// static array below, which every GPU that loads this library holds until the process exits.  Each device has its
// own copy of the array; calls on one device whose work overlaps on the GPU race on that copy.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "loss_host.h"

namespace lossk {

// 64 KiB: PMBC weights ((p + 1) * (2 n_nb + 1) doubles) followed by the two Thomas tables.
constexpr size_t kNoAllocScratchBytes = 64 * 1024;
constexpr size_t kNoAllocTableBytes = kTableLen * (sizeof(double) + sizeof(float));
constexpr size_t kNoAllocMaxWeights = (kNoAllocScratchBytes - kNoAllocTableBytes) / sizeof(double);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch per device.  In host code the symbol is only a stand-in, so the address is
// looked up once per device, with that device current, and then reused.
constexpr int kMaxDevices = 64;
static void* g_scratch_addr[kMaxDevices] = {};
static std::mutex g_scratch_mu;

static cudaError_t scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

template <typename T>
static loss_status_t noalloc_run(loss_ctx* h, Shot& s, int k, const T* f, T* d1, unsigned char* scratch) {
  const std::vector<double> W = pmbc_weights_scaled((int)s.n[k], s.p[k], s.d.n_nb);
  if (W.size() > kNoAllocMaxWeights) return LOSS_E_UNSUPPORTED;
  std::vector<double> t64;
  std::vector<float> t32;
  thomas_tables(t64, t32);
  // Layout in the scratch array: [t64][t32][W]; every byte the kernel reads is rewritten by this call.
  double* d_t64 = (double*)scratch;
  float* d_t32 = (float*)(scratch + kTableLen * sizeof(double));
  double* d_W = (double*)(scratch + kNoAllocTableBytes);
  if (cudaMemcpyAsync(d_t64, t64.data(), kTableLen * sizeof(double), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
      cudaMemcpyAsync(d_t32, t32.data(), kTableLen * sizeof(float), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
      cudaMemcpyAsync(d_W, W.data(), W.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
    return LOSS_E_CUDA;
  const int64_t sy = s.len[2], sz = s.len[2] * s.len[1];
  LineGeom g;
  int logc, threads;
  loss_status_t st = line_geom(h, s, k, sz, sy, &g, &logc, &threads, 2, 0, 0, 0);
  if (st != LOSS_OK) return st;
  DerivArgs<T> a{};
  a.g = g;
  a.tb = Tables{d_W, d_t32, d_t64};
  a.f = f;
  a.d1 = d1;
  a.d2 = nullptr;
  a.phi_out = nullptr;
  a.s1 = (T)(3.0 / s.h[k]);
  a.s1d = 3.0 / s.h[k];
  a.s2 = (T)(6.0 / (s.h[k] * s.h[k]));
  a.minf = (T)(2.0 - std::sqrt(3.0));
  a.lines_per_outer = (int)s.len[2];
  return launch_deriv<T>(a, logc, k != 2, threads, h->stream) == cudaSuccess ? LOSS_OK : LOSS_E_CUDA;
}

}  // namespace lossk

using namespace lossk;

extern "C" loss_status_t loss_derivative_noalloc(const loss_grid_desc_t* desc, int32_t axis, const void* f, void* d1,
                                                 void* cuda_stream) {
  if (!desc || !f || !d1) return LOSS_E_ARG;
  // Only the geometry matters here: physics and dt take neutral values, so a caller may leave them unset.
  loss_grid_desc_t geo = *desc;
  geo.physics = LOSS_ACOUSTIC;
  geo.dt = 1.0;
  std::string why;
  loss_status_t st = validate(geo, &why);
  if (st != LOSS_OK) return st;
  if (axis < 0 || axis >= desc->dim) return LOSS_E_ARG;
  int dev = 0, smem = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LOSS_E_CUDA;
  if (cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return LOSS_E_CUDA;
  void* scratch = nullptr;
  if (scratch_address(dev, &scratch) != cudaSuccess) return LOSS_E_CUDA;
  loss_ctx ctx;  // host-side launch parameters only; nothing is allocated on the device
  ctx.stream = (cudaStream_t)cuda_stream;
  ctx.device = dev;
  ctx.smem_optin = smem;
  Shot s;
  s.d = geo;
  shot_geometry(s);
  const int k = (s.dim == 3) ? axis : (axis == 0 ? 0 : 2);
  if (s.esize == 8)
    return noalloc_run<double>(&ctx, s, k, (const double*)f, (double*)d1, (unsigned char*)scratch);
  return noalloc_run<float>(&ctx, s, k, (const float*)f, (float*)d1, (unsigned char*)scratch);
}
