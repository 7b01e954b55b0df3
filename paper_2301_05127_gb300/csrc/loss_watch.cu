// Non-finite watchdog: one streaming pass over a field that records whether any value is Inf or NaN.
//
// A diverging run (a time step beyond the stability limit, a corrupted input) turns the fields non-finite within a
// few steps; the check runs every k steps (loss_set_watchdog) and its flag is read by loss_sync, which then
// reports LOSS_E_NUMERIC with the shot and field.  The pass reads the field once with 16-byte loads (the pitched
// arrays are zero-padded to a multiple of 32 elements and 128-byte aligned) and writes nothing but the flag.
#include <cuda_runtime.h>

#include "loss_host.h"

namespace lossk {

template <typename V, int E>
__global__ void __launch_bounds__(256) k_finite(const V* __restrict__ f, int64_t nvec, int* flag, int code) {
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvec; i += stride) {
    const V v = __ldcs(f + i);
    const auto* e = reinterpret_cast<const decltype(v.x)*>(&v);
#pragma unroll
    for (int k = 0; k < E; ++k) bad |= !isfinite(e[k]);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicCAS(flag, 0, code);
}

cudaError_t launch_finite(const void* f, int64_t n, size_t esize, int* flag, int code, int num_sms, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int threads = 256;
  if (esize == 8) {
    const int64_t nvec = n / 2;
    const int grid = (int)std::min<int64_t>((nvec + threads - 1) / threads, 4LL * num_sms);
    k_finite<double2, 2><<<grid, threads, 0, st>>>((const double2*)f, nvec, flag, code);
  } else {
    const int64_t nvec = n / 4;
    const int grid = (int)std::min<int64_t>((nvec + threads - 1) / threads, 4LL * num_sms);
    k_finite<float4, 4><<<grid, threads, 0, st>>>((const float4*)f, nvec, flag, code);
  }
  return cudaGetLastError();
}

}  // namespace lossk
