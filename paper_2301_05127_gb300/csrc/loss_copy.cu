// Dense -> pitched copy on the device, the second half of a host upload.
//
// Fields live in HBM with rows padded to a multiple of 32 elements.  Copying a dense host array straight into that
// layout takes a 2-D copy, which moves pinned host memory at about 130 GB/s on this machine against about 200 GB/s
// for a 1-D copy of the same bytes; so a pinned host array is first copied 1-D into a dense device staging buffer
// and then spread into the padded rows here, at HBM speed.
#include <cuda_runtime.h>

#include "loss_host.h"

namespace lossk {

template <typename T>
__global__ void __launch_bounds__(256) k_pitch_in(const T* __restrict__ src, T* __restrict__ dst, int64_t rows,
                                                  int64_t cols, int64_t pitch) {
  const int64_t n = rows * cols;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int64_t r = i / cols;
    dst[r * pitch + (i - r * cols)] = src[i];
  }
}

cudaError_t launch_pitch_in(const void* src, void* dst, int64_t rows, int64_t cols, int64_t pitch, size_t esize,
                            int num_sms, cudaStream_t st) {
  const int64_t n = rows * cols;
  if (n <= 0) return cudaSuccess;
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 8LL * num_sms);
  if (esize == 8)
    k_pitch_in<double><<<grid, 256, 0, st>>>((const double*)src, (double*)dst, rows, cols, pitch);
  else
    k_pitch_in<float><<<grid, 256, 0, st>>>((const float*)src, (float*)dst, rows, cols, pitch);
  return cudaGetLastError();
}

}  // namespace lossk
