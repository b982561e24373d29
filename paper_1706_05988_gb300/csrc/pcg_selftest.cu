// Self-check of the integer-pipe binary32 <-> binary64 conversions used by the
// mixed-precision kernels (pcg_convert.cuh), exposed through the C ABI so that a
// test can compare them with the IEEE conversions element by element.
#include <cuda_runtime.h>

#include "../../include/pcg.h"
#include "pcg_convert.cuh"

namespace {

__global__ void k_convert_check(const double* __restrict__ d_in, float* __restrict__ f_out,
                                const float* __restrict__ f_in, double* __restrict__ d_out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    f_out[i] = pcgk::f32_of(d_in[i]);
    d_out[i] = pcgk::f64_of(f_in[i]);
  }
}

}  // namespace

extern "C" pcg_status pcg_convert_check(const double* d_in, float* f_out, const float* f_in, double* d_out,
                                        int64_t n) {
  if (n < 0 || (n > 0 && (!d_in || !f_out || !f_in || !d_out))) return PCG_EINVAL;
  if (n == 0) return PCG_OK;
  const long long blocks = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
  k_convert_check<<<(int)blocks, 256>>>(d_in, f_out, f_in, d_out, n);
  if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return PCG_ECUDA;
  return PCG_OK;
}
