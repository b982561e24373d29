// Mixed-precision restart kernels (binary64 operator) and grid sizing.
#define PCG_KERNELS_IMPL
#include <algorithm>
#include <utility>

#include "pcg_mixed.cuh"
#include "pcg_mixed_jacobi.cuh"

namespace pcgk {

int mixed_iter_blocks_per_sm(const OpDesc& d);    // pcg_mixed_iter.cu
int mixedj_iter_blocks_per_sm(const OpDesc& d);   // pcg_mixed_iter.cu
int mixedj_vec(const OpDesc& d);                  // pcg_mixed_iter.cu

namespace {

template <int DIM, int MODE, int VEC>
StencilOp<DIM, MODE, VEC> make64(const OpDesc& d) {
  StencilOp<DIM, MODE, VEC> o;
  o.n = d.n;
  o.nx = d.nx;
  o.ny = d.ny;
  o.nz = d.nz;
  o.nxny = d.nx * d.ny;
  o.diag = d.diag;
  o.ax = d.ax;
  o.ay = d.ay;
  o.az = d.az;
  return o;
}

template <int DIM, class F>
cudaError_t with_stencil64(const OpDesc& d, F&& f) {
  const bool var = d.diag != nullptr;
  if (op_vec(d) == 2) {
    if (var) return f(make64<DIM, ST_VAR, 2>(d));
    if (d.fixed_sum) return f(make64<DIM, ST_LAP_FIXED, 2>(d));
    return f(make64<DIM, ST_LAP_FP64, 2>(d));
  }
  if (var) return f(make64<DIM, ST_VAR, 1>(d));
  if (d.fixed_sum) return f(make64<DIM, ST_LAP_FIXED, 1>(d));
  return f(make64<DIM, ST_LAP_FP64, 1>(d));
}

template <class F>
cudaError_t with_op64(const OpDesc& d, F&& f) {
  switch (d.layout) {
    case 0: return with_stencil64<2>(d, std::forward<F>(f));
    case 1: return with_stencil64<3>(d, std::forward<F>(f));
    case 2: {
      CsrOp o;
      o.n = d.n;
      o.row_ptr = d.row_ptr;
      o.col = d.col;
      o.val = d.val;
      return f(o);
    }
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_mx_restart(const OpDesc& d, const Launch& L, Vecs v, State* st, Hist h, double* partials) {
  return with_op64(d, [&](auto op) { return MixedRestartKernels<decltype(op)>::restart(op, L, v, st, h, partials); });
}
cudaError_t launch_mx_w0(const OpDesc& d, const Launch& L, Vecs v, State* st, Hist h, double* partials) {
  return with_op64(d, [&](auto op) { return MixedRestartKernels<decltype(op)>::w0(op, L, v, st, h, partials); });
}

cudaError_t launch_mxj_w0(const OpDesc& d, const Launch& L, const GenVecs& v, double* u64, State* st, Hist h,
                         double* partials) {
  return with_op64(d,
                   [&](auto op) { return MixedJacRestartKernels<decltype(op)>::w0(op, L, v, u64, st, h, partials); });
}

namespace {
__global__ void k_mxj_u0(GenVecs v, double* __restrict__ u64, int n, const State* st) {
  if (st->status != ST_RESTART) return;
  float* __restrict__ uf = reinterpret_cast<float*>(v.u);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float u32 = f32_of(v.dinv[i] * v.r[i]);
    uf[i] = u32;
    u64[i] = f64_of(u32);
  }
}
}  // namespace

cudaError_t launch_mxj_u0(const GenVecs& v, double* u64, int n, const State* st, cudaStream_t stream) {
  const int grid = n / 256 + 1 < 4096 ? n / 256 + 1 : 4096;
  k_mxj_u0<<<grid, 256, 0, stream>>>(v, u64, n, st);
  return cudaGetLastError();
}

int grid_for_mixed(const OpDesc& d, int kind, int block) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  int per_sm = 0;
  long long units = 0;
  if (kind == KM_ITER || kind == KM_ITER_JAC) {
    per_sm = kind == KM_ITER ? mixed_iter_blocks_per_sm(d) : mixedj_iter_blocks_per_sm(d);
    units = d.n / (kind == KM_ITER ? mixed_vec(d) : mixedj_vec(d));
  } else if (kind == KM_W0_JAC) {
    with_op64(d, [&](auto op) {
      per_sm = MixedJacRestartKernels<decltype(op)>::blocks_per_sm();
      return cudaSuccess;
    });
    units = d.n / op_vec(d);
  } else {
    with_op64(d, [&](auto op) {
      per_sm = MixedRestartKernels<decltype(op)>::blocks_per_sm(kind);
      return cudaSuccess;
    });
    units = d.n / op_vec(d);
  }
  if (per_sm <= 0) return 0;
  long long g = (long long)sms * per_sm;
  const long long need = (units + block - 1) / block;
  if (need < g) g = need;
  if (g < 1) g = 1;
  if (g > kMaxPartialBlocks) g = kMaxPartialBlocks;
  return (int)g;
}

// binary32 copy of a binary64 array (the operator's coefficients for the inner iteration)
__global__ void k_to_f32(const double* __restrict__ src, float* __restrict__ dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = f32_of(src[i]);
}

cudaError_t launch_to_f32(const double* src, float* dst, long long n, cudaStream_t stream) {
  const long long blocks = std::min<long long>((n + 255) / 256, 65535);
  k_to_f32<<<(int)(blocks > 0 ? blocks : 1), 256, 0, stream>>>(src, dst, n);
  return cudaGetLastError();
}

}  // namespace pcgk
