// Element-wise kernel of the general iteration (u_0 = D^{-1} r_0) and the instantiations
// of the general sweep for the 2D stencil and CSR operators.
#define PCG_KERNELS_IMPL
#include "pcg_general.cuh"

namespace pcgk {
namespace {

__global__ void k_diag_scale(const double* __restrict__ d, const double* __restrict__ x, double* __restrict__ y,
                             int n, const State* st) {
  if (st->status != ST_RUNNING) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = d[i] * x[i];
}

// D^{-1} from a matrix already on the device: 1/diag for variable coefficients, the
// CSR row's entries in its own column summed, 1/6 or 1/4 for the constant stencils.  A
// non-positive or non-finite diagonal entry raises *bad.
__global__ void k_jacobi_dinv(OpDesc d, double* __restrict__ dinv, int* bad) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.n; i += gridDim.x * blockDim.x) {
    double dg;
    if (d.layout == 2) {
      dg = 0.0;
      for (int k = d.row_ptr[i]; k < d.row_ptr[i + 1]; ++k)
        if (d.col[k] == i) dg += d.val[k];
    } else if (d.diag) {
      dg = d.diag[i];
    } else {
      dg = d.layout == 1 ? 6.0 : 4.0;
    }
    if (!(dg > 0.0) || !isfinite(dg)) *bad = 1;
    dinv[i] = 1.0 / dg;
  }
}

}  // namespace

cudaError_t launch_jacobi_dinv(const OpDesc& d, double* dinv, int* bad, cudaStream_t stream) {
  const int grid = d.n / 256 + 1 < 4096 ? d.n / 256 + 1 : 4096;
  k_jacobi_dinv<<<grid, 256, 0, stream>>>(d, dinv, bad);
  return cudaGetLastError();
}

cudaError_t launch_diag_scale(const double* d, const double* x, double* y, int n, const State* st,
                              cudaStream_t stream) {
  const int grid = n / 256 + 1 < 4096 ? n / 256 + 1 : 4096;
  k_diag_scale<<<grid, 256, 0, stream>>>(d, x, y, n, st);
  return cudaGetLastError();
}

PCG_INSTANTIATE_GENERAL(CsrOp)
using G2A1 = StencilOp<2, ST_LAP_FP64, 1>;
using G2A2 = StencilOp<2, ST_LAP_FP64, 2>;
using G2B1 = StencilOp<2, ST_LAP_FIXED, 1>;
using G2B2 = StencilOp<2, ST_LAP_FIXED, 2>;
using G2C1 = StencilOp<2, ST_VAR, 1>;
using G2C2 = StencilOp<2, ST_VAR, 2>;
PCG_INSTANTIATE_GENERAL(G2A1)
PCG_INSTANTIATE_GENERAL(G2A2)
PCG_INSTANTIATE_GENERAL(G2B1)
PCG_INSTANTIATE_GENERAL(G2B2)
PCG_INSTANTIATE_GENERAL(G2C1)
PCG_INSTANTIATE_GENERAL(G2C2)

}  // namespace pcgk
