// Kernel instantiations for the 3D 7-point stencil operators.
#define PCG_KERNELS_IMPL
#include "pcg_kernels.cuh"

namespace pcgk {
template struct Kernels<StencilOp<3, false, 1>>;
template struct Kernels<StencilOp<3, false, 2>>;
template struct Kernels<StencilOp<3, true, 1>>;
template struct Kernels<StencilOp<3, true, 2>>;
}  // namespace pcgk
