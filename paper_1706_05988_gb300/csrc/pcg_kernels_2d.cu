// Kernel instantiations for the 2D 5-point stencil operators.
#define PCG_KERNELS_IMPL
#include "pcg_kernels.cuh"

namespace pcgk {
template struct Kernels<StencilOp<2, false, 1>>;
template struct Kernels<StencilOp<2, false, 2>>;
template struct Kernels<StencilOp<2, true, 1>>;
template struct Kernels<StencilOp<2, true, 2>>;
}  // namespace pcgk
