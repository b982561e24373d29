// Kernel instantiations for the 3D 7-point stencil operators (FP64-sum, fixed-point-sum and
// variable-coefficient rows; one or two unknowns per thread).
#define PCG_KERNELS_IMPL
#include "pcg_kernels.cuh"
#include "pcg_persistent.cuh"

namespace pcgk {
template struct Kernels<StencilOp<3, ST_LAP_FP64, 1>>;
template struct Kernels<StencilOp<3, ST_LAP_FP64, 2>>;
template struct Kernels<StencilOp<3, ST_LAP_FIXED, 1>>;
template struct Kernels<StencilOp<3, ST_LAP_FIXED, 2>>;
template struct Kernels<StencilOp<3, ST_VAR, 1>>;
template struct Kernels<StencilOp<3, ST_VAR, 2>>;
template struct PersistentKernels<StencilOp<3, ST_LAP_FP64, 1>>;
template struct PersistentKernels<StencilOp<3, ST_LAP_FP64, 2>>;
template struct PersistentKernels<StencilOp<3, ST_LAP_FIXED, 1>>;
template struct PersistentKernels<StencilOp<3, ST_LAP_FIXED, 2>>;
template struct PersistentKernels<StencilOp<3, ST_VAR, 1>>;
template struct PersistentKernels<StencilOp<3, ST_VAR, 2>>;
}  // namespace pcgk
