// Instantiations of the general sweep (Jacobi and/or variable shift) for the 3D stencil operators.
#define PCG_KERNELS_IMPL
#include "pcg_general.cuh"

namespace pcgk {
using G3A1 = StencilOp<3, ST_LAP_FP64, 1>;
using G3A2 = StencilOp<3, ST_LAP_FP64, 2>;
using G3B1 = StencilOp<3, ST_LAP_FIXED, 1>;
using G3B2 = StencilOp<3, ST_LAP_FIXED, 2>;
using G3C1 = StencilOp<3, ST_VAR, 1>;
using G3C2 = StencilOp<3, ST_VAR, 2>;
PCG_INSTANTIATE_GENERAL(G3A1)
PCG_INSTANTIATE_GENERAL(G3A2)
PCG_INSTANTIATE_GENERAL(G3B1)
PCG_INSTANTIATE_GENERAL(G3B2)
PCG_INSTANTIATE_GENERAL(G3C1)
PCG_INSTANTIATE_GENERAL(G3C2)
}  // namespace pcgk
