// Kernel instantiations for the CSR (int32 indices) operators.
#define PCG_KERNELS_IMPL
#include "pcg_kernels.cuh"

namespace pcgk {
template struct Kernels<CsrOp>;
}  // namespace pcgk
