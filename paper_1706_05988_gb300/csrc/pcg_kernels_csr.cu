// Kernel instantiations for the CSR (int32 indices) operators.
#define PCG_KERNELS_IMPL
#include "pcg_kernels.cuh"
#include "pcg_persistent.cuh"

namespace pcgk {
template struct Kernels<CsrOp>;
template struct PersistentKernels<CsrOp>;
}  // namespace pcgk
