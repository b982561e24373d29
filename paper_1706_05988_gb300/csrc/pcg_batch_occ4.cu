// k_batch compiled for 4 resident blocks per SM (see pcg_batch_kernel.cuh).
#define PCG_KERNELS_IMPL
#define PCG_BATCH_KERNEL_IMPL
#include <cooperative_groups.h>

#include <type_traits>

#include "pcg_batch_kernel.cuh"

namespace pcgk {
PCG_BATCH_DEFINE_OCC(4)
}  // namespace pcgk
