// The large serving lane's kernel: k_server with wide binary32 sweeps, in a translation unit
// of its own so that it compiles in parallel with the rest of the server.
#define PCG_KERNELS_IMPL
#include "pcg_server_kernel.cuh"

namespace pcgk {
namespace srv {

int server_max_clusters_wide(int csize) { return server_max_clusters_t<true>(csize); }

cudaError_t launch_server_wide(const cudaLaunchConfig_t& cfg, ServerShared* sh, const WorkItem* items,
                               BatchOut* results, unsigned int* done, unsigned int cap, unsigned int* claim,
                               unsigned int* left) {
  return launch_server_t<true>(cfg, sh, items, results, done, cap, claim, left);
}

}  // namespace srv
}  // namespace pcgk
