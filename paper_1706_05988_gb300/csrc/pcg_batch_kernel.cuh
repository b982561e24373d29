// Device side of the batched launch: k_batch<family, mode, OCC>.
//
// Each thread-block cluster takes systems from a device work queue (largest first) and
// runs every iteration of Algorithm 3 for that system itself (pcg_cluster_solve.cuh,
// pcg_cluster_mixed.cuh): the blocks of the cluster split the system's unknowns, the dot
// products reduce warp -> block -> cluster through distributed shared memory, and one
// cluster barrier per iteration stands in for the global reduction.
//
// OCC is the number of resident blocks per SM the kernel is compiled for (register cap
// 65536 / (256 x OCC)).  The per-cluster sweeps of large systems wait on global loads, so
// with many systems more resident warps pay for the spills of a 64-register cap (OCC = 4:
// 79.4 / 109.2 solves/s FP64 / mixed + Jacobi on 512 high-contrast 2D systems, against
// 72.3 / 101.4 with OCC = 2); with fewer systems than an OCC = 2 grid holds, the spills
// only cost (64 large systems, mixed + Jacobi: 428.6 ms at OCC = 4, 294.8 ms at OCC = 2).
// Both are built, one per translation unit (pcg_batch_occ2.cu, pcg_batch_occ4.cu), and
// the host picks one per size class.
#pragma once
#include <cuda_runtime.h>

#include "pcg_cluster_mixed.cuh"

namespace pcgk {

// Solver per cluster: binary64 M = I, binary64 Jacobi, mixed M = I, mixed Jacobi.
enum { BM_FP64 = 0, BM_JAC, BM_MX, BM_MXJ, BM_NMODES };

struct BatchParams {
  double tol, eta;
  int maxit, max_restarts;
};

// Launch of k_batch<fam, mode, OCC> with `clusters` clusters of `csize` blocks on `stream`,
// and the most clusters of that shape the GPU holds at once (0 if it cannot launch it).
cudaError_t batch_launch_occ2(int fam, int mode, int clusters, int csize, cudaStream_t stream, const BatchSys* sys,
                              const int* order, int nsys, int* next, BatchVecs V, BatchOut* out, BatchParams prm);
cudaError_t batch_launch_occ4(int fam, int mode, int clusters, int csize, cudaStream_t stream, const BatchSys* sys,
                              const int* order, int nsys, int* next, BatchVecs V, BatchOut* out, BatchParams prm);
int batch_max_clusters_occ2(int fam, int mode, int csize);
int batch_max_clusters_occ4(int fam, int mode, int csize);

#ifdef PCG_BATCH_KERNEL_IMPL

template <int F, int MODE>
__device__ __forceinline__ void solve_one(cg::cluster_group& cl, double (*part)[4], int& slot, const BatchSys& d,
                                          const BatchVecs& V, const BatchParams& prm, BatchOut& res) {
  if constexpr (MODE == BM_FP64) cluster_solve<F>(cl, part, slot, d, V, prm.tol, prm.maxit, res);
  if constexpr (MODE == BM_JAC) cluster_solve_jac<F>(cl, part, slot, d, V, prm.tol, prm.maxit, res);
  if constexpr (MODE == BM_MX)
    cluster_solve_mx_auto<F, false>(cl, part, slot, d, V, prm.tol, prm.maxit, prm.eta, prm.max_restarts, res);
  if constexpr (MODE == BM_MXJ)
    cluster_solve_mx_auto<F, true>(cl, part, slot, d, V, prm.tol, prm.maxit, prm.eta, prm.max_restarts, res);
}

template <int F, int MODE, int OCC>
__global__ void __launch_bounds__(kBlock, OCC) k_batch(const BatchSys* __restrict__ sys, const int* __restrict__ order,
                                                    int nsys, int* next, BatchVecs V, BatchOut* out, BatchParams prm) {
  cg::cluster_group cl = cg::this_cluster();
  const unsigned rank = cl.block_rank();
  __shared__ double part[2][4];
  __shared__ int s_task;
  int slot = 0;
  for (;;) {
    if (rank == 0 && threadIdx.x == 0) s_task = atomicAdd(next, 1);
    cl.sync();
    const int task = *cl.map_shared_rank(&s_task, 0);
    cl.sync();                       // every block has read the task before rank 0 overwrites it
    if (task >= nsys) return;
    const int k = order[task];
    const BatchSys d = sys[k];
    BatchOut res;
    solve_one<F, MODE>(cl, part, slot, d, V, prm, res);
    if (rank == 0 && threadIdx.x == 0) out[k] = res;
    scalar_log_flush(sys[k].log);
  }
}

inline cudaLaunchAttribute cluster_attr(int csize) {
  cudaLaunchAttribute a;
  a.id = cudaLaunchAttributeClusterDimension;
  a.val.clusterDim.x = csize;
  a.val.clusterDim.y = 1;
  a.val.clusterDim.z = 1;
  return a;
}

template <int F, int MODE, int OCC>
cudaError_t launch_batch(int clusters, int csize, cudaStream_t stream, const BatchSys* sys, const int* order,
                         int nsys, int* next, BatchVecs V, BatchOut* out, BatchParams prm) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(clusters * csize);
  cfg.blockDim = dim3(kBlock);
  cfg.stream = stream;
  cudaLaunchAttribute attr[1] = {cluster_attr(csize)};
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_batch<F, MODE, OCC>, sys, order, nsys, next, V, out, prm);
}

template <int F, int MODE, int OCC>
int max_clusters(int csize) {
  if (csize > 8) {
    if (cudaFuncSetAttribute(k_batch<F, MODE, OCC>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
        cudaSuccess)
      return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(csize);
  cfg.blockDim = dim3(kBlock);
  cudaLaunchAttribute attr[1] = {cluster_attr(csize)};
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  return cudaOccupancyMaxActiveClusters(&n, k_batch<F, MODE, OCC>, &cfg) == cudaSuccess ? n : 0;
}

// fn(family, mode) with both as compile-time constants
template <int F, class Fn>
cudaError_t batch_with_mode(int mode, Fn&& fn) {
  switch (mode) {
    case BM_FP64: return fn(std::integral_constant<int, F>{}, std::integral_constant<int, BM_FP64>{});
    case BM_JAC: return fn(std::integral_constant<int, F>{}, std::integral_constant<int, BM_JAC>{});
    case BM_MX: return fn(std::integral_constant<int, F>{}, std::integral_constant<int, BM_MX>{});
    case BM_MXJ: return fn(std::integral_constant<int, F>{}, std::integral_constant<int, BM_MXJ>{});
    default: return cudaErrorInvalidValue;
  }
}

template <class Fn>
cudaError_t batch_with_family(int fam, int mode, Fn&& fn) {
  switch (fam) {
    case 0: return batch_with_mode<0>(mode, fn);
    case 1: return batch_with_mode<1>(mode, fn);
    case 2: return batch_with_mode<2>(mode, fn);
    case 3: return batch_with_mode<3>(mode, fn);
    case 4: return batch_with_mode<4>(mode, fn);
    default: return cudaErrorInvalidValue;
  }
}

#define PCG_BATCH_DEFINE_OCC(OCC)                                                                                 \
  cudaError_t batch_launch_occ##OCC(int fam, int mode, int clusters, int csize, cudaStream_t stream,             \
                                    const BatchSys* sys, const int* order, int nsys, int* next, BatchVecs V,     \
                                    BatchOut* out, BatchParams prm) {                                            \
    return batch_with_family(fam, mode, [&](auto F, auto M) {                                                    \
      return launch_batch<decltype(F)::value, decltype(M)::value, OCC>(clusters, csize, stream, sys, order,     \
                                                                      nsys, next, V, out, prm);                 \
    });                                                                                                          \
  }                                                                                                              \
  int batch_max_clusters_occ##OCC(int fam, int mode, int csize) {                                                \
    int n = 0;                                                                                                   \
    batch_with_family(fam, mode, [&](auto F, auto M) {                                                           \
      n = max_clusters<decltype(F)::value, decltype(M)::value, OCC>(csize);                                      \
      return cudaSuccess;                                                                                        \
    });                                                                                                          \
    return n;                                                                                                    \
  }

#endif  // PCG_BATCH_KERNEL_IMPL

}  // namespace pcgk
