// The serving kernel: persistent thread-block clusters that take solve requests from a
// ring in mapped host memory (see pcg_server.cu for the host side).  Instantiated twice:
// k_server<false> (small lane, one unknown per thread in every sweep) in pcg_server.cu and
// k_server<true> (large lane, wide binary32 sweeps) in pcg_server_wide.cu.
#pragma once
#include <cuda/atomic>
#include <cuda_runtime.h>

#include "pcg_cluster_mixed.cuh"

namespace pcgk {
namespace srv {

constexpr unsigned long long kIdleNs = 20ull * 1000 * 1000;   // an idle kernel exits after 20 ms

struct WorkItem {
  int family, maxit;
  int mode, max_restarts;    // mode: 0 binary64, 1 binary64 + Jacobi, 2 mixed, 3 mixed + Jacobi
  double tol, eta;
  BatchSys sys;        // operator (device pointers), sigma; off = 0
  BatchVecs vec;       // the request's vectors in the arena
};

// Shared between host and device (mapped pinned memory).
struct ServerShared {
  unsigned int tail;         // items published by the host
  unsigned int claimed;      // items taken by the kernel (mirror of the device counter)
  unsigned int live;         // 1 while a kernel runs (cleared by the last exiting cluster)
  unsigned int stop;         // host asks the kernel to exit
  unsigned int atomic_mirror;  // 1: the device may use system-scope atomics on this memory
  unsigned int pad[27];
};

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// WIDE: the mixed-precision sweeps take several unknowns per thread when the row length
// allows (the large lane); otherwise one, which keeps the small lane's kernel small.
template <int F, bool WIDE>
__device__ __forceinline__ void solve_item(cg::cluster_group& cl, double (*part)[4], int& slot, const WorkItem& w,
                                        BatchOut& res) {
  switch (w.mode) {
    case 1: cluster_solve_jac<F>(cl, part, slot, w.sys, w.vec, w.tol, w.maxit, res); break;
    case 2:
      if constexpr (WIDE) {
        cluster_solve_mx_auto<F, false>(cl, part, slot, w.sys, w.vec, w.tol, w.maxit, w.eta, w.max_restarts, res);
      } else {
        cluster_solve_mx<F, false>(cl, part, slot, w.sys, w.vec, w.tol, w.maxit, w.eta, w.max_restarts, res);
      }
      break;
    case 3:
      if constexpr (WIDE) {
        cluster_solve_mx_auto<F, true>(cl, part, slot, w.sys, w.vec, w.tol, w.maxit, w.eta, w.max_restarts, res);
      } else {
        cluster_solve_mx<F, true>(cl, part, slot, w.sys, w.vec, w.tol, w.maxit, w.eta, w.max_restarts, res);
      }
      break;
    default: cluster_solve<F>(cl, part, slot, w.sys, w.vec, w.tol, w.maxit, res); break;
  }
}

// Before a request is solved, its cluster derives the binary32 coefficient copies and, with
// Jacobi, D^{-1} in binary64 and binary32 (the diagonal of a CSR row found by column) from
// the binary64 data the host uploaded: the admission's host work stays one pass over the
// data, and no extra kernel has to wait for SMs the persistent clusters hold.
__device__ __forceinline__ void prepare_item(cg::cluster_group& cl, const WorkItem& w) {
  const int family = w.family, mode = w.mode;
  const bool jac = mode & 1, mixed = mode >= 2;
  if (!jac && !(mixed && family != 0 && family != 2)) return;   // nothing to derive
  const BatchSys& d = w.sys;
  double* dinv = const_cast<double*>(w.vec.dinv);
  float* dinv32 = reinterpret_cast<float*>(const_cast<double*>(w.vec.dinv32));
  const int n = d.n;
  const int stride = (int)(cl.num_blocks() * kBlock);
  for (int i = (int)(cl.block_rank() * kBlock + threadIdx.x); i < n; i += stride) {
    if (family == 4) {
      const int beg = d.row_ptr[i], end = d.row_ptr[i + 1];
      double dg = 0.0;
      for (int k = beg; k < end; ++k) {
        if (d.col[k] == i) dg += d.val[k];
        if (mixed) const_cast<float*>(d.val32)[k] = f32_of(d.val[k]);
      }
      if (jac) {
        dinv[i] = 1.0 / dg;
        dinv32[i] = f32_of(dinv[i]);
      }
    } else if (family == 1 || family == 3) {
      if (mixed) {
        const_cast<float*>(d.diag32)[i] = f32_of(d.diag[i]);
        const_cast<float*>(d.ax32)[i] = f32_of(d.ax[i]);
        const_cast<float*>(d.ay32)[i] = f32_of(d.ay[i]);
        if (family == 3) const_cast<float*>(d.az32)[i] = f32_of(d.az[i]);
      }
      if (jac) {
        dinv[i] = 1.0 / d.diag[i];
        dinv32[i] = f32_of(dinv[i]);
      }
    } else {
      dinv[i] = family == 2 ? 1.0 / 6.0 : 1.0 / 4.0;
      dinv32[i] = f32_of(dinv[i]);
    }
  }
  cl.sync();   // cluster-scope release/acquire: every block sees the derived arrays
}

// Copy of a work item from mapped host memory, bypassing the caches (a ring slot is reused).
__device__ __forceinline__ void load_item(const WorkItem* src, WorkItem* dst) {
  static_assert(sizeof(WorkItem) % 8 == 0, "word copy");
  const unsigned long long* a = reinterpret_cast<const unsigned long long*>(src);
  unsigned long long* b = reinterpret_cast<unsigned long long*>(dst);
  for (unsigned i = 0; i < sizeof(WorkItem) / 8; ++i) b[i] = __ldcv(a + i);
}

// Resident blocks per SM k_server is compiled for (register cap 65536 / (256 x this)).
#ifndef PCG_SERVER_MIN_BLOCKS
#define PCG_SERVER_MIN_BLOCKS 2
#endif

template <bool WIDE>
__global__ void __launch_bounds__(kBlock, PCG_SERVER_MIN_BLOCKS) k_server(ServerShared* sh, const WorkItem* items, BatchOut* results,
                                                   unsigned int* done, unsigned int cap, unsigned int* claim,
                                                   unsigned int* left) {
  cg::cluster_group cl = cg::this_cluster();
  const unsigned rank = cl.block_rank();
  __shared__ double part[2][4];
  __shared__ long long s_task;
  __shared__ WorkItem s_item;
  int slot = 0;
  cuda::atomic_ref<unsigned, cuda::thread_scope_system> tail(sh->tail), stop(sh->stop);
  for (;;) {
    if (rank == 0 && threadIdx.x == 0) {
      long long task = -1;
      const unsigned long long t0 = now_ns();
      for (;;) {
        if (stop.load(cuda::memory_order_acquire)) break;
        const unsigned t = tail.load(cuda::memory_order_acquire);
        const unsigned h = *(volatile unsigned*)claim;
        if (h < t) {
          if (atomicCAS(claim, h, h + 1) == h) {
            task = h;
            // the mirror only grows: an atomic maximum where the host link has native
            // atomics (two leaders' plain stores could land out of order and leave it
            // behind the device counter, which the host would read as unclaimed work)
            if (sh->atomic_mirror) {
              atomicMax_system(&sh->claimed, h + 1);
            } else {
              *(volatile unsigned*)&sh->claimed = h + 1 > sh->claimed ? h + 1 : sh->claimed;
            }
            break;
          }
          continue;
        }
        if (now_ns() - t0 > kIdleNs) break;   // idle: give the GPU back
        __nanosleep(2000);
      }
      s_task = task;
    }
    cl.sync();
    const long long task = *cl.map_shared_rank(&s_task, 0);
    if (task >= 0 && threadIdx.x == 0) {
      // every block copies the item (written by the host before it published `tail`)
      load_item(items + task % cap, &s_item);
    }
    cl.sync();
    if (task < 0) {
      if (rank == 0 && threadIdx.x == 0) {
        if (atomicSub(left, 1u) == 1u) {
          __threadfence_system();
          cuda::atomic_ref<unsigned, cuda::thread_scope_system> live(sh->live);
          live.store(0u, cuda::memory_order_release);
        }
      }
      return;
    }
    const WorkItem w = s_item;
    prepare_item(cl, w);
    BatchOut res;
    switch (w.family) {
      case 0: solve_item<0, WIDE>(cl, part, slot, w, res); break;
      case 1: solve_item<1, WIDE>(cl, part, slot, w, res); break;
      case 2: solve_item<2, WIDE>(cl, part, slot, w, res); break;
      case 3: solve_item<3, WIDE>(cl, part, slot, w, res); break;
      default: solve_item<4, WIDE>(cl, part, slot, w, res); break;
    }
    scalar_log_flush(s_item.sys.log);
    cl.sync();   // every block's writes to x (and the scalar log) are done before the flag is raised
    if (rank == 0 && threadIdx.x == 0) {
      results[task % cap] = res;
      __threadfence_system();
      cuda::atomic_ref<unsigned, cuda::thread_scope_system> d(done[task % cap]);
      d.store(1u, cuda::memory_order_release);
    }
  }
}

template <bool WIDE>
int server_max_clusters_t(int csize) {
  if (csize > 8 &&
      cudaFuncSetAttribute(k_server<WIDE>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    return 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(csize);
  cfg.blockDim = dim3(kBlock);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  return cudaOccupancyMaxActiveClusters(&n, k_server<WIDE>, &cfg) == cudaSuccess ? n : 0;
}

template <bool WIDE>
cudaError_t launch_server_t(const cudaLaunchConfig_t& cfg, ServerShared* sh, const WorkItem* items,
                            BatchOut* results, unsigned int* done, unsigned int cap, unsigned int* claim,
                            unsigned int* left) {
  return cudaLaunchKernelEx(&cfg, k_server<WIDE>, sh, items, results, done, cap, claim, left);
}

// The large lane's instances live in their own translation unit (compiled in parallel).
int server_max_clusters_wide(int csize);
cudaError_t launch_server_wide(const cudaLaunchConfig_t& cfg, ServerShared* sh, const WorkItem* items,
                               BatchOut* results, unsigned int* done, unsigned int cap, unsigned int* claim,
                               unsigned int* left);

}  // namespace srv
}  // namespace pcgk
