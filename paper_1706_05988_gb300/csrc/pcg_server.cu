// Continuous-batching solve server (pcg_server_*, pcg_submit, pcg_poll).
//
// Requests are admitted into a device arena of fixed size (first fit); a request that
// does not fit waits on the host until earlier requests are polled and free their
// memory.  Admitted requests are published to a ring of work items in mapped host
// memory.  A persistent kernel of thread-block clusters takes items as clusters come
// free (compare-and-swap on a device counter), solves each one with the per-cluster
// solver of the batched launch, and raises the item's completion flag with a
// system-scope release.  Work that arrives while other requests run is taken by the
// next free cluster: requests overlap on the device.  With no published work for
// kIdleNs the kernel's clusters exit; the host relaunches the kernel when work arrives.
// Every wait of the kernel is bounded by %globaltimer.
#include <cuda/atomic>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <deque>
#include <map>
#include <mutex>
#include <atomic>
#include <cstring>
#include <new>
#include <vector>

#define PCG_KERNELS_IMPL
#include "../../include/pcg.h"
#include "pcg_cluster_mixed.cuh"

namespace pcgk {
namespace {

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
  unsigned int pad[28];
};

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <int F>
__device__ __forceinline__ void solve_item(cg::cluster_group& cl, double (*part)[4], int& slot, const WorkItem& w,
                                        BatchOut& res) {
  switch (w.mode) {
    case 1: cluster_solve_jac<F>(cl, part, slot, w.sys, w.vec, w.tol, w.maxit, res); break;
    case 2:
      cluster_solve_mx<F, false>(cl, part, slot, w.sys, w.vec, w.tol, w.maxit, w.eta, w.max_restarts, res);
      break;
    case 3:
      cluster_solve_mx<F, true>(cl, part, slot, w.sys, w.vec, w.tol, w.maxit, w.eta, w.max_restarts, res);
      break;
    default: cluster_solve<F>(cl, part, slot, w.sys, w.vec, w.tol, w.maxit, res); break;
  }
}

// Copy of a work item from mapped host memory, bypassing the caches (a ring slot is reused).
__device__ __forceinline__ void load_item(const WorkItem* src, WorkItem* dst) {
  static_assert(sizeof(WorkItem) % 8 == 0, "word copy");
  const unsigned long long* a = reinterpret_cast<const unsigned long long*>(src);
  unsigned long long* b = reinterpret_cast<unsigned long long*>(dst);
  for (unsigned i = 0; i < sizeof(WorkItem) / 8; ++i) b[i] = __ldcv(a + i);
}

__global__ void __launch_bounds__(kBlock, 2) k_server(ServerShared* sh, const WorkItem* items, BatchOut* results,
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
            *(volatile unsigned*)&sh->claimed = h + 1 > sh->claimed ? h + 1 : sh->claimed;
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
    BatchOut res;
    switch (w.family) {
      case 0: solve_item<0>(cl, part, slot, w, res); break;
      case 1: solve_item<1>(cl, part, slot, w, res); break;
      case 2: solve_item<2>(cl, part, slot, w, res); break;
      case 3: solve_item<3>(cl, part, slot, w, res); break;
      default: solve_item<4>(cl, part, slot, w, res); break;
    }
    cl.sync();   // every block's writes to x are done before the flag is raised
    if (rank == 0 && threadIdx.x == 0) {
      results[task % cap] = res;
      __threadfence_system();
      cuda::atomic_ref<unsigned, cuda::thread_scope_system> d(done[task % cap]);
      d.store(1u, cuda::memory_order_release);
    }
  }
}

int server_max_clusters(int csize) {
  if (csize > 8 && cudaFuncSetAttribute(k_server, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
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
  return cudaOccupancyMaxActiveClusters(&n, k_server, &cfg) == cudaSuccess ? n : 0;
}

}  // namespace
}  // namespace pcgk

using namespace pcgk;

namespace {

struct Request {
  uint64_t ticket;
  pcg_matrix A;                     // host arrays, kept by the request until admitted
  std::vector<double> b;
  std::vector<int32_t> row_ptr, col;
  std::vector<double> val, diag, ax, ay, az;
  double tol, sigma;
  int method, maxit, family;
  int mode;                         // 0 binary64, 1 + Jacobi, 2 mixed, 3 mixed + Jacobi
  std::vector<double> dinv;         // Jacobi: D^{-1}
  long long n, nnz;
  size_t bytes;                     // arena bytes
  size_t arena_off = 0;
  long long ring = -1;              // work-item index once published
};

}  // namespace

struct pcg_server {
  std::mutex mu;
  int device = 0;
  size_t budget = 0;
  int max_slots = 0;
  unsigned cap = 0;                 // ring capacity
  int csize = 2;
  int clusters = 0;
  char* arena = nullptr;            // device
  std::map<size_t, size_t> free_blocks;   // offset -> size (first fit, coalesced)
  ServerShared* sh = nullptr;       // mapped host
  ServerShared* d_sh = nullptr;
  WorkItem* items = nullptr;        // mapped host
  WorkItem* d_items = nullptr;
  unsigned* done = nullptr;         // mapped host
  unsigned* d_done = nullptr;
  BatchOut* results = nullptr;      // mapped host
  BatchOut* d_results = nullptr;
  unsigned* d_claim = nullptr;      // device: items taken
  unsigned* d_left = nullptr;       // device: clusters still running
  std::vector<char> occupied;       // ring slot holds an item that was not polled yet
  cudaStream_t kstream = nullptr, cstream = nullptr;
  uint64_t next_ticket = 1;
  unsigned published = 0;
  std::deque<Request*> waiting;                 // not yet admitted
  std::map<uint64_t, Request*> inflight;        // admitted, not yet polled
  std::map<uint64_t, Request*> all;
};

namespace {

bool arena_alloc(pcg_server* S, size_t bytes, size_t* off) {
  for (auto it = S->free_blocks.begin(); it != S->free_blocks.end(); ++it) {
    if (it->second >= bytes) {
      *off = it->first;
      const size_t rest = it->second - bytes;
      const size_t o = it->first + bytes;
      S->free_blocks.erase(it);
      if (rest) S->free_blocks[o] = rest;
      return true;
    }
  }
  return false;
}

void arena_free(pcg_server* S, size_t off, size_t bytes) {
  auto it = S->free_blocks.emplace(off, bytes).first;
  auto nx = std::next(it);
  if (nx != S->free_blocks.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    S->free_blocks.erase(nx);
  }
  if (it != S->free_blocks.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      S->free_blocks.erase(it);
    }
  }
}

size_t pad256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t request_bytes(const Request& R) {
  const size_t n = (size_t)R.n, npad = (n + 31) & ~(size_t)31;
  const bool jac = R.mode & 1, mixed = R.mode >= 2;
  size_t b = (jac ? 16 : 8) * npad * sizeof(double);   // b, x, r, w0, w1, z, s, p (+ Jacobi vectors)
  if (R.family == 4) b += pad256((n + 1) * 4) + pad256(R.nnz * 4) + pad256(R.nnz * 8) + (mixed ? pad256(R.nnz * 4) : 0);
  if (R.family == 1 || R.family == 3) b += 4 * pad256(n * 8) + (mixed ? 4 * pad256(n * 4) : 0);
  return b;
}

int family_of(const pcg_matrix& A) {
  if (A.layout == PCG_CSR32) return 4;
  if (A.layout == PCG_STENCIL5_2D) return A.diag ? 1 : 0;
  if (A.layout == PCG_STENCIL7_3D) return A.diag ? 3 : 2;
  return -1;
}

// Places the request's data in its arena block and fills its work item.
pcg_status upload(pcg_server* S, Request* R, WorkItem* w) {
  char* base = S->arena + R->arena_off;
  const size_t n = (size_t)R->n, npad = (n + 31) & ~(size_t)31;
  const bool jac = R->mode & 1, mixed = R->mode >= 2;
  double* v = (double*)base;
  size_t at = (jac ? 16 : 8) * npad * sizeof(double);
  std::deque<std::vector<float>> stage;   // binary32 copies, alive until the final synchronisation
  auto put32 = [&](const double* src, size_t count) -> const float* {
    stage.emplace_back(count ? count : 1);
    std::vector<float>& f = stage.back();
    for (size_t i = 0; i < count; ++i) f[i] = (float)src[i];
    const void* dst = base + at;
    at += pad256(count * 4);
    if (count && cudaMemcpyAsync((void*)dst, f.data(), count * 4, cudaMemcpyHostToDevice, S->cstream) != cudaSuccess)
      return nullptr;
    return (const float*)dst;
  };
  auto put = [&](const void* src, size_t bytes) -> void* {
    void* dst = base + at;
    at += pad256(bytes);
    if (bytes && cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, S->cstream) != cudaSuccess) return nullptr;
    return dst;
  };
  BatchSys d{};
  d.layout = R->A.layout;
  d.n = (int)R->n;
  d.off = 0;
  d.sigma = R->method == PCG_SPCG ? R->sigma : 0.0;
  if (R->family == 4) {
    d.row_ptr = (const int*)put(R->row_ptr.data(), (n + 1) * 4);
    d.col = (const int*)put(R->col.data(), R->nnz * 4);
    d.val = (const double*)put(R->val.data(), R->nnz * 8);
    if (!d.row_ptr || !d.col || !d.val) return PCG_ECUDA;
    if (mixed && !(d.val32 = put32(R->val.data(), R->nnz))) return PCG_ECUDA;
  } else {
    d.nx = (int)R->A.nx;
    d.ny = (int)R->A.ny;
    d.nz = R->A.layout == PCG_STENCIL7_3D ? (int)R->A.nz : 1;
    if (R->family == 1 || R->family == 3) {
      d.diag = (const double*)put(R->diag.data(), n * 8);
      d.ax = (const double*)put(R->ax.data(), n * 8);
      d.ay = (const double*)put(R->ay.data(), n * 8);
      d.az = R->family == 3 ? (const double*)put(R->az.data(), n * 8) : nullptr;
      if (mixed) {
        d.diag32 = put32(R->diag.data(), n);
        d.ax32 = put32(R->ax.data(), n);
        d.ay32 = put32(R->ay.data(), n);
        d.az32 = R->family == 3 ? put32(R->az.data(), n) : nullptr;
        if (!d.diag32 || !d.ax32 || !d.ay32 || (R->family == 3 && !d.az32)) return PCG_ECUDA;
      }
    }
  }
  if (cudaMemcpyAsync(v, R->b.data(), n * 8, cudaMemcpyHostToDevice, S->cstream) != cudaSuccess) return PCG_ECUDA;
  if (jac) {
    if (cudaMemcpyAsync(v + 14 * npad, R->dinv.data(), n * 8, cudaMemcpyHostToDevice, S->cstream) != cudaSuccess)
      return PCG_ECUDA;
    stage.emplace_back(n);
    std::vector<float>& f = stage.back();
    for (size_t i = 0; i < n; ++i) f[i] = (float)R->dinv[i];
    if (cudaMemcpyAsync(v + 15 * npad, f.data(), n * 4, cudaMemcpyHostToDevice, S->cstream) != cudaSuccess)
      return PCG_ECUDA;
  }
  if (cudaStreamSynchronize(S->cstream) != cudaSuccess) return PCG_ECUDA;
  w->family = R->family;
  w->maxit = R->maxit;
  w->mode = R->mode;
  w->max_restarts = 200;
  w->eta = 1.0 / 1024.0;
  w->tol = R->tol;
  w->sys = d;
  w->vec.b = v;
  w->vec.x = v + npad;
  w->vec.r = v + 2 * npad;
  w->vec.w0 = v + 3 * npad;
  w->vec.w1 = v + 4 * npad;
  w->vec.z = v + 5 * npad;
  w->vec.s = v + 6 * npad;
  w->vec.p = v + 7 * npad;
  w->vec.u = w->vec.q = w->vec.t = w->vec.m0 = w->vec.m1 = w->vec.u64 = nullptr;
  w->vec.dinv = w->vec.dinv32 = nullptr;
  if (jac) {
    w->vec.u = v + 8 * npad;
    w->vec.q = v + 9 * npad;
    w->vec.t = v + 10 * npad;
    w->vec.m0 = v + 11 * npad;
    w->vec.m1 = v + 12 * npad;
    w->vec.u64 = v + 13 * npad;
    w->vec.dinv = v + 14 * npad;
    w->vec.dinv32 = v + 15 * npad;
  }
  return PCG_OK;
}

pcg_status launch_server(pcg_server* S) {
  const unsigned left = (unsigned)S->clusters;
  if (cudaMemcpyAsync(S->d_left, &left, sizeof(unsigned), cudaMemcpyHostToDevice, S->kstream) != cudaSuccess)
    return PCG_ECUDA;
  if (cudaStreamSynchronize(S->kstream) != cudaSuccess) return PCG_ECUDA;
  S->sh->stop = 0;
  cuda::atomic_ref<unsigned, cuda::thread_scope_system> live(S->sh->live);
  live.store(1u, cuda::memory_order_release);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(S->clusters * S->csize);
  cfg.blockDim = dim3(kBlock);
  cfg.stream = S->kstream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = S->csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, k_server, S->d_sh, (const WorkItem*)S->d_items, S->d_results, S->d_done, S->cap,
                         S->d_claim, S->d_left) != cudaSuccess) {
    cudaGetLastError();
    live.store(0u, cuda::memory_order_release);
    return PCG_ECUDA;
  }
  return PCG_OK;
}

// Admits waiting requests (FIFO) while memory and ring slots allow; publishes them;
// makes sure a kernel runs while published work is unclaimed.
pcg_status pump(pcg_server* S) {
  while (!S->waiting.empty()) {
    Request* R = S->waiting.front();
    if ((int)S->inflight.size() >= S->max_slots) break;
    if (S->occupied[S->published % S->cap]) break;   // its ring slot still holds an unpolled request
    size_t off;
    if (!arena_alloc(S, R->bytes, &off)) break;
    R->arena_off = off;
    const unsigned idx = S->published;
    WorkItem w;
    pcg_status s = upload(S, R, &w);
    if (s != PCG_OK) {
      arena_free(S, off, R->bytes);
      return s;
    }
    S->items[idx % S->cap] = w;
    S->done[idx % S->cap] = 0;
    S->occupied[idx % S->cap] = 1;
    R->ring = idx;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    cuda::atomic_ref<unsigned, cuda::thread_scope_system> tail(S->sh->tail);
    tail.store(idx + 1, cuda::memory_order_release);
    S->published = idx + 1;
    S->waiting.pop_front();
    S->inflight[R->ticket] = R;
    // host copies of the operator are no longer needed
    R->row_ptr.clear(); R->row_ptr.shrink_to_fit();
    R->col.clear(); R->col.shrink_to_fit();
    R->val.clear(); R->val.shrink_to_fit();
    R->diag.clear(); R->diag.shrink_to_fit();
    R->ax.clear(); R->ax.shrink_to_fit();
    R->ay.clear(); R->ay.shrink_to_fit();
    R->az.clear(); R->az.shrink_to_fit();
    R->b.clear(); R->b.shrink_to_fit();
    R->dinv.clear(); R->dinv.shrink_to_fit();
  }
  cuda::atomic_ref<unsigned, cuda::thread_scope_system> live(S->sh->live);
  if (S->published > S->sh->claimed && live.load(cuda::memory_order_acquire) == 0) {
    // the previous kernel (if any) has exited: wait for its stream, then relaunch
    if (cudaStreamSynchronize(S->kstream) != cudaSuccess) return PCG_ECUDA;
    return launch_server(S);
  }
  return PCG_OK;
}

}  // namespace

extern "C" {

pcg_status pcg_server_create(size_t hbm_budget_bytes, int32_t max_slots, pcg_server** out) {
  if (!out) return PCG_EINVAL;
  *out = nullptr;
  if (hbm_budget_bytes < (1u << 20) || max_slots < 1 || max_slots > (1 << 20)) return PCG_EINVAL;
  pcg_server* S = new (std::nothrow) pcg_server();
  if (!S) return PCG_ENOMEM;
  auto bail = [&](pcg_status s) {
    pcg_server_destroy(S);
    return s;
  };
  if (cudaGetDevice(&S->device) != cudaSuccess) return bail(PCG_ECUDA);
  S->budget = hbm_budget_bytes & ~(size_t)255;
  S->max_slots = max_slots;
  S->cap = (unsigned)(4 * max_slots);
  S->occupied.assign(S->cap, 0);
  void* p;
  if (cudaMalloc(&p, S->budget) != cudaSuccess) {
    cudaGetLastError();
    return bail(PCG_ENOMEM);
  }
  S->arena = (char*)p;
  S->free_blocks[0] = S->budget;
  if (cudaHostAlloc(&p, sizeof(ServerShared), cudaHostAllocMapped) != cudaSuccess) return bail(PCG_ENOMEM);
  S->sh = (ServerShared*)p;
  memset(S->sh, 0, sizeof(ServerShared));
  if (cudaHostGetDevicePointer((void**)&S->d_sh, S->sh, 0) != cudaSuccess) return bail(PCG_ECUDA);
  if (cudaHostAlloc(&p, S->cap * sizeof(WorkItem), cudaHostAllocMapped) != cudaSuccess) return bail(PCG_ENOMEM);
  S->items = (WorkItem*)p;
  if (cudaHostGetDevicePointer((void**)&S->d_items, S->items, 0) != cudaSuccess) return bail(PCG_ECUDA);
  if (cudaHostAlloc(&p, S->cap * sizeof(unsigned), cudaHostAllocMapped) != cudaSuccess) return bail(PCG_ENOMEM);
  S->done = (unsigned*)p;
  memset(S->done, 0, S->cap * sizeof(unsigned));
  if (cudaHostGetDevicePointer((void**)&S->d_done, S->done, 0) != cudaSuccess) return bail(PCG_ECUDA);
  if (cudaHostAlloc(&p, S->cap * sizeof(BatchOut), cudaHostAllocMapped) != cudaSuccess) return bail(PCG_ENOMEM);
  S->results = (BatchOut*)p;
  if (cudaHostGetDevicePointer((void**)&S->d_results, S->results, 0) != cudaSuccess) return bail(PCG_ECUDA);
  if (cudaMalloc(&p, 2 * sizeof(unsigned)) != cudaSuccess) return bail(PCG_ENOMEM);
  S->d_claim = (unsigned*)p;
  S->d_left = S->d_claim + 1;
  if (cudaMemset(S->d_claim, 0, 2 * sizeof(unsigned)) != cudaSuccess) return bail(PCG_ECUDA);
  if (cudaStreamCreateWithFlags(&S->kstream, cudaStreamNonBlocking) != cudaSuccess) return bail(PCG_ECUDA);
  if (cudaStreamCreateWithFlags(&S->cstream, cudaStreamNonBlocking) != cudaSuccess) return bail(PCG_ECUDA);
  const int mc = server_max_clusters(S->csize);
  if (mc <= 0) return bail(PCG_ECUDA);
  S->clusters = mc;
  *out = S;
  return PCG_OK;
}

void pcg_server_destroy(pcg_server* S) {
  if (!S) return;
  if (S->sh) {
    cuda::atomic_ref<unsigned, cuda::thread_scope_system> stop(S->sh->stop);
    stop.store(1u, cuda::memory_order_release);
  }
  if (S->kstream) cudaStreamSynchronize(S->kstream);
  if (S->cstream) cudaStreamSynchronize(S->cstream);
  for (auto& kv : S->all) delete kv.second;
  if (S->arena) cudaFree(S->arena);
  if (S->d_claim) cudaFree(S->d_claim);
  if (S->sh) cudaFreeHost(S->sh);
  if (S->items) cudaFreeHost(S->items);
  if (S->done) cudaFreeHost(S->done);
  if (S->results) cudaFreeHost(S->results);
  if (S->kstream) cudaStreamDestroy(S->kstream);
  if (S->cstream) cudaStreamDestroy(S->cstream);
  cudaGetLastError();
  delete S;
}

pcg_status pcg_submit(pcg_server* S, const pcg_matrix* A, const double* b, double tol, int32_t method, double sigma,
                      int32_t maxit, uint64_t* ticket) {
  return pcg_submit_ex(S, A, b, tol, method, sigma, maxit, 0, PCG_FP64, ticket);
}

pcg_status pcg_submit_ex(pcg_server* S, const pcg_matrix* A, const double* b, double tol, int32_t method,
                         double sigma, int32_t maxit, uint32_t flags, int32_t precision, uint64_t* ticket) {
  if (!S || !A || !b || !ticket) return PCG_EINVAL;
  if (method != PCG_PCG && method != PCG_SPCG) return PCG_EINVAL;
  if ((flags & ~PCG_JACOBI) || (precision != PCG_FP64 && precision != PCG_MIXED_IR)) return PCG_EINVAL;
  if (!(tol >= 0.0) || !isfinite(tol) || maxit < 0 || !isfinite(sigma)) return PCG_EINVAL;
  const int fam = family_of(*A);
  if (fam < 0) return PCG_EINVAL;
  Request* R = new (std::nothrow) Request();
  if (!R) return PCG_ENOMEM;
  R->A = *A;
  R->family = fam;
  R->tol = tol;
  R->method = method;
  R->maxit = maxit;
  R->mode = (precision == PCG_MIXED_IR ? 2 : 0) + ((flags & PCG_JACOBI) ? 1 : 0);
  const bool jac = (flags & PCG_JACOBI) != 0;
  long long n;
  double diag_sum = 0.0;
  if (fam == 4) {
    if (A->n < 1 || A->n > INT32_MAX - 64 || A->nnz < 0 || A->nnz > INT32_MAX || !A->row_ptr || !A->col || !A->val ||
        A->row_ptr[0] != 0 || A->row_ptr[A->n] != A->nnz) {
      delete R;
      return PCG_EINVAL;
    }
    n = A->n;
    R->nnz = A->nnz;
    R->row_ptr.assign(A->row_ptr, A->row_ptr + n + 1);
    R->col.assign(A->col, A->col + A->nnz);
    R->val.assign(A->val, A->val + A->nnz);
    for (long long i = 0; i < n; ++i)
      for (int k = A->row_ptr[i]; k < A->row_ptr[i + 1]; ++k) {
        if (A->col[k] < 0 || A->col[k] >= n) {
          delete R;
          return PCG_EINVAL;
        }
        if (A->col[k] == i) diag_sum += A->val[k];
      }
  } else {
    const long long nz = A->layout == PCG_STENCIL7_3D ? A->nz : 1;
    if (A->nx < 1 || A->ny < 1 || nz < 1 || A->nx * A->ny * nz > INT32_MAX - 64) {
      delete R;
      return PCG_EINVAL;
    }
    n = A->nx * A->ny * nz;
    if (fam == 1 || fam == 3) {
      if (!A->ax || !A->ay || (fam == 3 && !A->az)) {
        delete R;
        return PCG_EINVAL;
      }
      R->diag.assign(A->diag, A->diag + n);
      R->ax.assign(A->ax, A->ax + n);
      R->ay.assign(A->ay, A->ay + n);
      if (fam == 3) R->az.assign(A->az, A->az + n);
      for (long long i = 0; i < n; ++i) diag_sum += A->diag[i];
    } else {
      diag_sum = (double)n * (fam == 2 ? 6.0 : 4.0);
    }
  }
  R->n = n;
  if (jac) {
    // D^{-1}: the diagonal as for pcg_create(..., PCG_JACOBI)
    R->dinv.resize(n);
    for (long long i = 0; i < n; ++i) {
      double dg;
      if (fam == 4) {
        dg = 0.0;
        for (int k = A->row_ptr[i]; k < A->row_ptr[i + 1]; ++k)
          if (A->col[k] == i) dg += A->val[k];
      } else if (fam == 1 || fam == 3) {
        dg = A->diag[i];
      } else {
        dg = fam == 2 ? 6.0 : 4.0;
      }
      if (!(dg > 0.0) || !isfinite(dg)) {
        delete R;
        return PCG_EINVAL;
      }
      R->dinv[i] = 1.0 / dg;
    }
  }
  // sigma < 0: the mean diagonal entry (for the unscaled Laplacians half the top of
  // the spectrum, the shift Table 1 uses for lapl200)
  // (with Jacobi, of M^{-1} A, which is 1)
  R->sigma = sigma >= 0.0 ? sigma : jac ? 1.0 : diag_sum / (double)n;
  R->b.assign(b, b + n);
  R->bytes = request_bytes(*R);
  std::lock_guard<std::mutex> lock(S->mu);
  if (R->bytes > S->budget) {
    delete R;
    return PCG_ENOMEM;                 // can never be admitted
  }
  if (cudaSetDevice(S->device) != cudaSuccess) {
    delete R;
    return PCG_ECUDA;
  }
  R->ticket = S->next_ticket++;
  S->all[R->ticket] = R;
  S->waiting.push_back(R);
  *ticket = R->ticket;
  return pump(S);
}

pcg_status pcg_poll(pcg_server* S, uint64_t ticket, double* x_out, pcg_result* res) {
  if (!S) return PCG_EINVAL;
  std::lock_guard<std::mutex> lock(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return PCG_EINVAL;
  Request* R = it->second;
  if (cudaSetDevice(S->device) != cudaSuccess) return PCG_ECUDA;
  pcg_status s = pump(S);
  if (s != PCG_OK) return s;
  if (R->ring < 0) return PCG_PENDING;
  const unsigned k = (unsigned)(R->ring % S->cap);
  cuda::atomic_ref<unsigned, cuda::thread_scope_system> d(S->done[k]);
  if (d.load(cuda::memory_order_acquire) == 0) return PCG_PENDING;
  const BatchOut o = S->results[k];
  const WorkItem& w = S->items[k];
  if (x_out && cudaMemcpyAsync(x_out, w.vec.x, (size_t)R->n * 8, cudaMemcpyDeviceToHost, S->cstream) != cudaSuccess)
    return PCG_ECUDA;
  if (cudaStreamSynchronize(S->cstream) != cudaSuccess) return PCG_ECUDA;
  const pcg_status code = o.status == ST_CONVERGED ? PCG_OK : o.status == ST_BREAKDOWN ? PCG_EBREAKDOWN : PCG_ENOTCONV;
  if (res) {
    res->iters = o.iters;
    res->status = code;
    res->final_true_relres = o.bnorm > 0 ? o.true_res / o.bnorm : o.true_res;
    res->final_rec_relres = NAN;
  }
  arena_free(S, R->arena_off, R->bytes);
  S->occupied[k] = 0;
  S->inflight.erase(ticket);
  S->all.erase(it);
  delete R;
  s = pump(S);                          // memory came free: admit waiting requests
  if (s != PCG_OK) return s;
  return code;
}

pcg_status pcg_server_stats(pcg_server* S, int64_t* waiting, int64_t* inflight, size_t* free_bytes) {
  if (!S) return PCG_EINVAL;
  std::lock_guard<std::mutex> lock(S->mu);
  if (waiting) *waiting = (int64_t)S->waiting.size();
  if (inflight) *inflight = (int64_t)S->inflight.size();
  if (free_bytes) {
    size_t f = 0;
    for (auto& kv : S->free_blocks) f += kv.second;
    *free_bytes = f;
  }
  return PCG_OK;
}

}  // extern "C"
