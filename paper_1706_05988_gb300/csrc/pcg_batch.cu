// Batched shifted pipelined CG: many independent systems in one persistent launch (host
// side; the kernel is in pcg_batch_kernel.cuh).
//
// Each thread-block cluster takes systems from a device work queue (largest first)
// and runs every iteration of Algorithm 3 for that system itself: the blocks of the
// cluster split the system's unknowns, the dot products reduce warp -> block ->
// cluster through distributed shared memory, and one cluster barrier per iteration
// stands in for the global reduction.  Every block sums the cluster's partials in rank
// order, so all blocks hold identical scalars and take the same stop decision.  Blocks
// of different clusters never wait on each other; the only barrier is the hardware
// cluster barrier.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <numeric>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#define PCG_KERNELS_IMPL
#include "../../include/pcg.h"
#include "pcg_batch_kernel.cuh"

using namespace pcgk;

namespace {

// Systems are grouped into size classes by unknowns; each class has its own work queue
// (largest first), cluster size and kernel launch, and the classes run concurrently on
// their own streams inside one captured CUDA graph.  Large systems then get large
// clusters while small ones keep small clusters, instead of one cluster size for all.
constexpr int kNumClasses = 3;
constexpr long long kClassBound[kNumClasses] = {8192, 65536, 1LL << 40};   // n below the bound

struct SizeClass {
  int nsys = 0;
  int csize = 4;
  int occ = 0;                  // resident blocks per SM of its kernel: 2, 4, or 0 = chosen per launch
  int occ_used = 0;             // the value the last graph was built with
  int* d_order = nullptr;       // the class's systems, largest first (device)
  int* d_next = nullptr;        // queue head (device)
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
};

// Parameters the captured graph was built for.
struct GraphKey {
  int mode = -1, mask = 0;
  int csize[kNumClasses] = {0, 0, 0};
  int occ[kNumClasses] = {0, 0, 0};
  double tol = 0.0, eta = 0.0;
  int maxit = 0, max_restarts = 0;
  bool operator==(const GraphKey& o) const {
    for (int k = 0; k < kNumClasses; ++k)
      if (csize[k] != o.csize[k] || occ[k] != o.occ[k]) return false;
    return mode == o.mode && mask == o.mask && tol == o.tol && eta == o.eta && maxit == o.maxit &&
           max_restarts == o.max_restarts;
  }
};

}  // namespace

static_assert(kScalarLog == PCG_SCALAR_LOG, "scalar log length in pcg.h");

struct pcg_batch {
  int device = 0;
  int family = -1;
  int nsys = 0;
  std::vector<int> n;             // unknowns per system
  std::vector<long long> off;     // offsets in the batch vectors
  long long total = 0;            // padded length of every batch vector
  std::vector<void*> owned;
  std::vector<BatchSys> host_sys;
  BatchSys* d_sys = nullptr;
  SizeClass cls[kNumClasses];
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t graph = nullptr;
  GraphKey graph_key;
  BatchOut* d_out = nullptr;
  double* d_log = nullptr;        // [nsys][2][kScalarLog]: alpha_i, beta_i of the last solve
  double* d_vec = nullptr;        // b, x, r, w0, w1, z, s, p (+ u, q, t, m0, m1, u64, dinv, dinv32)
  bool jacobi = false;
  int precision = PCG_FP64;
  double eta = kClusterMixedEta;  // inner tolerance factor of the mixed-precision restarts
  int max_restarts = 200;
  double* h_stage = nullptr;      // pinned staging of b / x (total doubles)
  cudaStream_t stream = nullptr;
  int tuned = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double last_kernel_ms = 0.0;
};

namespace {

pcg_status balloc(pcg_batch* B, void** p, size_t bytes) {
  if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) {
    cudaGetLastError();
    return PCG_ENOMEM;
  }
  B->owned.push_back(*p);
  return PCG_OK;
}

int family_of(const pcg_matrix& A) {
  if (A.layout == PCG_CSR32) return 4;
  if (A.layout == PCG_STENCIL5_2D) return A.diag ? 1 : 0;
  if (A.layout == PCG_STENCIL7_3D) return A.diag ? 3 : 2;
  return -1;
}

BatchVecs vecs_of(pcg_batch* B) {
  const long long t = B->total;
  double* base = B->d_vec;
  BatchVecs V;
  V.stride = t;
  V.b = base;
  V.x = base + t;
  V.r = base + 2 * t;
  V.w0 = base + 3 * t;
  V.w1 = base + 4 * t;
  V.z = base + 5 * t;
  V.s = base + 6 * t;
  V.p = base + 7 * t;
  V.u = V.q = V.t = V.m0 = V.m1 = V.u64 = nullptr;
  V.dinv = V.dinv32 = nullptr;
  if (B->jacobi) {
    V.u = base + 8 * t;
    V.q = base + 9 * t;
    V.t = base + 10 * t;
    V.m0 = base + 11 * t;
    V.m1 = base + 12 * t;
    V.u64 = base + 13 * t;
    V.dinv = base + 14 * t;
    V.dinv32 = base + 15 * t;
  }
  return V;
}

int mode_of(const pcg_batch* B) { return (B->precision == PCG_MIXED_IR ? BM_MX : BM_FP64) + (B->jacobi ? 1 : 0); }

int max_clusters_of(int fam, int mode, int csize, int occ) {
  return occ == 4 ? batch_max_clusters_occ4(fam, mode, csize) : batch_max_clusters_occ2(fam, mode, csize);
}

// The kernel variant of a size class: as set, or 4 resident blocks per SM when the class
// has more systems than a 2-block grid holds clusters (more warps then pay for the spills
// of the 64-register cap), else 2.
int occ_for(const pcg_batch* B, int mode, const SizeClass& c) {
  if (c.occ == 2 || c.occ == 4) return c.occ;
  const int m2 = max_clusters_of(B->family, mode, c.csize, 2);
  return c.nsys > m2 && max_clusters_of(B->family, mode, c.csize, 4) > 0 ? 4 : 2;
}

// Builds (or reuses) the graph that launches every class in `mask` on its own stream, then
// replays it; records the CUDA-event time of the whole graph.
pcg_status run_batch(pcg_batch* B, int mask, double tol, int maxit) {
  const int mode = mode_of(B);
  GraphKey key;
  key.mode = mode;
  key.mask = mask;
  for (int k = 0; k < kNumClasses; ++k) {
    key.csize[k] = B->cls[k].csize;
    key.occ[k] = B->cls[k].nsys > 0 && ((mask >> k) & 1) ? occ_for(B, mode, B->cls[k]) : 0;
  }
  key.tol = tol;
  key.maxit = maxit;
  key.eta = B->eta;
  key.max_restarts = B->max_restarts;
  if (!B->graph || !(key == B->graph_key)) {
    if (B->graph) {
      cudaGraphExecDestroy(B->graph);
      B->graph = nullptr;
    }
    // grid per class: as many clusters as can be resident (at most one per system).  The
    // largest class is launched first and fills the GPU; the smaller classes' blocks start
    // as its clusters run out of systems, so they fill its tail.
    int clusters[kNumClasses] = {0, 0, 0};
    for (int k = 0; k < kNumClasses; ++k) {
      const SizeClass& c = B->cls[k];
      if (!((mask >> k) & 1) || c.nsys == 0) continue;
      const int maxc = max_clusters_of(B->family, mode, c.csize, key.occ[k]);
      if (maxc <= 0) {
        cudaGetLastError();
        return PCG_ECUDA;
      }
      clusters[k] = std::min(maxc, c.nsys);
    }
    BatchParams prm;
    prm.tol = tol;
    prm.maxit = maxit;
    prm.eta = B->eta;
    prm.max_restarts = B->max_restarts;
    const BatchVecs V = vecs_of(B);
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return PCG_ECUDA;
    cudaError_t e = cudaEventRecord(B->fork, B->stream);
    for (int kk = kNumClasses - 1; kk >= 0 && e == cudaSuccess; --kk) {   // largest class first
      const int k = kk;
      SizeClass& c = B->cls[k];
      if (clusters[k] == 0) continue;
      e = cudaStreamWaitEvent(c.stream, B->fork, 0);
      if (e == cudaSuccess) e = cudaMemsetAsync(c.d_next, 0, sizeof(int), c.stream);
      if (e == cudaSuccess)
        e = (key.occ[k] == 4 ? batch_launch_occ4 : batch_launch_occ2)(B->family, mode, clusters[k], c.csize,
                                                                       c.stream, B->d_sys, c.d_order, c.nsys,
                                                                       c.d_next, V, B->d_out, prm);
      if (e == cudaSuccess) e = cudaEventRecord(c.done, c.stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(B->stream, c.done, 0);
    }
    const cudaError_t ee = cudaStreamEndCapture(B->stream, &g);
    if (e != cudaSuccess || ee != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return PCG_ECUDA;
    }
    e = cudaGraphInstantiate(&B->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      B->graph = nullptr;
      cudaGetLastError();
      return PCG_ECUDA;
    }
    B->graph_key = key;
    for (int k = 0; k < kNumClasses; ++k)
      if (key.occ[k]) B->cls[k].occ_used = key.occ[k];
  }
  if (cudaEventRecord(B->e0, B->stream) != cudaSuccess) return PCG_ECUDA;
  if (cudaGraphLaunch(B->graph, B->stream) != cudaSuccess) {
    cudaGetLastError();
    return PCG_ECUDA;
  }
  if (cudaEventRecord(B->e1, B->stream) != cudaSuccess) return PCG_ECUDA;
  if (cudaStreamSynchronize(B->stream) != cudaSuccess) return PCG_ECUDA;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, B->e0, B->e1);
  B->last_kernel_ms = ms;
  return PCG_OK;
}

int all_classes(const pcg_batch* B) {
  int m = 0;
  for (int k = 0; k < kNumClasses; ++k)
    if (B->cls[k].nsys > 0) m |= 1 << k;
  return m;
}

}  // namespace

extern "C" {

pcg_status pcg_batch_create(const pcg_matrix* systems, int32_t nsys, uint32_t flags, pcg_batch** out) {
  if (!out) return PCG_EINVAL;
  *out = nullptr;
  if (!systems || nsys < 1 || (flags & ~PCG_JACOBI)) return PCG_EINVAL;
  const int fam = family_of(systems[0]);
  if (fam < 0) return PCG_EINVAL;
  pcg_batch* B = new (std::nothrow) pcg_batch();
  if (!B) return PCG_ENOMEM;
  auto bail = [&](pcg_status s) {
    pcg_batch_destroy(B);
    return s;
  };
  B->family = fam;
  B->nsys = nsys;
  B->jacobi = (flags & PCG_JACOBI) != 0;
  if (cudaGetDevice(&B->device) != cudaSuccess) return bail(PCG_ECUDA);
  long long total = 0;
  for (int k = 0; k < nsys; ++k) {
    const pcg_matrix& A = systems[k];
    if (family_of(A) != fam) return bail(PCG_EINVAL);   // one operator family per batch
    long long n;
    if (fam == 4) {
      if (A.n < 1 || A.n > INT32_MAX || A.nnz < 0 || A.nnz > INT32_MAX || !A.row_ptr || !A.col || !A.val)
        return bail(PCG_EINVAL);
      if (A.row_ptr[0] != 0 || A.row_ptr[A.n] != A.nnz) return bail(PCG_EINVAL);
      for (long long i = 0; i < A.nnz; ++i)
        if (A.col[i] < 0 || A.col[i] >= A.n) return bail(PCG_EINVAL);
      n = A.n;
    } else {
      const long long nz = A.layout == PCG_STENCIL7_3D ? A.nz : 1;
      if (A.nx < 1 || A.ny < 1 || nz < 1) return bail(PCG_EINVAL);
      n = A.nx * A.ny * nz;
      if ((fam == 1 || fam == 3) && (!A.ax || !A.ay || (fam == 3 && !A.az))) return bail(PCG_EINVAL);
    }
    if (n > INT32_MAX - 64) return bail(PCG_EINVAL);
    B->n.push_back((int)n);
    B->off.push_back(total);
    total += (n + 31) & ~31LL;
  }
  B->total = total;
  // device copies of every operator's arrays
  B->host_sys.resize(nsys);
  for (int k = 0; k < nsys; ++k) {
    const pcg_matrix& A = systems[k];
    BatchSys d{};
    d.layout = A.layout;
    d.n = B->n[k];
    d.off = B->off[k];
    auto put = [&](const void* src, size_t bytes, const void** dst) -> pcg_status {
      void* p;
      pcg_status s = balloc(B, &p, bytes);
      if (s != PCG_OK) return s;
      if (cudaMemcpy(p, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return PCG_ECUDA;
      *dst = p;
      return PCG_OK;
    };
    // binary32 copy (round to nearest) for the mixed-precision inner iteration
    auto put32 = [&](const double* src, long long count, const float** dst) -> pcg_status {
      std::vector<float> f(count > 0 ? count : 1);
      for (long long i = 0; i < count; ++i) f[i] = (float)src[i];
      return put(f.data(), f.size() * sizeof(float), (const void**)dst);
    };
    pcg_status s = PCG_OK;
    if (fam == 4) {
      s = put(A.row_ptr, (A.n + 1) * sizeof(int), (const void**)&d.row_ptr);
      if (s == PCG_OK) s = put(A.col, A.nnz * sizeof(int), (const void**)&d.col);
      if (s == PCG_OK) s = put(A.val, A.nnz * sizeof(double), (const void**)&d.val);
      if (s == PCG_OK) s = put32(A.val, A.nnz, &d.val32);
    } else {
      d.nx = (int)A.nx;
      d.ny = (int)A.ny;
      d.nz = A.layout == PCG_STENCIL7_3D ? (int)A.nz : 1;
      if (fam == 1 || fam == 3) {
        s = put(A.diag, d.n * sizeof(double), (const void**)&d.diag);
        if (s == PCG_OK) s = put(A.ax, d.n * sizeof(double), (const void**)&d.ax);
        if (s == PCG_OK) s = put(A.ay, d.n * sizeof(double), (const void**)&d.ay);
        if (s == PCG_OK && fam == 3) s = put(A.az, d.n * sizeof(double), (const void**)&d.az);
        if (s == PCG_OK) s = put32(A.diag, d.n, &d.diag32);
        if (s == PCG_OK) s = put32(A.ax, d.n, &d.ax32);
        if (s == PCG_OK) s = put32(A.ay, d.n, &d.ay32);
        if (s == PCG_OK && fam == 3) s = put32(A.az, d.n, &d.az32);
      }
    }
    if (s != PCG_OK) return bail(s);
    B->host_sys[k] = d;
  }
  void* p;
  if (balloc(B, &p, (size_t)nsys * 2 * kScalarLog * sizeof(double)) != PCG_OK) return bail(PCG_ENOMEM);
  B->d_log = (double*)p;
  if (cudaMemset(B->d_log, 0xFF, (size_t)nsys * 2 * kScalarLog * sizeof(double)) != cudaSuccess)   // NaN
    return bail(PCG_ECUDA);
  for (int k = 0; k < nsys; ++k) B->host_sys[k].log = B->d_log + (size_t)k * 2 * kScalarLog;
  if (balloc(B, &p, nsys * sizeof(BatchSys)) != PCG_OK) return bail(PCG_ENOMEM);
  B->d_sys = (BatchSys*)p;
  if (balloc(B, &p, nsys * sizeof(BatchOut)) != PCG_OK) return bail(PCG_ENOMEM);
  B->d_out = (BatchOut*)p;
  const int nvec = B->jacobi ? 16 : 8;
  if (balloc(B, &p, nvec * (size_t)total * sizeof(double)) != PCG_OK) return bail(PCG_ENOMEM);
  B->d_vec = (double*)p;
  if (cudaMallocHost(&p, (size_t)total * sizeof(double)) != cudaSuccess) return bail(PCG_ENOMEM);
  B->h_stage = (double*)p;
  if (B->jacobi) {
    // D^{-1} of every system (binary64, and rounded to binary32 in a binary32 slot)
    const BatchVecs V = vecs_of(B);
    std::fill(B->h_stage, B->h_stage + total, 0.0);
    for (int k = 0; k < nsys; ++k) {
      const pcg_matrix& A = systems[k];
      double* dk = B->h_stage + B->off[k];
      const int n = B->n[k];
      for (int i = 0; i < n; ++i) {
        double dg;
        if (fam == 4) {
          dg = 0.0;
          for (int32_t e = A.row_ptr[i]; e < A.row_ptr[i + 1]; ++e)
            if (A.col[e] == i) dg += A.val[e];
        } else if (fam == 1 || fam == 3) {
          dg = A.diag[i];
        } else {
          dg = fam == 2 ? 6.0 : 4.0;
        }
        if (!(dg > 0.0) || !isfinite(dg)) return bail(PCG_EINVAL);   // Jacobi needs a positive diagonal
        dk[i] = 1.0 / dg;
      }
    }
    if (cudaMemcpy((double*)V.dinv, B->h_stage, (size_t)total * sizeof(double), cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return bail(PCG_ECUDA);
    std::vector<double> slot32(total, 0.0);
    for (int k = 0; k < nsys; ++k) {
      float* f = reinterpret_cast<float*>(slot32.data() + B->off[k]);
      for (int i = 0; i < B->n[k]; ++i) f[i] = (float)B->h_stage[B->off[k] + i];
    }
    if (cudaMemcpy((double*)V.dinv32, slot32.data(), (size_t)total * sizeof(double), cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return bail(PCG_ECUDA);
  }
  // size classes, each with its queue ordered largest first (the queue then balances the
  // clusters' work), its own stream and a default cluster size growing with the class
  std::vector<int> order(nsys);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return B->n[a] > B->n[b]; });
  if (cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(PCG_ECUDA);
  if (cudaEventCreate(&B->e0) != cudaSuccess || cudaEventCreate(&B->e1) != cudaSuccess) return bail(PCG_ECUDA);
  if (cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) != cudaSuccess) return bail(PCG_ECUDA);
  static const int kDefaultCluster[kNumClasses] = {2, 4, 8};
  for (int c = 0; c < kNumClasses; ++c) {
    SizeClass& sc = B->cls[c];
    const long long lo = c == 0 ? 0 : kClassBound[c - 1];
    std::vector<int> mine;
    for (int k : order)
      if (B->n[k] >= lo && B->n[k] < kClassBound[c]) mine.push_back(k);
    sc.nsys = (int)mine.size();
    sc.csize = kDefaultCluster[c];
    if (balloc(B, &p, (mine.empty() ? 1 : mine.size()) * sizeof(int)) != PCG_OK) return bail(PCG_ENOMEM);
    sc.d_order = (int*)p;
    if (!mine.empty() &&
        cudaMemcpy(sc.d_order, mine.data(), mine.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(PCG_ECUDA);
    if (balloc(B, &p, sizeof(int)) != PCG_OK) return bail(PCG_ENOMEM);
    sc.d_next = (int*)p;
    if (cudaStreamCreateWithFlags(&sc.stream, cudaStreamNonBlocking) != cudaSuccess) return bail(PCG_ECUDA);
    if (cudaEventCreateWithFlags(&sc.done, cudaEventDisableTiming) != cudaSuccess) return bail(PCG_ECUDA);
  }
  *out = B;
  return PCG_OK;
}

void pcg_batch_destroy(pcg_batch* B) {
  if (!B) return;
  if (B->stream) cudaStreamSynchronize(B->stream);
  for (void* p : B->owned) cudaFree(p);
  if (B->h_stage) cudaFreeHost(B->h_stage);
  if (B->graph) cudaGraphExecDestroy(B->graph);
  for (SizeClass& sc : B->cls) {
    if (sc.stream) {
      cudaStreamSynchronize(sc.stream);
      cudaStreamDestroy(sc.stream);
    }
    if (sc.done) cudaEventDestroy(sc.done);
  }
  if (B->fork) cudaEventDestroy(B->fork);
  if (B->e0) cudaEventDestroy(B->e0);
  if (B->e1) cudaEventDestroy(B->e1);
  if (B->stream) cudaStreamDestroy(B->stream);
  cudaGetLastError();
  delete B;
}

pcg_status pcg_batch_solve(pcg_batch* B, const double* const* b, double* const* x_out, int32_t method,
                           const double* sigma, double tol, int32_t maxit, int32_t* iters, int32_t* status,
                           double* true_relres) {
  if (!B || !b || !x_out) return PCG_EINVAL;
  if (method != PCG_PCG && method != PCG_SPCG) return PCG_EINVAL;
  if (!(tol >= 0.0) || !isfinite(tol) || maxit < 0) return PCG_EINVAL;
  if (method == PCG_SPCG && !sigma) return PCG_EINVAL;
  for (int k = 0; k < B->nsys; ++k) {
    if (!b[k] || !x_out[k]) return PCG_EINVAL;
    const double sg = method == PCG_SPCG ? sigma[k] : 0.0;
    if (!(sg >= 0.0) || !isfinite(sg)) return PCG_EINVAL;
    B->host_sys[k].sigma = sg;
  }
  if (cudaSetDevice(B->device) != cudaSuccess) return PCG_ECUDA;
  if (cudaMemcpyAsync(B->d_sys, B->host_sys.data(), B->nsys * sizeof(BatchSys), cudaMemcpyHostToDevice, B->stream) !=
      cudaSuccess)
    return PCG_ECUDA;
  for (int k = 0; k < B->nsys; ++k) std::copy(b[k], b[k] + B->n[k], B->h_stage + B->off[k]);
  const BatchVecs V = vecs_of(B);
  if (cudaMemcpyAsync((double*)V.b, B->h_stage, (size_t)B->total * sizeof(double), cudaMemcpyHostToDevice,
                      B->stream) != cudaSuccess)
    return PCG_ECUDA;
  pcg_status s = run_batch(B, all_classes(B), tol, maxit);
  if (s != PCG_OK) return s;
  if (cudaMemcpyAsync(B->h_stage, V.x, (size_t)B->total * sizeof(double), cudaMemcpyDeviceToHost, B->stream) !=
      cudaSuccess)
    return PCG_ECUDA;
  std::vector<BatchOut> o(B->nsys);
  if (cudaMemcpyAsync(o.data(), B->d_out, B->nsys * sizeof(BatchOut), cudaMemcpyDeviceToHost, B->stream) !=
      cudaSuccess)
    return PCG_ECUDA;
  if (cudaStreamSynchronize(B->stream) != cudaSuccess) return PCG_ECUDA;
  bool all_ok = true;
  for (int k = 0; k < B->nsys; ++k) {
    std::copy(B->h_stage + B->off[k], B->h_stage + B->off[k] + B->n[k], x_out[k]);
    const int st = o[k].status;
    const int code = st == ST_CONVERGED ? PCG_OK : st == ST_BREAKDOWN ? PCG_EBREAKDOWN : PCG_ENOTCONV;
    if (iters) iters[k] = o[k].iters;
    if (status) status[k] = code;
    if (true_relres) true_relres[k] = o[k].bnorm > 0 ? o[k].true_res / o[k].bnorm : o[k].true_res;
    all_ok = all_ok && code == PCG_OK;
  }
  return all_ok ? PCG_OK : PCG_ENOTCONV;
}

pcg_status pcg_batch_autotune(pcg_batch* B, const double* const* b, const double* sigma, int32_t probe_iters,
                              int32_t* cluster_out, double* ms_out) {
  if (!B || !b || !sigma || probe_iters < 1) return PCG_EINVAL;
  std::vector<double*> xs(B->nsys);
  std::vector<std::vector<double>> store(B->nsys);
  for (int k = 0; k < B->nsys; ++k) {
    store[k].resize(B->n[k]);
    xs[k] = store[k].data();
  }
  const int cand[] = {1, 2, 4, 8, 16};
  // 1. one size for every class: the whole batch per candidate (ms_out, cluster_out)
  double best = INFINITY;
  int best_c = B->cls[1].csize;
  int saved[kNumClasses];
  for (int k = 0; k < kNumClasses; ++k) saved[k] = B->cls[k].csize;
  for (int ci = 0; ci < 5; ++ci) {
    const int c = cand[ci];
    for (SizeClass& sc : B->cls) sc.csize = c;
    if (ms_out) ms_out[ci] = NAN;
    pcg_status s = pcg_batch_solve(B, b, xs.data(), PCG_SPCG, sigma, 0.0, probe_iters, nullptr, nullptr, nullptr);
    if (s != PCG_OK && s != PCG_ENOTCONV) continue;   // a shape this GPU cannot launch is skipped
    if (ms_out) ms_out[ci] = B->last_kernel_ms;
    if (B->last_kernel_ms < best) {
      best = B->last_kernel_ms;
      best_c = c;
    }
  }
  if (!std::isfinite(best)) {
    for (int k = 0; k < kNumClasses; ++k) B->cls[k].csize = saved[k];
    return PCG_ECUDA;
  }
  // 2. each size class alone: its fastest cluster size and kernel variant (2 or 4 resident
  //    blocks per SM) -- the per-class shape cache
  for (SizeClass& sc : B->cls) sc.csize = best_c;
  for (int k = 0; k < kNumClasses; ++k) {
    SizeClass& sc = B->cls[k];
    if (sc.nsys == 0) continue;
    const int saved_occ = sc.occ;
    double bk = INFINITY;
    int ck = best_c, ok = saved_occ;
    for (int ci = 0; ci < 5; ++ci) {
      for (int occ : {2, 4}) {
        sc.csize = cand[ci];
        sc.occ = occ;
        pcg_status s = PCG_OK;
        for (int j = 0; j < B->nsys; ++j) B->host_sys[j].sigma = sigma[j];
        if (cudaMemcpyAsync(B->d_sys, B->host_sys.data(), B->nsys * sizeof(BatchSys), cudaMemcpyHostToDevice,
                            B->stream) != cudaSuccess)
          return PCG_ECUDA;
        s = run_batch(B, 1 << k, 0.0, probe_iters);
        if (s != PCG_OK) {
          cudaGetLastError();
          continue;
        }
        if (B->last_kernel_ms < bk) {
          bk = B->last_kernel_ms;
          ck = cand[ci];
          ok = occ;
        }
      }
    }
    sc.csize = ck;
    sc.occ = ok;
  }
  B->tuned = 1;
  if (cluster_out) *cluster_out = best_c;
  return PCG_OK;
}

pcg_status pcg_batch_set_precision(pcg_batch* B, int32_t precision) {
  if (!B || (precision != PCG_FP64 && precision != PCG_MIXED_IR)) return PCG_EINVAL;
  B->precision = precision;
  return PCG_OK;
}

pcg_status pcg_batch_set_param(pcg_batch* B, int32_t param, double value) {
  if (!B) return PCG_EINVAL;
  if (param == PCG_PARAM_MIXED_ETA) {
    if (!(value > 0.0 && value < 1.0)) return PCG_EINVAL;
    B->eta = value;
    return PCG_OK;
  }
  if (param == PCG_PARAM_MAX_RESTARTS) {
    if (!(value >= 1.0 && value <= 1e9)) return PCG_EINVAL;
    B->max_restarts = (int)value;
    return PCG_OK;
  }
  return PCG_EINVAL;
}

pcg_status pcg_batch_classes(const pcg_batch* B, int32_t* nsys, int32_t* cluster, int32_t* blocks_per_sm) {
  if (!B) return PCG_EINVAL;
  for (int k = 0; k < kNumClasses; ++k) {
    if (nsys) nsys[k] = B->cls[k].nsys;
    if (cluster) cluster[k] = B->cls[k].csize;
    if (blocks_per_sm) blocks_per_sm[k] = B->cls[k].occ ? B->cls[k].occ : B->cls[k].occ_used;
  }
  return PCG_OK;
}

pcg_status pcg_batch_set_class_occupancy(pcg_batch* B, int32_t size_class, int32_t blocks_per_sm) {
  if (!B || size_class < 0 || size_class >= kNumClasses) return PCG_EINVAL;
  if (blocks_per_sm != 0 && blocks_per_sm != 2 && blocks_per_sm != 4) return PCG_EINVAL;
  B->cls[size_class].occ = blocks_per_sm;
  return PCG_OK;
}

pcg_status pcg_batch_set_class_cluster(pcg_batch* B, int32_t size_class, int32_t cluster_size) {
  if (!B || size_class < 0 || size_class >= kNumClasses) return PCG_EINVAL;
  if (cluster_size != 1 && cluster_size != 2 && cluster_size != 4 && cluster_size != 8 && cluster_size != 16)
    return PCG_EINVAL;
  B->cls[size_class].csize = cluster_size;
  return PCG_OK;
}

pcg_status pcg_batch_set_cluster(pcg_batch* B, int32_t cluster_size) {
  if (!B) return PCG_EINVAL;
  if (cluster_size != 1 && cluster_size != 2 && cluster_size != 4 && cluster_size != 8 && cluster_size != 16)
    return PCG_EINVAL;
  for (SizeClass& sc : B->cls) sc.csize = cluster_size;
  return PCG_OK;
}

pcg_status pcg_batch_last_kernel_ms(const pcg_batch* B, double* ms) {
  if (!B || !ms) return PCG_EINVAL;
  *ms = B->last_kernel_ms;
  return PCG_OK;
}

pcg_status pcg_batch_scalars(const pcg_batch* B, int32_t k, double* alpha, double* beta) {
  if (!B || k < 1 || k > PCG_SCALAR_LOG || (!alpha && !beta)) return PCG_EINVAL;
  if (cudaSetDevice(B->device) != cudaSuccess) return PCG_ECUDA;
  std::vector<double> h((size_t)B->nsys * 2 * kScalarLog);
  if (cudaStreamSynchronize(B->stream) != cudaSuccess ||
      cudaMemcpy(h.data(), B->d_log, h.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return PCG_ECUDA;
  }
  for (int s = 0; s < B->nsys; ++s) {
    const double* l = h.data() + (size_t)s * 2 * kScalarLog;
    for (int i = 0; i < k; ++i) {
      if (alpha) alpha[(size_t)s * k + i] = l[i];
      if (beta) beta[(size_t)s * k + i] = l[kScalarLog + i];
    }
  }
  return PCG_OK;
}

}  // extern "C"
