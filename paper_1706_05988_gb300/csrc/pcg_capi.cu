// C ABI of libpcg (declared in include/pcg.h): context management, argument
// checking, device memory, and the launch sequence of one solve.  Every
// arithmetic step of a solve runs in the kernels of pcg_kernels.cuh.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "../../include/pcg.h"
#include "pcg_internal.h"
#include "pcg_general.cuh"
#include "pcg_host_parallel.h"

using namespace pcgk;

struct pcg_ctx {
  int device = 0;
  uint32_t flags = 0;
  OpDesc op{};
  int64_t n = 0, nnz = 0;
  std::vector<void*> owned;             // device allocations owned by the context
  cudaStream_t own_stream = nullptr, stream = nullptr;
  // work vectors: x, r, w0, w1, z, s, p, b (internal copy) in one allocation
  double* vec_base = nullptr;
  size_t vec_stride = 0;                // doubles between consecutive vectors
  Vecs v{};
  double* d_b = nullptr;
  State* d_state = nullptr;
  State* h_state = nullptr;             // pinned mirror
  double* d_hist = nullptr;
  int hist_cap = 0;
  Hist h{};
  double* d_partials = nullptr;
  double* d_small = nullptr;            // psi workspace
  int small_cap = 0;
  int grid[K_NKINDS] = {0};
  // mixed precision: binary32 copies of the operator's coefficients, grids, parameters
  bool mixed_ready = false;
  int grid_mx[KM_NKINDS] = {0};
  double mx_eta = 0.0009765625;        // 2^-10
  int mx_max_restarts = 200;
  double true_tol = 0.0;                // PCG_PARAM_TRUE_TOL
  // general iteration (Jacobi M^-1 and/or variable shift)
  double* gen_base = nullptr;           // u, q, p, m (two buffers); t is v.p
  const float* dinv32 = nullptr;        // mixed precision with PCG_JACOBI
  double* mx_u64 = nullptr;             // u_0 widened to binary64 at a restart
  double* d_dinv = nullptr;
  double* d_shifts = nullptr;
  int shifts_cap = 0;
  std::vector<double> var_shifts;       // pcg_set_shifts (empty: constant shift)
  int grid_gen[4] = {0, 0, 0, 0};       // by variant: 2 * jac + var
  // persistent kernel
  int grid_persistent = 0;
  double barrier_timeout_ms = 2000.0;
  unsigned barrier_phantoms = 0;
  int64_t launches = 0, iter_launches = 0;
  double iter_ms = 0.0;
  std::vector<cudaEvent_t> ev;          // PCG_PROFILE: pairs around iteration launches
  // Launch-per-iteration path without profiling: kIterGraphLen launches of the fused
  // iteration kernel captured once as a CUDA graph and replayed (the launches are
  // identical: the iteration index lives in device memory).  Rebuilt when a launch
  // argument changes.
  cudaGraphExec_t iter_graph = nullptr;
  struct IterGraphKey {
    OpDesc op;
    Vecs v;
    Hist h;
    State* st;
    double* partials;
    cudaStream_t stream;
    int grid;
  } iter_key;
  std::string err;
};

namespace {

const char* kVersion = "libpcg 0.2 (sm_103a, FP64 shifted pipelined CG)";

// Depth of the TMA-staged ring of the fused iteration (PCG_PARAM_ITER_STAGES); 0 = the
// register sweep, which is the faster one on GB300 at every size measured.
constexpr int kDefaultIterStages = 0;

pcg_status fail(pcg_ctx* c, pcg_status s, const char* msg) {
  if (c) c->err = msg;
  return s;
}

#define CUDA_TRY(ctx, call)                                                                    \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(e_);                          \
      return e_ == cudaErrorMemoryAllocation ? PCG_ENOMEM : PCG_ECUDA;                         \
    }                                                                                          \
  } while (0)

pcg_status dev_alloc(pcg_ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    c->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? PCG_ENOMEM : PCG_ECUDA;
  }
  c->owned.push_back(*p);
  return PCG_OK;
}

// Copies a matrix array to the device (or references it with PCG_DEVICE_PTRS).
template <class T>
pcg_status place(pcg_ctx* c, const T* src, size_t count, const T** dst) {
  if (c->flags & PCG_DEVICE_PTRS) {
    *dst = src;
    return PCG_OK;
  }
  void* p;
  pcg_status s = dev_alloc(c, &p, count * sizeof(T));
  if (s != PCG_OK) return s;
  CUDA_TRY(c, cudaMemcpy(p, src, count * sizeof(T), cudaMemcpyHostToDevice));
  *dst = (const T*)p;
  return PCG_OK;
}

pcg_status ensure_vectors(pcg_ctx* c) {
  if (c->vec_base) return PCG_OK;
  const size_t stride = ((size_t)c->n + 31) & ~(size_t)31;   // 256-byte aligned vectors
  void* p;
  pcg_status s = dev_alloc(c, &p, 8 * stride * sizeof(double));
  if (s != PCG_OK) return s;
  c->vec_base = (double*)p;
  c->vec_stride = stride;
  double* b = c->vec_base;
  c->v.x = b + 0 * stride;
  c->v.r = b + 1 * stride;
  c->v.w0 = b + 2 * stride;
  c->v.w1 = b + 3 * stride;
  c->v.z = b + 4 * stride;
  c->v.s = b + 5 * stride;
  c->v.p = b + 6 * stride;
  c->d_b = b + 7 * stride;
  c->v.b = c->d_b;
  return PCG_OK;
}

pcg_status ensure_hist(pcg_ctx* c, int entries) {
  if (c->hist_cap >= entries) return PCG_OK;
  if (c->d_hist) {
    cudaFree(c->d_hist);
    c->owned.erase(std::find(c->owned.begin(), c->owned.end(), (void*)c->d_hist));
    c->d_hist = nullptr;
    c->hist_cap = 0;
  }
  const int cap = std::max(entries, 1024);
  void* p;
  pcg_status s = dev_alloc(c, &p, 7 * (size_t)cap * sizeof(double));
  if (s != PCG_OK) return s;
  c->d_hist = (double*)p;
  c->hist_cap = cap;
  double* b = c->d_hist;
  c->h.alpha = b;
  c->h.beta = b + cap;
  c->h.gamma = b + 2 * cap;
  c->h.delta = b + 3 * cap;
  c->h.rec = b + 4 * cap;
  c->h.tru = b + 5 * cap;
  c->h.gap = b + 6 * cap;
  return PCG_OK;
}

pcg_status ensure_events(pcg_ctx* c, size_t pairs) {
  while (c->ev.size() < 2 * pairs) {
    cudaEvent_t e;
    CUDA_TRY(c, cudaEventCreate(&e));
    c->ev.push_back(e);
  }
  return PCG_OK;
}

Launch launch_of(pcg_ctx* c, int kind) { return Launch{c->grid[kind], kBlockThreads, c->stream}; }

}  // namespace

namespace pcgk {
// Readers of the checked build's per-translation-unit failure words (pcg_check.cuh),
// registered by static initialisers when the library loads.
std::vector<unsigned (*)(bool)>& check_readers() {
  static std::vector<unsigned (*)(bool)> readers;
  return readers;
}
void register_check_reader(unsigned (*reader)(bool)) { check_readers().push_back(reader); }
}  // namespace pcgk

extern "C" {

const char* pcg_version(void) { return kVersion; }

pcg_status pcg_check_status(uint32_t* code, int32_t* checked) {
  if (!code) return PCG_EINVAL;
#ifdef PCG_CHECKED
  if (checked) *checked = 1;
#else
  if (checked) *checked = 0;
#endif
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return PCG_ECUDA;
  }
  unsigned first = 0;
  for (auto reader : pcgk::check_readers()) {
    const unsigned v = reader(true);
    if (first == 0) first = v;
  }
  *code = first;
  return PCG_OK;
}

const char* pcg_last_error(const pcg_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

pcg_status pcg_create(const pcg_matrix* A, uint32_t flags, pcg_ctx** out) {
  if (!out) return PCG_EINVAL;
  *out = nullptr;
  if (!A) return PCG_EINVAL;
  if (flags & ~(PCG_DEVICE_PTRS | PCG_PROFILE | PCG_STENCIL_FP64_SUM | PCG_PERSISTENT | PCG_JACOBI | PCG_DOTS_SPLIT32))
    return PCG_EINVAL;
  OpDesc op{};
  op.layout = A->layout;
  op.fixed_sum = (flags & PCG_STENCIL_FP64_SUM) ? 0 : 1;
  op.ff_dots = (flags & PCG_DOTS_SPLIT32) ? 1 : 0;
  op.iter_stages = kDefaultIterStages;
  int64_t n = 0, nnz = 0;
  if (A->layout == PCG_STENCIL5_2D || A->layout == PCG_STENCIL7_3D) {
    const int64_t nz = A->layout == PCG_STENCIL7_3D ? A->nz : 1;
    if (A->nx < 1 || A->ny < 1 || nz < 1) return PCG_EINVAL;
    if (A->nx > INT32_MAX || A->ny > INT32_MAX || nz > INT32_MAX) return PCG_EINVAL;
    n = A->nx * A->ny * nz;
    if (n > (int64_t)INT32_MAX - 64) return PCG_EINVAL;
    const bool var = A->diag != nullptr;
    if (var && (!A->ax || !A->ay || (A->layout == PCG_STENCIL7_3D && !A->az))) return PCG_EINVAL;
    if (!var && (A->ax || A->ay || A->az)) return PCG_EINVAL;
    op.nx = (int)A->nx;
    op.ny = (int)A->ny;
    op.nz = (int)nz;
  } else if (A->layout == PCG_CSR32) {
    if (A->n < 1 || A->n > (int64_t)INT32_MAX - 64 || A->nnz < 0 || A->nnz > INT32_MAX) return PCG_EINVAL;
    if (!A->row_ptr || (A->nnz > 0 && (!A->col || !A->val))) return PCG_EINVAL;
    n = A->n;
    nnz = A->nnz;
    if (!(flags & PCG_DEVICE_PTRS)) {   // host arrays can be validated here
      if (A->row_ptr[0] != 0 || A->row_ptr[n] != nnz) return PCG_EINVAL;
      // every row's range inside [0, nnz] and ordered, every column index in [0, n)
      // (chunks of rows on several threads)
      std::vector<char> bad((size_t)pcgk::host::row_chunks(n), 0);
      pcgk::host::for_chunks((long long)bad.size(), [&](long long ch) {
        const int64_t i1 = std::min<int64_t>(n, (ch + 1) * pcgk::host::kRowsPerChunk);
        for (int64_t i = ch * pcgk::host::kRowsPerChunk; i < i1; ++i) {
          const int64_t beg = A->row_ptr[i], end = A->row_ptr[i + 1];
          if (beg < 0 || end < beg || end > nnz) {
            bad[(size_t)ch] = 1;
            return;
          }
          for (int64_t k = beg; k < end; ++k) {
            if (A->col[k] < 0 || A->col[k] >= n) {
              bad[(size_t)ch] = 1;
              return;
            }
          }
        }
      });
      for (char b : bad)
        if (b) return PCG_EINVAL;
    }
  } else {
    return PCG_EINVAL;
  }
  op.n = (int)n;

  pcg_ctx* c = new (std::nothrow) pcg_ctx();
  if (!c) return PCG_ENOMEM;
  c->flags = flags;
  c->n = n;
  c->nnz = nnz;
  pcg_status s = PCG_OK;
  auto bail = [&](pcg_status st) {
    pcg_destroy(c);
    return st;
  };
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    cudaGetLastError();
    return bail(PCG_ECUDA);
  }
  if (A->layout == PCG_CSR32) {
    if ((s = place<int32_t>(c, A->row_ptr, n + 1, &op.row_ptr)) != PCG_OK) return bail(s);
    if ((s = place<int32_t>(c, A->col, nnz, &op.col)) != PCG_OK) return bail(s);
    if ((s = place<double>(c, A->val, nnz, &op.val)) != PCG_OK) return bail(s);
  } else if (A->diag) {
    if ((s = place<double>(c, A->diag, n, &op.diag)) != PCG_OK) return bail(s);
    if ((s = place<double>(c, A->ax, n, &op.ax)) != PCG_OK) return bail(s);
    if ((s = place<double>(c, A->ay, n, &op.ay)) != PCG_OK) return bail(s);
    if (A->layout == PCG_STENCIL7_3D && (s = place<double>(c, A->az, n, &op.az)) != PCG_OK) return bail(s);
  }
  c->op = op;
  if (cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return bail(PCG_ECUDA);
  }
  c->stream = c->own_stream;
  void* p;
  if ((s = dev_alloc(c, &p, sizeof(State))) != PCG_OK) return bail(s);
  c->d_state = (State*)p;
  if ((s = dev_alloc(c, &p, (size_t)kMaxPartialBlocks * kPartialsPerBlock * sizeof(double))) != PCG_OK) return bail(s);
  c->d_partials = (double*)p;
  if (cudaMallocHost(&p, sizeof(State)) != cudaSuccess) {
    cudaGetLastError();
    return bail(PCG_ENOMEM);
  }
  c->h_state = (State*)p;
  if ((flags & PCG_JACOBI) && (flags & PCG_DEVICE_PTRS)) {
    // M^{-1} = diag(A)^{-1}, formed on the device from the caller's device arrays
    void* p;
    if ((s = dev_alloc(c, &p, (size_t)n * sizeof(double) + 256)) != PCG_OK) return bail(s);
    c->d_dinv = (double*)p;
    int* d_bad = (int*)((char*)p + (size_t)n * sizeof(double));
    int bad = 0;
    if (cudaMemsetAsync(d_bad, 0, sizeof(int), c->stream) != cudaSuccess ||
        launch_jacobi_dinv(c->op, c->d_dinv, d_bad, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
      cudaGetLastError();
      return bail(fail(c, PCG_ECUDA, "could not form the Jacobi diagonal"));
    }
    if (bad) return bail(fail(c, PCG_EINVAL, "PCG_JACOBI needs a positive diagonal"));
  } else if (flags & PCG_JACOBI) {
    // M^{-1} = diag(A)^{-1}, formed on the host from the operator's description
    pcgk::host::buffer<double> dinv((size_t)n);
    std::vector<char> bad((size_t)pcgk::host::row_chunks(n), 0);
    pcgk::host::for_chunks((long long)bad.size(), [&](long long ch) {
      const int64_t i0 = ch * pcgk::host::kRowsPerChunk, i1 = std::min<int64_t>(n, i0 + pcgk::host::kRowsPerChunk);
      for (int64_t i = i0; i < i1; ++i) {
        double d;
        if (A->layout == PCG_CSR32) {
          d = 0.0;
          for (int32_t k = A->row_ptr[i]; k < A->row_ptr[i + 1]; ++k)
            if (A->col[k] == i) d += A->val[k];
        } else if (A->diag) {
          d = A->diag[i];
        } else {
          d = A->layout == PCG_STENCIL7_3D ? 6.0 : 4.0;
        }
        if (!(d > 0.0)) bad[(size_t)ch] = 1;
        dinv[i] = 1.0 / d;
      }
    });
    for (char b : bad)
      if (b) return bail(fail(c, PCG_EINVAL, "PCG_JACOBI needs a positive diagonal"));
    const double* dd = nullptr;
    c->flags &= ~PCG_DEVICE_PTRS;
    if ((s = place<double>(c, dinv.data(), n, &dd)) != PCG_OK) return bail(s);
    c->d_dinv = (double*)dd;
  }
  if (flags & PCG_PERSISTENT) {
    c->grid_persistent = grid_for_persistent(c->op);
    if (c->grid_persistent <= 0) {
      cudaGetLastError();
      return bail(fail(c, PCG_ECUDA, "could not size the persistent grid"));
    }
  }
  c->op.iter_stages = resolve_iter_stages(c->op, c->op.iter_stages);
  for (int k = 0; k < K_NKINDS; ++k) {
    c->grid[k] = grid_for(c->op, k, kBlockThreads);
    if (c->grid[k] <= 0) {
      cudaGetLastError();
      return bail(fail(c, PCG_ECUDA, "could not size the kernel grids"));
    }
  }
  *out = c;
  return PCG_OK;
}

void pcg_destroy(pcg_ctx* c) {
  if (!c) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(c->device);
  if (c->own_stream) cudaStreamSynchronize(c->own_stream);
  if (c->iter_graph) cudaGraphExecDestroy(c->iter_graph);
  for (void* p : c->owned) cudaFree(p);
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  if (c->h_state) cudaFreeHost(c->h_state);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  cudaGetLastError();
  cudaSetDevice(prev);
  delete c;
}

pcg_status pcg_set_stream(pcg_ctx* c, void* stream) {
  if (!c) return PCG_EINVAL;
  c->stream = stream ? (cudaStream_t)stream : c->own_stream;
  return PCG_OK;
}

pcg_status pcg_set_shifts(pcg_ctx* c, const double* shifts, int32_t count) {
  if (!c) return PCG_EINVAL;
  if (!shifts || count <= 0) {
    c->var_shifts.clear();
    return PCG_OK;
  }
  for (int32_t k = 0; k < count; ++k)
    if (!(shifts[k] >= 0.0) || !isfinite(shifts[k])) return fail(c, PCG_EINVAL, "shifts must be finite and >= 0");
  c->var_shifts.assign(shifts, shifts + count);
  return PCG_OK;
}

pcg_status pcg_set_param(pcg_ctx* c, int32_t param, double value) {
  if (!c) return PCG_EINVAL;
  switch (param) {
    case PCG_PARAM_MIXED_ETA:
      if (!(value > 0.0 && value < 1.0)) return fail(c, PCG_EINVAL, "eta must lie in (0, 1)");
      c->mx_eta = value;
      return PCG_OK;
    case PCG_PARAM_BARRIER_TIMEOUT_MS:
      if (!(value >= 1.0 && value <= 600000.0)) return fail(c, PCG_EINVAL, "timeout must lie in [1, 600000] ms");
      c->barrier_timeout_ms = value;
      return PCG_OK;
    case PCG_PARAM_TEST_BARRIER_PHANTOMS:
      if (!(value >= 0.0 && value <= 1024.0)) return fail(c, PCG_EINVAL, "phantoms must lie in [0, 1024]");
      c->barrier_phantoms = (unsigned)value;
      return PCG_OK;
    case PCG_PARAM_MAX_RESTARTS:
      if (!(value >= 1.0 && value <= 1e6)) return fail(c, PCG_EINVAL, "max restarts must lie in [1, 1e6]");
      c->mx_max_restarts = (int)value;
      return PCG_OK;
    case PCG_PARAM_ITER_STAGES: {
      if (!(value == 0.0 || value == 2.0 || value == 3.0)) return fail(c, PCG_EINVAL, "stages must be 0, 2 or 3");
      const int old_stages = c->op.iter_stages;
      c->op.iter_stages = resolve_iter_stages(c->op, (int)value);
      const int g = grid_for(c->op, K_SPCG_ITER, kBlockThreads);
      if (g <= 0) {
        cudaGetLastError();
        c->op.iter_stages = old_stages;
        return fail(c, PCG_ECUDA, "could not size the iteration grid");
      }
      c->grid[K_SPCG_ITER] = g;
      return PCG_OK;
    }
    case PCG_PARAM_TRUE_TOL:
      if (!(value >= 0.0) || !isfinite(value)) return fail(c, PCG_EINVAL, "true tolerance must be finite and >= 0");
      c->true_tol = value;
      return PCG_OK;
    default:
      return fail(c, PCG_EINVAL, "unknown parameter");
  }
}

pcg_status pcg_get_param(const pcg_ctx* c, int32_t param, double* value) {
  if (!c || !value) return PCG_EINVAL;
  switch (param) {
    case PCG_PARAM_MIXED_ETA: *value = c->mx_eta; return PCG_OK;
    case PCG_PARAM_MAX_RESTARTS: *value = c->mx_max_restarts; return PCG_OK;
    case PCG_PARAM_BARRIER_TIMEOUT_MS: *value = c->barrier_timeout_ms; return PCG_OK;
    case PCG_PARAM_TEST_BARRIER_PHANTOMS: *value = c->barrier_phantoms; return PCG_OK;
    case PCG_PARAM_TRUE_TOL: *value = c->true_tol; return PCG_OK;
    case PCG_PARAM_ITER_STAGES: *value = c->op.iter_stages; return PCG_OK;
    default: return PCG_EINVAL;
  }
}

pcg_status pcg_kernel_stats(pcg_ctx* c, int64_t* launches_total, int64_t* iter_launches, double* iter_ms) {
  if (!c) return PCG_EINVAL;
  if (launches_total) *launches_total = c->launches;
  if (iter_launches) *iter_launches = c->iter_launches;
  if (iter_ms) *iter_ms = c->iter_ms;
  return PCG_OK;
}

pcg_status pcg_kernel_stats_reset(pcg_ctx* c) {
  if (!c) return PCG_EINVAL;
  c->launches = c->iter_launches = 0;
  c->iter_ms = 0.0;
  return PCG_OK;
}

}  // extern "C"

namespace {

constexpr int kIterGraphLen = 32;

// The graph of kIterGraphLen iteration launches for the current launch arguments (built
// on first use).  PCG_ENOTIMPL when the stream cannot be captured (the legacy default
// stream): the caller then launches directly.
pcg_status ensure_iter_graph(pcg_ctx* c) {
  pcg_ctx::IterGraphKey key;
  memset(&key, 0, sizeof key);
  key.op = c->op;
  key.v = c->v;
  key.h = c->h;
  key.st = c->d_state;
  key.partials = c->d_partials;
  key.stream = c->stream;
  key.grid = c->grid[K_SPCG_ITER];
  if (c->iter_graph && memcmp(&key, &c->iter_key, sizeof key) == 0) return PCG_OK;
  if (c->iter_graph) {
    cudaGraphExecDestroy(c->iter_graph);
    c->iter_graph = nullptr;
  }
  if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return PCG_ENOTIMPL;
  }
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < kIterGraphLen && e == cudaSuccess; ++k)
    e = launch_spcg_iter(c->op, launch_of(c, K_SPCG_ITER), c->v, c->d_state, c->h, c->d_partials);
  cudaGraph_t g = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(c->stream, &g);
  if (e != cudaSuccess || ee != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return PCG_ENOTIMPL;
  }
  e = cudaGraphInstantiate(&c->iter_graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    c->iter_graph = nullptr;
    cudaGetLastError();
    return PCG_ENOTIMPL;
  }
  memcpy(&c->iter_key, &key, sizeof key);
  return PCG_OK;
}

// The launch sequence of one solve.  b (device, 16-byte aligned or the
// context's copy), x0 already placed in v.x when has_x0.
pcg_status run_solve(pcg_ctx* c, bool has_x0, int method, double sigma, double tol, int maxit, int true_every,
                     int* iters_out, int* status_out) {
  const bool profile = (c->flags & PCG_PROFILE) != 0;
  State st{};
  st.iter = 0;
  st.status = ST_RUNNING;
  st.maxit = maxit;
  st.sigma = method == PCG_SPCG ? sigma : 0.0;
  st.tol_abs = tol;   // relative until the residual kernel scales it by ||b||
  st.tol_true = c->true_tol;
  *c->h_state = st;
  CUDA_TRY(c, cudaMemcpyAsync(c->d_state, c->h_state, sizeof(State), cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(c->d_hist, 0xff, 7 * (size_t)c->hist_cap * sizeof(double), c->stream));  // NaN
  if (profile) {
    pcg_status s = ensure_events(c, (size_t)maxit);
    if (s != PCG_OK) return s;
  }
  auto L = [&](int kind) { return launch_of(c, kind); };
  CUDA_TRY(c, launch_residual(c->op, L(K_RESIDUAL), c->v.b, has_x0 ? c->v.x : nullptr, c->v.x, c->v.r, c->d_state,
                              c->d_partials));
  ++c->launches;
  const bool cg = method == PCG_CG;
  if (cg) {
    CUDA_TRY(c, launch_cg_p0(c->op, L(K_CG_P0), c->v, c->d_state, c->h, c->d_partials));
  } else {
    CUDA_TRY(c, launch_spcg_w0(c->op, L(K_SPCG_W0), c->v, c->d_state, c->h, c->d_partials));
  }
  ++c->launches;
  if (true_every > 0) {
    CUDA_TRY(c, launch_true_res(c->op, L(K_TRUE_RES), c->v, c->d_state, c->h, c->d_partials));
    ++c->launches;
  }
  if (!cg && (c->flags & PCG_PERSISTENT) && true_every <= 0 && maxit > 0) {
    // every iteration inside one cooperative launch
    if (profile) CUDA_TRY(c, cudaEventRecord(c->ev[0], c->stream));
    CUDA_TRY(c, launch_spcg_persistent(c->op, c->grid_persistent, c->stream, c->v, c->d_state, c->h, c->d_partials,
                                       (unsigned long long)(c->barrier_timeout_ms * 1e6), c->barrier_phantoms));
    if (profile) CUDA_TRY(c, cudaEventRecord(c->ev[1], c->stream));
    ++c->launches;
    CUDA_TRY(c, launch_true_res(c->op, L(K_TRUE_RES), c->v, c->d_state, c->h, c->d_partials));
    ++c->launches;
    CUDA_TRY(c, cudaMemcpyAsync(c->h_state, c->d_state, sizeof(State), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (profile) {
      float ms = 0.f;
      CUDA_TRY(c, cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
      c->iter_ms += ms;
      c->iter_launches += c->h_state->iter;   // iterations run inside the launch
    }
    *iters_out = c->h_state->iter;
    *status_out = c->h_state->status;
    return PCG_OK;
  }
  int done = 0;            // iteration launches issued
  int prof_pairs = 0;
  int chunk = 16;
  while (done < maxit) {
    const bool poll = tol > 0.0 || (c->true_tol > 0.0 && true_every > 0);   // the solve may stop early
    const int todo = poll ? std::min(chunk, maxit - done) : maxit - done;
    int k = 0;
    if (!cg && !profile && true_every <= 0 && todo >= kIterGraphLen && ensure_iter_graph(c) == PCG_OK) {
      // whole graphs of kIterGraphLen iterations; the remainder is launched directly below
      for (; k + kIterGraphLen <= todo; k += kIterGraphLen) {
        CUDA_TRY(c, cudaGraphLaunch(c->iter_graph, c->stream));
        c->launches += kIterGraphLen;
        c->iter_launches += kIterGraphLen;
        done += kIterGraphLen;
      }
    }
    for (; k < todo; ++k) {
      if (cg) {
        CUDA_TRY(c, launch_cg_spmv(c->op, L(K_CG_SPMV), c->v, c->d_state, c->h, c->d_partials));
        CUDA_TRY(c, launch_cg_update(c->op, L(K_CG_UPDATE), c->v, c->d_state, c->h, c->d_partials));
        CUDA_TRY(c, launch_cg_p(c->op, L(K_CG_P), c->v, c->d_state, c->h));
        c->launches += 3;
      } else {
        if (profile) CUDA_TRY(c, cudaEventRecord(c->ev[2 * prof_pairs], c->stream));
        CUDA_TRY(c, launch_spcg_iter(c->op, L(K_SPCG_ITER), c->v, c->d_state, c->h, c->d_partials));
        if (profile) CUDA_TRY(c, cudaEventRecord(c->ev[2 * prof_pairs + 1], c->stream));
        prof_pairs += profile;
        ++c->launches;
        ++c->iter_launches;
      }
      ++done;
      if (true_every > 0 && done % true_every == 0) {
        CUDA_TRY(c, launch_true_res(c->op, L(K_TRUE_RES), c->v, c->d_state, c->h, c->d_partials));
        ++c->launches;
      }
    }
    if (poll && done < maxit) {
      CUDA_TRY(c, cudaMemcpyAsync(c->h_state, c->d_state, sizeof(State), cudaMemcpyDeviceToHost, c->stream));
      CUDA_TRY(c, cudaStreamSynchronize(c->stream));
      if (c->h_state->status != ST_RUNNING) break;
      chunk = std::min(chunk * 2, 256);
    }
  }
  // true residual at the final iterate
  CUDA_TRY(c, launch_true_res(c->op, L(K_TRUE_RES), c->v, c->d_state, c->h, c->d_partials));
  ++c->launches;
  CUDA_TRY(c, cudaMemcpyAsync(c->h_state, c->d_state, sizeof(State), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (profile) {
    for (int k = 0; k < prof_pairs; ++k) {
      float ms = 0.f;
      CUDA_TRY(c, cudaEventElapsedTime(&ms, c->ev[2 * k], c->ev[2 * k + 1]));
      c->iter_ms += ms;
    }
  }
  *iters_out = c->h_state->iter;
  *status_out = c->h_state->status;
  return PCG_OK;
}

pcg_status ensure_mixed(pcg_ctx* c) {
  if (c->mixed_ready) return PCG_OK;
  auto copy32 = [&](const double* src, const float** dst) -> pcg_status {
    void* p;
    const long long count = src == c->op.val ? c->nnz : (long long)c->n;
    pcg_status s = dev_alloc(c, &p, (size_t)(count > 0 ? count : 1) * sizeof(float));
    if (s != PCG_OK) return s;
    CUDA_TRY(c, launch_to_f32(src, (float*)p, count, c->stream));
    *dst = (const float*)p;
    return PCG_OK;
  };
  pcg_status s;
  if (c->op.layout == PCG_CSR32) {
    if ((s = copy32(c->op.val, &c->op.val32)) != PCG_OK) return s;
  } else if (c->op.diag) {
    if ((s = copy32(c->op.diag, &c->op.diag32)) != PCG_OK) return s;
    if ((s = copy32(c->op.ax, &c->op.ax32)) != PCG_OK) return s;
    if ((s = copy32(c->op.ay, &c->op.ay32)) != PCG_OK) return s;
    if (c->op.layout == PCG_STENCIL7_3D && (s = copy32(c->op.az, &c->op.az32)) != PCG_OK) return s;
  }
  if (c->d_dinv) {
    if ((s = copy32(c->d_dinv, &c->dinv32)) != PCG_OK) return s;
    void* p;
    if ((s = dev_alloc(c, &p, c->vec_stride * sizeof(double))) != PCG_OK) return s;
    c->mx_u64 = (double*)p;
  }
  for (int k = 0; k < KM_NKINDS; ++k) {
    c->grid_mx[k] = grid_for_mixed(c->op, k, kBlockThreads);
    if (c->grid_mx[k] <= 0) {
      cudaGetLastError();
      return fail(c, PCG_ECUDA, "could not size the mixed-precision grids");
    }
  }
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->mixed_ready = true;
  return PCG_OK;
}

// Mixed precision with restarts: the restart pair (binary64 true residual, w_0)
// is queued after every kRestartEvery iteration launches and does nothing unless
// the inner iteration asked for it, so the refinement loop runs on the device;
// the host only polls between chunks to stop queueing once the solve has ended.
pcg_status run_solve_mixed(pcg_ctx* c, bool has_x0, int method, double sigma, double tol, int maxit,
                           int true_every, int* iters_out, int* status_out) {
  constexpr int kRestartEvery = 4;
  State st{};
  st.iter = 0;
  st.status = ST_RESTART;
  st.maxit = maxit;
  st.sigma = method == PCG_SPCG ? sigma : 0.0;
  st.tol_abs = 0.0;
  st.tol_rel = tol;
  st.eta = c->mx_eta;
  st.rprev = INFINITY;
  st.restarts = 0;
  st.max_restarts = c->mx_max_restarts;
  *c->h_state = st;
  CUDA_TRY(c, cudaMemcpyAsync(c->d_state, c->h_state, sizeof(State), cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(c->d_hist, 0xff, 7 * (size_t)c->hist_cap * sizeof(double), c->stream));  // NaN
  if (!has_x0) CUDA_TRY(c, cudaMemsetAsync(c->v.x, 0, (size_t)c->n * sizeof(double), c->stream));
  const bool jac = c->d_dinv != nullptr;
  const Launch Lr{c->grid_mx[KM_RESTART], kBlockThreads, c->stream};
  const Launch Lw{c->grid_mx[jac ? KM_W0_JAC : KM_W0], kBlockThreads, c->stream};
  const Launch Li{c->grid_mx[jac ? KM_ITER_JAC : KM_ITER], kBlockThreads, c->stream};
  GenVecs g{};
  if (jac) {
    if (!c->gen_base) {
      void* p;
      pcg_status s = dev_alloc(c, &p, 5 * c->vec_stride * sizeof(double));
      if (s != PCG_OK) return s;
      c->gen_base = (double*)p;
    }
    g.b = c->v.b;
    g.x = c->v.x;
    g.r = c->v.r;
    g.w0 = c->v.w0;
    g.w1 = c->v.w1;
    g.z = c->v.z;
    g.s = c->v.s;
    g.t = c->v.p;
    g.u = c->gen_base;
    g.q = c->gen_base + c->vec_stride;
    g.p = c->gen_base + 2 * c->vec_stride;
    g.m0 = c->gen_base + 3 * c->vec_stride;
    g.m1 = c->gen_base + 4 * c->vec_stride;
    g.dinv = c->d_dinv;
    g.dinv32 = c->dinv32;
  }
  auto restart_pair = [&]() -> pcg_status {
    CUDA_TRY(c, launch_mx_restart(c->op, Lr, c->v, c->d_state, c->h, c->d_partials));
    if (jac) {
      CUDA_TRY(c, launch_mxj_u0(g, c->mx_u64, (int)c->n, c->d_state, c->stream));
      CUDA_TRY(c, launch_mxj_w0(c->op, Lw, g, c->mx_u64, c->d_state, c->h, c->d_partials));
      c->launches += 3;
    } else {
      CUDA_TRY(c, launch_mx_w0(c->op, Lw, c->v, c->d_state, c->h, c->d_partials));
      c->launches += 2;
    }
    return PCG_OK;
  };
  pcg_status s = restart_pair();
  if (s != PCG_OK) return s;
  (void)true_every;   // the true residual is logged at every restart and at exit
  const long long max_launches = (long long)maxit + (long long)kRestartEvery * (c->mx_max_restarts + 2) + 64;
  long long launched = 0;
  int chunk = 32;
  for (;;) {
    CUDA_TRY(c, cudaMemcpyAsync(c->h_state, c->d_state, sizeof(State), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    const int stt = c->h_state->status;
    if (stt != ST_RUNNING && stt != ST_RESTART) break;
    if (launched >= max_launches) break;
    for (int k = 0; k < chunk; ++k) {
      if (jac) {
        CUDA_TRY(c, launch_mxj_iter(c->op, Li, g, c->d_state, c->h, c->d_partials));
      } else {
        CUDA_TRY(c, launch_mx_iter(c->op, Li, c->v, c->d_state, c->h, c->d_partials));
      }
      ++c->launches;
      ++launched;
      if (launched % kRestartEvery == 0) {
        if ((s = restart_pair()) != PCG_OK) return s;
      }
    }
    chunk = std::min(chunk * 2, 512);
  }
  CUDA_TRY(c, launch_true_res(c->op, launch_of(c, K_TRUE_RES), c->v, c->d_state, c->h, c->d_partials));
  ++c->launches;
  CUDA_TRY(c, cudaMemcpyAsync(c->h_state, c->d_state, sizeof(State), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  *iters_out = c->h_state->iter;
  *status_out = c->h_state->status;
  return PCG_OK;
}

pcg_status ensure_general(pcg_ctx* c, int maxit, bool jac, bool var) {
  if (jac && !c->gen_base) {
    void* p;
    pcg_status s = dev_alloc(c, &p, 5 * c->vec_stride * sizeof(double));
    if (s != PCG_OK) return s;
    c->gen_base = (double*)p;
  }
  int& grid = c->grid_gen[2 * jac + var];
  if (grid <= 0) {
    grid = grid_for_general(c->op, jac, var);
    if (grid <= 0) {
      cudaGetLastError();
      return fail(c, PCG_ECUDA, "could not size the general grid");
    }
  }
  if (c->shifts_cap < maxit + 1) {
    if (c->d_shifts) {
      cudaFree(c->d_shifts);
      c->owned.erase(std::find(c->owned.begin(), c->owned.end(), (void*)c->d_shifts));
      c->d_shifts = nullptr;
    }
    void* p;
    const int cap = std::max(maxit + 1, 1024);
    pcg_status s = dev_alloc(c, &p, cap * sizeof(double));
    if (s != PCG_OK) return s;
    c->d_shifts = (double*)p;
    c->shifts_cap = cap;
  }
  return PCG_OK;
}

// Jacobi M^{-1} and/or a variable shift: Algorithm 4 (Algorithm 3 for a constant shift).
// sh: maxit + 1 shifts (sh[0] = sigma_{-1}).
pcg_status run_solve_general(pcg_ctx* c, bool has_x0, const std::vector<double>& sh, bool var, double tol,
                             int maxit, int true_every, int* iters_out, int* status_out) {
  const bool jac = c->d_dinv != nullptr;
  pcg_status s = ensure_general(c, maxit, jac, var);
  if (s != PCG_OK) return s;
  CUDA_TRY(c, cudaMemcpyAsync(c->d_shifts, sh.data(), (maxit + 1) * sizeof(double), cudaMemcpyHostToDevice,
                              c->stream));
  GenVecs g{};
  g.b = c->v.b;
  g.x = c->v.x;
  g.r = c->v.r;
  g.w0 = c->v.w0;
  g.w1 = c->v.w1;
  g.z = c->v.z;
  g.s = c->v.s;
  g.t = c->v.p;
  if (jac) {
    g.u = c->gen_base;
    g.q = c->gen_base + c->vec_stride;
    g.p = c->gen_base + 2 * c->vec_stride;
    g.m0 = c->gen_base + 3 * c->vec_stride;
    g.m1 = c->gen_base + 4 * c->vec_stride;
    g.dinv = c->d_dinv;
  }
  g.shifts = c->d_shifts;
  State st{};
  st.status = ST_RUNNING;
  st.maxit = maxit;
  st.sigma = sh[0];
  st.tol_abs = tol;   // relative until the residual kernel scales it by ||b||
  st.tol_true = c->true_tol;
  *c->h_state = st;
  CUDA_TRY(c, cudaMemcpyAsync(c->d_state, c->h_state, sizeof(State), cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(c->d_hist, 0xff, 7 * (size_t)c->hist_cap * sizeof(double), c->stream));  // NaN
  auto L = [&](int kind) { return launch_of(c, kind); };
  const Launch Lg{c->grid_gen[2 * jac + var], kBlockThreads, c->stream};
  CUDA_TRY(c, launch_residual(c->op, L(K_RESIDUAL), c->v.b, has_x0 ? c->v.x : nullptr, c->v.x, c->v.r, c->d_state,
                              c->d_partials));
  ++c->launches;
  if (jac) {
    CUDA_TRY(c, launch_diag_scale(c->d_dinv, c->v.r, g.u, (int)c->n, c->d_state, c->stream));   // u_0
    ++c->launches;
  }
  CUDA_TRY(c, launch_gen_w0(c->op, Lg, g, c->d_state, c->h, c->d_partials, jac, var));
  ++c->launches;
  if (true_every > 0) {
    CUDA_TRY(c, launch_true_res(c->op, L(K_TRUE_RES), c->v, c->d_state, c->h, c->d_partials));
    ++c->launches;
  }
  int done = 0, chunk = 16;
  while (done < maxit) {
    const bool poll = tol > 0.0 || (c->true_tol > 0.0 && true_every > 0);   // the solve may stop early
    const int todo = poll ? std::min(chunk, maxit - done) : maxit - done;
    for (int k = 0; k < todo; ++k) {
      CUDA_TRY(c, launch_gen_iter(c->op, Lg, g, c->d_state, c->h, c->d_partials, jac, var));
      ++c->launches;
      ++done;
      if (true_every > 0 && done % true_every == 0) {
        CUDA_TRY(c, launch_true_res(c->op, L(K_TRUE_RES), c->v, c->d_state, c->h, c->d_partials));
        ++c->launches;
      }
    }
    if (poll && done < maxit) {
      CUDA_TRY(c, cudaMemcpyAsync(c->h_state, c->d_state, sizeof(State), cudaMemcpyDeviceToHost, c->stream));
      CUDA_TRY(c, cudaStreamSynchronize(c->stream));
      if (c->h_state->status != ST_RUNNING) break;
      chunk = std::min(chunk * 2, 256);
    }
  }
  CUDA_TRY(c, launch_true_res(c->op, L(K_TRUE_RES), c->v, c->d_state, c->h, c->d_partials));
  ++c->launches;
  CUDA_TRY(c, cudaMemcpyAsync(c->h_state, c->d_state, sizeof(State), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  *iters_out = c->h_state->iter;
  *status_out = c->h_state->status;
  return PCG_OK;
}

pcg_status solve_common(pcg_ctx* c, const double* b, const double* x0, int32_t method, double sigma, double tol,
                        int32_t maxit, int32_t precision, double* x_out, pcg_result* res, bool host) {
  if (!c) return PCG_EINVAL;
  c->err.clear();
  if (!b || !x_out) return fail(c, PCG_EINVAL, "b and x_out must not be NULL");
  if (method < PCG_CG || method > PCG_SPCG) return fail(c, PCG_EINVAL, "unknown method");
  if (!(sigma >= 0.0) || !isfinite(sigma)) return fail(c, PCG_EINVAL, "sigma must be finite and >= 0");
  if (!(tol >= 0.0) || !isfinite(tol)) return fail(c, PCG_EINVAL, "tol must be finite and >= 0");
  if (maxit < 0 || maxit > (1 << 28)) return fail(c, PCG_EINVAL, "maxit out of range");
  if (precision != PCG_FP64 && precision != PCG_MIXED_IR) return fail(c, PCG_EINVAL, "unknown precision");
  if (precision == PCG_MIXED_IR && method == PCG_CG)
    return fail(c, PCG_ENOTIMPL, "PCG_MIXED_IR runs Algorithm 3 (PCG_PCG or PCG_SPCG), not classic CG");
  // the shift schedule: pcg_set_shifts (PCG_SPCG only), else the constant sigma (0 for PCG_PCG)
  const bool scheduled = method == PCG_SPCG && !c->var_shifts.empty();
  if (scheduled && (int)c->var_shifts.size() < maxit + 1)
    return fail(c, PCG_EINVAL, "pcg_set_shifts gave fewer than maxit + 1 shifts");
  std::vector<double> sh(maxit + 1, method == PCG_SPCG ? sigma : 0.0);
  bool var = false;
  if (scheduled) {
    std::copy(c->var_shifts.begin(), c->var_shifts.begin() + maxit + 1, sh.begin());
    for (int k = 1; k <= maxit; ++k) var = var || sh[k] != sh[0];
    sigma = sh[0];
  }
  // Algorithm 1 takes M^{-1} in its own kernels; Algorithms 2-4 with M^{-1} or a variable shift
  // run the general sweeps
  const bool general = method != PCG_CG && (c->d_dinv != nullptr || var);
  if (var && precision == PCG_MIXED_IR)
    return fail(c, PCG_ENOTIMPL, "PCG_MIXED_IR with a variable shift is not implemented");
  CUDA_TRY(c, cudaSetDevice(c->device));
  pcg_status s;
  if ((s = ensure_vectors(c)) != PCG_OK) return s;
  if (precision == PCG_MIXED_IR && (s = ensure_mixed(c)) != PCG_OK) return s;
  if ((s = ensure_hist(c, maxit + 1)) != PCG_OK) return s;
  c->v.dinv = method == PCG_CG ? c->d_dinv : nullptr;
  const size_t bytes = (size_t)c->n * sizeof(double);
  const cudaMemcpyKind in = host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const cudaMemcpyKind outk = host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (!host && ((uintptr_t)b % 16) == 0) {
    c->v.b = b;                                   // aligned caller buffer: read in place
  } else {
    CUDA_TRY(c, cudaMemcpyAsync(c->d_b, b, bytes, in, c->stream));
    c->v.b = c->d_b;
  }
  if (x0) CUDA_TRY(c, cudaMemcpyAsync(c->v.x, x0, bytes, in, c->stream));
  const int true_every = res ? res->true_every : 0;
  int iters = 0, st = ST_RUNNING;
  s = precision == PCG_MIXED_IR ? run_solve_mixed(c, x0 != nullptr, method, sigma, tol, maxit, true_every, &iters, &st)
      : general                  ? run_solve_general(c, x0 != nullptr, sh, var, tol, maxit, true_every, &iters, &st)
                                 : run_solve(c, x0 != nullptr, method, sigma, tol, maxit, true_every, &iters, &st);
  c->v.b = c->d_b;
  if (s != PCG_OK) return s;
  CUDA_TRY(c, cudaMemcpyAsync(x_out, c->v.x, bytes, outk, c->stream));
  pcg_status ret = st == ST_CONVERGED ? PCG_OK : st == ST_BREAKDOWN ? PCG_EBREAKDOWN
                   : st == ST_TIMEOUT ? PCG_ETIMEOUT : PCG_ENOTCONV;
  if (st == ST_TIMEOUT)
    c->err = "a bounded device wait (the persistent kernel's grid barrier or a staged sweep's copy) exceeded its time limit";
  if (st == ST_STALLED) c->err = "iterative refinement stalled: a restart did not lower the true residual";
  if (res) {
    const size_t k = (size_t)iters + 1;
    auto get = [&](double* dst, const double* src) -> cudaError_t {
      if (!dst) return cudaSuccess;
      return cudaMemcpyAsync(dst, src, k * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    };
    CUDA_TRY(c, get(res->rec_hist, c->h.rec));
    CUDA_TRY(c, get(res->true_hist, c->h.tru));
    CUDA_TRY(c, get(res->gap_hist, c->h.gap));
    CUDA_TRY(c, get(res->alpha_hist, c->h.alpha));
    CUDA_TRY(c, get(res->beta_hist, c->h.beta));
    double fin[2] = {NAN, NAN};
    CUDA_TRY(c, cudaMemcpyAsync(&fin[0], c->h.tru + iters, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(&fin[1], c->h.rec + iters, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    const double bn = c->h_state->bnorm;
    res->iters = iters;
    res->status = ret;
    res->final_true_relres = bn > 0 ? fin[0] / bn : fin[0];
    res->final_rec_relres = bn > 0 ? fin[1] / bn : fin[1];
  }
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (ret == PCG_EBREAKDOWN) c->err = "breakdown: non-positive or non-finite curvature (delta or 1/alpha)";
  return ret;
}

}  // namespace

extern "C" {

pcg_status pcg_solve(pcg_ctx* c, const double* b, const double* x0, int32_t method, double sigma, double tol,
                     int32_t maxit, int32_t precision, double* x_out, pcg_result* res) {
  return solve_common(c, b, x0, method, sigma, tol, maxit, precision, x_out, res, true);
}

pcg_status pcg_solve_device(pcg_ctx* c, const double* b, const double* x0, int32_t method, double sigma, double tol,
                            int32_t maxit, int32_t precision, double* x_out, pcg_result* res) {
  return solve_common(c, b, x0, method, sigma, tol, maxit, precision, x_out, res, false);
}

pcg_status pcg_apply(pcg_ctx* c, const double* x, double* y) {
  if (!c) return PCG_EINVAL;
  c->err.clear();
  if (!x || !y) return fail(c, PCG_EINVAL, "x and y must not be NULL");
  CUDA_TRY(c, cudaSetDevice(c->device));
  pcg_status s = ensure_vectors(c);
  if (s != PCG_OK) return s;
  const size_t bytes = (size_t)c->n * sizeof(double);
  CUDA_TRY(c, cudaMemcpyAsync(c->v.w0, x, bytes, cudaMemcpyDeviceToDevice, c->stream));
  CUDA_TRY(c, launch_apply(c->op, launch_of(c, K_APPLY), c->v.w0, c->v.w1));
  ++c->launches;
  CUDA_TRY(c, cudaMemcpyAsync(y, c->v.w1, bytes, cudaMemcpyDeviceToDevice, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return PCG_OK;
}

pcg_status pcg_psi(pcg_ctx* c, const double* alpha, const double* beta, int32_t i, const double* grid, int32_t ngrid,
                   double* psi_out) {
  if (!c) return PCG_EINVAL;
  c->err.clear();
  if (!alpha || !beta || !grid || !psi_out || i < 1 || ngrid < 1) return fail(c, PCG_EINVAL, "bad psi arguments");
  CUDA_TRY(c, cudaSetDevice(c->device));
  const int need = 2 * (i + 1) + 2 * ngrid;
  if (c->small_cap < need) {
    if (c->d_small) {
      cudaFree(c->d_small);
      c->owned.erase(std::find(c->owned.begin(), c->owned.end(), (void*)c->d_small));
      c->d_small = nullptr;
    }
    void* p;
    pcg_status s = dev_alloc(c, &p, (size_t)need * sizeof(double));
    if (s != PCG_OK) return s;
    c->d_small = (double*)p;
    c->small_cap = need;
  }
  double* da = c->d_small;
  double* db = da + (i + 1);
  double* dg = db + (i + 1);
  double* dp = dg + ngrid;
  CUDA_TRY(c, cudaMemcpyAsync(da, alpha, (i + 1) * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(db, beta, (i + 1) * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(dg, grid, ngrid * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, launch_psi(da, db, i, dg, ngrid, dp, c->stream));
  ++c->launches;
  CUDA_TRY(c, cudaMemcpyAsync(psi_out, dp, ngrid * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return PCG_OK;
}

pcg_status pcg_psi_varsh(pcg_ctx* c, const double* alpha, const double* beta, int32_t i, const double* schedules,
                         int32_t stride, int32_t nsched, double* psi_out) {
  if (!c) return PCG_EINVAL;
  c->err.clear();
  if (!alpha || !beta || !schedules || !psi_out || i < 1 || nsched < 1 || stride < i + 2)
    return fail(c, PCG_EINVAL, "bad psi_varsh arguments");
  CUDA_TRY(c, cudaSetDevice(c->device));
  const long long need = 2LL * (i + 1) + (long long)stride * nsched + nsched;
  if (need > INT32_MAX) return fail(c, PCG_EINVAL, "psi_varsh arguments too large");
  if (c->small_cap < need) {
    if (c->d_small) {
      cudaFree(c->d_small);
      c->owned.erase(std::find(c->owned.begin(), c->owned.end(), (void*)c->d_small));
      c->d_small = nullptr;
    }
    void* p;
    pcg_status s = dev_alloc(c, &p, (size_t)need * sizeof(double));
    if (s != PCG_OK) return s;
    c->d_small = (double*)p;
    c->small_cap = (int)need;
  }
  double* da = c->d_small;
  double* db = da + (i + 1);
  double* ds = db + (i + 1);
  double* dp = ds + (size_t)stride * nsched;
  CUDA_TRY(c, cudaMemcpyAsync(da, alpha, (i + 1) * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(db, beta, (i + 1) * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(ds, schedules, (size_t)stride * nsched * sizeof(double), cudaMemcpyHostToDevice,
                              c->stream));
  CUDA_TRY(c, launch_psi_var(da, db, i, ds, stride, nsched, dp, c->stream));
  ++c->launches;
  CUDA_TRY(c, cudaMemcpyAsync(psi_out, dp, nsched * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return PCG_OK;
}

pcg_status pcg_select_sigma(pcg_ctx* c, const double* b, int32_t iters, const double* grid, int32_t ngrid,
                            double* sigma_out, double* psi_out) {
  if (!c) return PCG_EINVAL;
  if (!b || !grid || !sigma_out || iters < 2 || ngrid < 1) return fail(c, PCG_EINVAL, "bad select_sigma arguments");
  for (int k = 0; k < ngrid; ++k)
    if (!(grid[k] >= 0.0) || !isfinite(grid[k])) return fail(c, PCG_EINVAL, "negative or non-finite shift");
  std::vector<double> al(iters + 1), be(iters + 1), ps(ngrid);
  std::vector<double> x(c->n);
  pcg_result r{};
  r.alpha_hist = al.data();
  r.beta_hist = be.data();
  pcg_status s = pcg_solve(c, b, nullptr, PCG_PCG, 0.0, 0.0, iters, PCG_FP64, x.data(), &r);
  if (s != PCG_OK && s != PCG_ENOTCONV && s != PCG_EBREAKDOWN) return s;
  const int i = r.iters - 1;   // alpha/beta exist for iterations 0 .. iters-1
  if (i < 1) return fail(c, PCG_EINVAL, "pilot run too short for psi");
  s = pcg_psi(c, al.data(), be.data(), i, grid, ngrid, ps.data());
  if (s != PCG_OK) return s;
  double mn = INFINITY;
  for (double v : ps)
    if (v < mn) mn = v;
  double best = NAN;
  for (int k = 0; k < ngrid; ++k)
    if (ps[k] <= 2.0 * mn && !(grid[k] >= best)) best = grid[k];
  *sigma_out = best;
  if (psi_out) memcpy(psi_out, ps.data(), ngrid * sizeof(double));
  return PCG_OK;
}

}  // extern "C"
