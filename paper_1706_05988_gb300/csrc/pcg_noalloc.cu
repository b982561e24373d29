// pcg_true_residual_noalloc: ||b - A x||_2 and ||(b - A x) - r||_2 without any
// device allocation, for callers that cannot call cudaMalloc (see include/pcg.h).
//
// The kernel is a variant of the solver's true-residual kernel: each block
// reduces one fixed chunk of kNoallocChunk unknowns to one partial per norm,
// and the last block to finish (atomic ticket) sums the partials in block
// order.  The partials and the ticket live in one file-scope __device__ array,
// so the largest problem is kNoallocMaxBlocks * kNoallocChunk unknowns.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>
#include <utility>

#define PCG_KERNELS_IMPL
#include "../../include/pcg.h"
#include "pcg_kernels.cuh"

namespace pcgk {
namespace {

constexpr int kNoallocChunk = 4096;         // unknowns per block
constexpr int kNoallocMaxBlocks = 4096;     // partial-sum slots -> n <= 16,777,216
static_assert((long long)kNoallocChunk * kNoallocMaxBlocks == PCG_NOALLOC_MAX_N, "limit in pcg.h");

struct NoallocScratch {
  double partials[2 * kNoallocMaxBlocks];
  unsigned int ticket;
};

// 64 KiB + 4 B, held by every GPU that loads the library until the process exits.
static __device__ __align__(256) NoallocScratch g_noalloc;

template <class Op>
__global__ void __launch_bounds__(kBlock) k_true_res_noalloc(Op op, const double* __restrict__ b,
                                                            const double* __restrict__ x,
                                                            const double* __restrict__ r, NoallocScratch* sc,
                                                            double* __restrict__ norms) {
  constexpr int VEC = Op::VEC;
  const unsigned n = (unsigned)op.units() * VEC;
  const unsigned beg = blockIdx.x * (unsigned)kNoallocChunk;
  const unsigned end = min(beg + (unsigned)kNoallocChunk, n);
  double t2 = 0.0, f2 = 0.0;
  const auto stp = op.step(kBlock);
  for (auto q = op.cursor((int)(beg / VEC) + threadIdx.x); q.c0 < end; op.advance(q, stp)) {
    const int c0 = (int)q.c0;
    double xc[VEC], ax[VEC], bv[VEC], rv[VEC];
    op.apply(x, q, xc, ax);
    ld_stream<VEC>(b + c0, bv);
    if (r != nullptr) {
      ld_stream<VEC>(r + c0, rv);
    } else {
#pragma unroll
      for (int e = 0; e < VEC; ++e) rv[e] = 0.0;
    }
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      const double t = bv[e] - ax[e];
      const double f = t - rv[e];
      t2 = fma(t, t, t2);
      f2 = fma(f, f, f2);
    }
  }
  double vals[2] = {t2, f2}, tot[2];
  if (!reduce_last_block<2>(vals, sc->partials, &sc->ticket, tot)) return;
  if (threadIdx.x == 0) {
    norms[0] = sqrt(tot[0]);
    norms[1] = r != nullptr ? sqrt(tot[1]) : NAN;
    sc->ticket = 0;
  }
}

template <int DIM, int MODE, int VEC>
StencilOp<DIM, MODE, VEC> stencil_of(const OpDesc& d) {
  StencilOp<DIM, MODE, VEC> o;
  o.n = d.n;
  o.nx = d.nx;
  o.ny = d.ny;
  o.nz = d.nz;
  o.nxny = d.nx * d.ny;
  o.diag = d.diag;
  o.ax = d.ax;
  o.ay = d.ay;
  o.az = d.az;
  return o;
}

template <int DIM, class F>
cudaError_t stencil_dispatch(const OpDesc& d, F&& f) {
  const bool var = d.diag != nullptr;
  if (op_vec(d) == 2) {
    if (var) return f(stencil_of<DIM, ST_VAR, 2>(d));
    return f(stencil_of<DIM, ST_LAP_FIXED, 2>(d));
  }
  if (var) return f(stencil_of<DIM, ST_VAR, 1>(d));
  return f(stencil_of<DIM, ST_LAP_FIXED, 1>(d));
}

template <class F>
cudaError_t op_dispatch(const OpDesc& d, F&& f) {
  switch (d.layout) {
    case 0: return stencil_dispatch<2>(d, std::forward<F>(f));
    case 1: return stencil_dispatch<3>(d, std::forward<F>(f));
    default: {
      CsrOp o;
      o.n = d.n;
      o.row_ptr = d.row_ptr;
      o.col = d.col;
      o.val = d.val;
      return f(o);
    }
  }
}

// Device address of g_noalloc.  The address belongs to the module loaded into the
// device's current context, and a context that is destroyed and created again
// (cudaDeviceReset) may load the module at another address.  So every call made
// outside stream capture looks the address up again (a host-side table lookup,
// no device work) and refreshes the per-device copy; a call inside a capture uses
// that copy, taken by the last call outside capture on the same device.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
NoallocScratch* g_scratch_ptr[kMaxDevices] = {nullptr};

cudaError_t scratch_for(int dev, cudaStream_t s, NoallocScratch** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    // e.g. the legacy stream while another thread captures in global mode: treat as
    // capturing (no lookup) and clear the error
    cudaGetLastError();
    cap = cudaStreamCaptureStatusActive;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (cap == cudaStreamCaptureStatusNone || g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = (NoallocScratch*)p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace pcgk

extern "C" pcg_status pcg_true_residual_noalloc(const pcg_matrix* A, const double* b, const double* x,
                                                const double* r, double* norms, void* stream) {
  using namespace pcgk;
  if (!A || !b || !x || !norms) return PCG_EINVAL;
  OpDesc op{};
  op.layout = A->layout;
  op.fixed_sum = 1;
  long long n = 0;
  if (A->layout == PCG_STENCIL5_2D || A->layout == PCG_STENCIL7_3D) {
    const long long nz = A->layout == PCG_STENCIL7_3D ? A->nz : 1;
    if (A->nx < 1 || A->ny < 1 || nz < 1 || A->nx > INT32_MAX || A->ny > INT32_MAX || nz > INT32_MAX)
      return PCG_EINVAL;
    n = (long long)A->nx * A->ny * nz;
    if (n > PCG_NOALLOC_MAX_N) return PCG_EINVAL;
    const bool var = A->diag != nullptr;
    if (var && (!A->ax || !A->ay || (A->layout == PCG_STENCIL7_3D && !A->az))) return PCG_EINVAL;
    if (!var && (A->ax || A->ay || A->az)) return PCG_EINVAL;
    op.nx = (int)A->nx;
    op.ny = (int)A->ny;
    op.nz = (int)nz;
    op.diag = A->diag;
    op.ax = A->ax;
    op.ay = A->ay;
    op.az = A->az;
  } else if (A->layout == PCG_CSR32) {
    if (A->n < 1 || A->nnz < 0 || A->nnz > INT32_MAX || !A->row_ptr || (A->nnz > 0 && (!A->col || !A->val)))
      return PCG_EINVAL;
    n = A->n;
    if (n > PCG_NOALLOC_MAX_N) return PCG_EINVAL;
    op.row_ptr = A->row_ptr;
    op.col = A->col;
    op.val = A->val;
  } else {
    return PCG_EINVAL;
  }
  op.n = (int)n;
  // every vector holds doubles (8-byte alignment); b, x and r are read with 128-bit
  // loads when the operator takes two unknowns per thread
  const uintptr_t vec_bits = (uintptr_t)b | (uintptr_t)x | (uintptr_t)(r ? r : b);
  if ((vec_bits | (uintptr_t)norms) % 8 != 0) return PCG_EINVAL;
  if (op_vec(op) == 2 && vec_bits % 16 != 0) return PCG_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return PCG_ECUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  NoallocScratch* sc = nullptr;
  if (scratch_for(dev, s, &sc) != cudaSuccess) {
    cudaGetLastError();
    return PCG_ECUDA;
  }
  // the ticket must start at zero (a finished launch leaves it at zero; this also
  // clears it after an aborted one); the partials are fully rewritten by every launch
  if (cudaMemsetAsync(&sc->ticket, 0, sizeof(unsigned int), s) != cudaSuccess) {
    cudaGetLastError();
    return PCG_ECUDA;
  }
  const int grid = (int)((n + kNoallocChunk - 1) / kNoallocChunk);
  const cudaError_t e = op_dispatch(op, [&](auto o) {
    k_true_res_noalloc<decltype(o)><<<grid, kBlock, 0, s>>>(o, b, x, r, sc, norms);
    return cudaGetLastError();
  });
  return e == cudaSuccess ? PCG_OK : PCG_ECUDA;
}
