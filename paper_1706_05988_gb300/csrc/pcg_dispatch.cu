// Maps a runtime operator description onto the compiled kernel instance.
#include <utility>

#include "pcg_kernels.cuh"
#include "pcg_persistent.cuh"
#include "pcg_general.cuh"

// Largest number of unknowns per thread for stencil operators (2 = 128-bit accesses).
#ifndef PCG_STENCIL_MAX_VEC
#define PCG_STENCIL_MAX_VEC 2
#endif

namespace pcgk {
namespace {

template <int DIM, int MODE, int VEC>
StencilOp<DIM, MODE, VEC> make_stencil(const OpDesc& d) {
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
cudaError_t with_stencil(const OpDesc& d, F&& f, int vec) {
  const bool var = d.diag != nullptr;
  if (vec == 2) {
    if (var) return f(make_stencil<DIM, ST_VAR, 2>(d));
    if (d.fixed_sum) return f(make_stencil<DIM, ST_LAP_FIXED, 2>(d));
    return f(make_stencil<DIM, ST_LAP_FP64, 2>(d));
  }
  if (var) return f(make_stencil<DIM, ST_VAR, 1>(d));
  if (d.fixed_sum) return f(make_stencil<DIM, ST_LAP_FIXED, 1>(d));
  return f(make_stencil<DIM, ST_LAP_FP64, 1>(d));
}

// vec: unknowns per thread of a stencil operator (default: op_vec)
template <class F>
cudaError_t with_op(const OpDesc& d, F&& f, int vec = 0) {
  if (vec <= 0) vec = op_vec(d);
  switch (d.layout) {
    case 0: return with_stencil<2>(d, std::forward<F>(f), vec);
    case 1: return with_stencil<3>(d, std::forward<F>(f), vec);
    case 2: {
      CsrOp o;
      o.n = d.n;
      o.row_ptr = d.row_ptr;
      o.col = d.col;
      o.val = d.val;
      return f(o);
    }
    default: return cudaErrorInvalidValue;
  }
}

template <class Op>
using K = Kernels<std::decay_t<Op>>;

}  // namespace

int op_vec(const OpDesc& d) {
  if (d.layout == 2 || PCG_STENCIL_MAX_VEC < 2) return 1;
  if (d.nx % 2 != 0) return 1;
  if (d.diag != nullptr) {
    const uintptr_t m = (uintptr_t)d.diag | (uintptr_t)d.ax | (uintptr_t)d.ay | (d.layout == 1 ? (uintptr_t)d.az : 0);
    if (m % 16 != 0) return 1;
  }
  return 2;
}

int resolve_iter_stages(const OpDesc& d, int stages) {
  int r = 0;
  with_op(d, [&](auto op) {
    r = K<decltype(op)>::iter_stages(op, stages);
    return cudaSuccess;
  });
  return r;
}

int grid_for(const OpDesc& d, int kind, int block) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  int per_sm = 0;
  with_op(d, [&](auto op) {
    per_sm = K<decltype(op)>::blocks_per_sm(op, kind, d.iter_stages);
    return cudaSuccess;
  });
  if (per_sm <= 0) return 0;
  const long long units = d.n / op_vec(d);
  long long g = (long long)sms * per_sm;
  const long long need = (units + block - 1) / block;
  if (need < g) g = need;
  if (g < 1) g = 1;
  if (g > kMaxPartialBlocks) g = kMaxPartialBlocks;
  return (int)g;
}

cudaError_t launch_residual(const OpDesc& d, const Launch& L, const double* b, const double* x0, double* x, double* r,
                            State* st, double* partials) {
  return with_op(d, [&](auto op) { return K<decltype(op)>::residual(op, L, b, x0, x, r, st, partials); });
}
cudaError_t launch_spcg_w0(const OpDesc& d, const Launch& L, Vecs v, State* st, Hist h, double* partials) {
  return with_op(d, [&](auto op) { return K<decltype(op)>::spcg_w0(op, L, v, st, h, partials); });
}
cudaError_t launch_spcg_iter(const OpDesc& d, const Launch& L, Vecs v, State* st, Hist h, double* partials) {
  return with_op(d, [&](auto op) { return K<decltype(op)>::spcg_iter(op, L, v, st, h, partials, d.ff_dots != 0, d.iter_stages); });
}
cudaError_t launch_true_res(const OpDesc& d, const Launch& L, Vecs v, State* st, Hist h, double* partials) {
  return with_op(d, [&](auto op) { return K<decltype(op)>::true_res(op, L, v, st, h, partials); });
}
cudaError_t launch_cg_p0(const OpDesc& d, const Launch& L, Vecs v, State* st, Hist h, double* partials) {
  return with_op(d, [&](auto op) { return K<decltype(op)>::cg_p0(op, L, v, st, h, partials); });
}
cudaError_t launch_cg_spmv(const OpDesc& d, const Launch& L, Vecs v, State* st, Hist h, double* partials) {
  return with_op(d, [&](auto op) { return K<decltype(op)>::cg_spmv(op, L, v, st, h, partials); });
}
cudaError_t launch_cg_update(const OpDesc& d, const Launch& L, Vecs v, State* st, Hist h, double* partials) {
  return with_op(d, [&](auto op) { return K<decltype(op)>::cg_update(op, L, v, st, h, partials); });
}
cudaError_t launch_cg_p(const OpDesc& d, const Launch& L, Vecs v, State* st, Hist h) {
  return with_op(d, [&](auto op) { return K<decltype(op)>::cg_p(op, L, v, st, h); });
}
// (jac, var) -> the instantiated variant; M = I with a constant shift has no general variant
template <class Op, class F>
cudaError_t with_general(bool jac, bool var, F&& f) {
  if (jac && var) return f(GeneralKernels<Op, true, true>{});
  if (jac) return f(GeneralKernels<Op, true, false>{});
  if (var) return f(GeneralKernels<Op, false, true>{});
  return cudaErrorInvalidValue;
}

// The Jacobi sweeps carry nine vectors: at most PCG_GEN_JAC_MAX_VEC unknowns per thread.
int gen_vec(const OpDesc& d, bool jac) {
  const int v = op_vec(d);
  return jac && v > PCG_GEN_JAC_MAX_VEC ? PCG_GEN_JAC_MAX_VEC : v;
}

int grid_for_general(const OpDesc& d, bool jac, bool var) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  int per_sm = 0;
  with_op(
      d,
      [&](auto op) {
        return with_general<std::decay_t<decltype(op)>>(jac, var, [&](auto K) {
          per_sm = decltype(K)::blocks_per_sm();
          return cudaSuccess;
        });
      },
      gen_vec(d, jac));
  if (per_sm <= 0) return 0;
  const long long units = d.n / gen_vec(d, jac);
  long long g = (long long)sms * per_sm;
  const long long need = (units + kBlock - 1) / kBlock;
  if (need < g) g = need;
  if (g < 1) g = 1;
  if (g > kMaxPartialBlocks * 2 / 3) g = kMaxPartialBlocks * 2 / 3;   // three partials per block
  return (int)g;
}

cudaError_t launch_gen_w0(const OpDesc& d, const Launch& L, const GenVecs& v, State* st, Hist h, double* partials,
                          bool jac, bool var) {
  return with_op(
      d,
      [&](auto op) {
        return with_general<std::decay_t<decltype(op)>>(jac, var,
                                                        [&](auto K) { return K.w0(op, L, v, st, h, partials); });
      },
      gen_vec(d, jac));
}
cudaError_t launch_gen_iter(const OpDesc& d, const Launch& L, const GenVecs& v, State* st, Hist h, double* partials,
                            bool jac, bool var) {
  return with_op(
      d,
      [&](auto op) {
        return with_general<std::decay_t<decltype(op)>>(jac, var,
                                                        [&](auto K) { return K.iter(op, L, v, st, h, partials); });
      },
      gen_vec(d, jac));
}

int grid_for_persistent(const OpDesc& d) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  int per_sm = 0;
  with_op(d, [&](auto op) {
    per_sm = PersistentKernels<std::decay_t<decltype(op)>>::blocks_per_sm();
    return cudaSuccess;
  });
  if (per_sm <= 0) return 0;
  const long long units = d.n / op_vec(d);
  long long g = (long long)sms * per_sm;       // every block resident: a cooperative launch
  const long long need = (units + kBlock - 1) / kBlock;
  if (need < g) g = need;
  if (g < 1) g = 1;
  if (g > kMaxPartialBlocks / 2) g = kMaxPartialBlocks / 2;   // two partial slots per block
  return (int)g;
}
cudaError_t launch_spcg_persistent(const OpDesc& d, int grid, cudaStream_t stream, Vecs v, State* st, Hist h,
                                   double* partials, unsigned long long timeout_ns, unsigned phantoms) {
  return with_op(d, [&](auto op) {
    return PersistentKernels<std::decay_t<decltype(op)>>::spcg(op, grid, stream, v, st, h, partials, timeout_ns,
                                                                phantoms);
  });
}
cudaError_t launch_apply(const OpDesc& d, const Launch& L, const double* x, double* y) {
  return with_op(d, [&](auto op) { return K<decltype(op)>::apply(op, L, x, y); });
}

}  // namespace pcgk
