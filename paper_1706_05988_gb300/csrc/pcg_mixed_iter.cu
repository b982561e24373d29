// Mixed-precision inner iteration: operator dispatch and kernel instances.
#define PCG_KERNELS_IMPL
#include <utility>

#include "pcg_mixed.cuh"
#include "pcg_mixed_jacobi.cuh"

namespace pcgk {
namespace {

template <int DIM, bool VAR, int VEC>
StencilOp32<DIM, VAR, VEC> make32(const OpDesc& d) {
  StencilOp32<DIM, VAR, VEC> o;
  o.n = d.n;
  o.nx = d.nx;
  o.ny = d.ny;
  o.nz = d.nz;
  o.nxny = d.nx * d.ny;
  o.diag = d.diag32;
  o.ax = d.ax32;
  o.ay = d.ay32;
  o.az = d.az32;
  return o;
}

template <int DIM, bool VAR, class F>
cudaError_t with_vec(const OpDesc& d, int vec, F&& f) {
  switch (vec) {
    case 4: return f(make32<DIM, VAR, 4>(d));
    case 2: return f(make32<DIM, VAR, 2>(d));
    default: return f(make32<DIM, VAR, 1>(d));
  }
}

// vec: unknowns per thread (mixed_vec or mixedj_vec)
template <class F>
cudaError_t with_op32(const OpDesc& d, int vec, F&& f) {
  const bool var = d.diag != nullptr;
  switch (d.layout) {
    case 0:
      return var ? with_vec<2, true>(d, vec, std::forward<F>(f)) : with_vec<2, false>(d, vec, std::forward<F>(f));
    case 1:
      return var ? with_vec<3, true>(d, vec, std::forward<F>(f)) : with_vec<3, false>(d, vec, std::forward<F>(f));
    case 2: {
      CsrOp32 o;
      o.n = d.n;
      o.row_ptr = d.row_ptr;
      o.col = d.col;
      o.val = d.val32;
      return f(o);
    }
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

int mixed_vec(const OpDesc& d) {
  if (d.layout == 2) return 1;
  if (d.nx % 4 == 0) return 4;
  if (d.nx % 2 == 0) return 2;
  return 1;
}

// The Jacobi inner iteration carries twice the vectors: fewer unknowns per thread keep it
// within the register cap of PCG_MIXED_MIN_BLOCKS resident blocks.
int mixedj_vec(const OpDesc& d) { return mixed_vec(d) < PCG_MIXED_JAC_MAX_VEC ? mixed_vec(d) : PCG_MIXED_JAC_MAX_VEC; }

cudaError_t launch_mx_iter(const OpDesc& d, const Launch& L, Vecs v, State* st, Hist h, double* partials) {
  return with_op32(d, mixed_vec(d),
                   [&](auto op) { return MixedIterKernels<decltype(op)>::iter(op, L, v, st, h, partials); });
}

cudaError_t launch_mxj_iter(const OpDesc& d, const Launch& L, const GenVecs& v, State* st, Hist h, double* partials) {
  return with_op32(d, mixedj_vec(d),
                   [&](auto op) { return MixedJacIterKernels<decltype(op)>::iter(op, L, v, st, h, partials); });
}

int grid_for_mixed(const OpDesc& d, int kind, int block);   // defined with the restart kernels

int mixedj_iter_blocks_per_sm(const OpDesc& d) {
  int nb = 0;
  with_op32(d, mixedj_vec(d), [&](auto op) {
    nb = MixedJacIterKernels<decltype(op)>::blocks_per_sm();
    return cudaSuccess;
  });
  return nb;
}

int mixed_iter_blocks_per_sm(const OpDesc& d) {
  int nb = 0;
  with_op32(d, mixed_vec(d), [&](auto op) {
    nb = MixedIterKernels<decltype(op)>::blocks_per_sm();
    return cudaSuccess;
  });
  return nb;
}

}  // namespace pcgk
