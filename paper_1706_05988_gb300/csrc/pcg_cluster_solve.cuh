// Per-cluster solve of one system (Algorithm 3, M = I, binary64): shared by the batched
// launch (pcg_batch.cu) and the serving kernel (pcg_server.cu).
//
// The blocks of a thread-block cluster split the system's unknowns; every dot product
// reduces warp -> block -> cluster through distributed shared memory, and one cluster
// barrier per reduction stands in for the paper's global reduction.  Every block sums
// the cluster's partials in rank order, so all blocks hold identical scalars and take
// the same stop decisions.
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>

#ifndef PCG_KERNELS_IMPL
#define PCG_KERNELS_IMPL
#endif
#include "pcg_kernels.cuh"

namespace pcgk {
namespace cg = cooperative_groups;

// One system of the batch (device table).
struct BatchSys {
  int layout, n, nx, ny, nz, pad;
  const double *diag, *ax, *ay, *az;   // variable coefficients (stencils)
  const int *row_ptr, *col;            // CSR
  const double* val;
  const float *diag32, *ax32, *ay32, *az32, *val32;   // binary32 copies (mixed precision)
  long long off;                       // offset of the system's unknowns in every batch vector
  double sigma;
  double* log;                         // alpha_i, beta_i of iterations i < kScalarLog (nullptr: none)
};

// alpha_i, beta_i recorded per system and solve: log[i] = alpha_i, log[kScalarLog + i] =
// beta_i (NaN where the solve did not reach iteration i).  With mixed precision, i counts
// the inner iterations across restarts (a restart starts again from beta = 0).
constexpr int kScalarLog = 32;

// The values are collected in the block's shared memory while the solve runs (a constant
// address, and the cluster rank read from its special register: no register stays live
// for them across the iteration loop); the caller copies them to the system's log after
// the solve (scalar_log_flush), reading the log's address from global memory then.
__device__ __forceinline__ double* scalar_log_smem() {
  __shared__ double s[2 * kScalarLog];
  return s;
}

__device__ __forceinline__ bool scalar_log_owner() {
  return threadIdx.x == 0 && cg::this_cluster().block_rank() == 0;
}

__device__ __forceinline__ void scalar_log_clear(const BatchSys& d, unsigned rank) {
  (void)d;
  (void)rank;
  if (scalar_log_owner()) {
    double* s = scalar_log_smem();
    for (int i = 0; i < 2 * kScalarLog; ++i) s[i] = __longlong_as_double(0x7FF8000000000000LL);
  }
}

__device__ __forceinline__ void scalar_log(const BatchSys& d, unsigned rank, int i, double alpha, double beta) {
  (void)d;
  (void)rank;
  if (i < kScalarLog && scalar_log_owner()) {
    double* s = scalar_log_smem();
    s[i] = alpha;
    s[kScalarLog + i] = beta;
  }
}

// Copies the last solve's values to `log` (nullptr: none); thread 0 of the cluster's first block.
__device__ __forceinline__ void scalar_log_flush(double* log) {
  if (log != nullptr && scalar_log_owner()) {
    const double* s = scalar_log_smem();
    for (int i = 0; i < 2 * kScalarLog; ++i) log[i] = s[i];
  }
}

// Per-system results written by the kernel.
struct BatchOut {
  int iters, status;
  double bnorm, true_res;
};

// Every vector holds the batch's systems at their offsets.  Mixed precision keeps the
// binary32 vectors in the first half of a system's binary64-sized slot.
struct BatchVecs {
  const double* b;
  double *x, *r, *w0, *w1, *z, *s, *p;
  double *u, *q, *t, *m0, *m1, *u64;   // Jacobi only (u64: binary64 scratch of a mixed restart)
  const double* dinv;                  // Jacobi: D^{-1}
  const double* dinv32;                // Jacobi, mixed: D^{-1} rounded to binary32 (binary32 slot)
  long long stride;                    // vector k of this list lies at b + k * stride
};


template <int F>
struct FamilyOp;
template <>
struct FamilyOp<0> {
  using T = StencilOp<2, ST_LAP_FIXED, 1>;
};
template <>
struct FamilyOp<1> {
  using T = StencilOp<2, ST_VAR, 1>;
};
template <>
struct FamilyOp<2> {
  using T = StencilOp<3, ST_LAP_FIXED, 1>;
};
template <>
struct FamilyOp<3> {
  using T = StencilOp<3, ST_VAR, 1>;
};
template <>
struct FamilyOp<4> {
  using T = CsrOp;
};

template <int F>
__device__ __forceinline__ typename FamilyOp<F>::T make_op(const BatchSys& d) {
  typename FamilyOp<F>::T o;
  if constexpr (F == 4) {
    o.n = d.n;
    o.row_ptr = d.row_ptr;
    o.col = d.col;
    o.val = d.val;
  } else {
    o.n = d.n;
    o.nx = d.nx;
    o.ny = d.ny;
    o.nz = d.nz;
    o.nxny = d.nx * d.ny;
    o.diag = d.diag;
    o.ax = d.ax;
    o.ay = d.ay;
    o.az = d.az;
  }
  return o;
}

// Sum of NV values over the cluster: warp shuffles, block (shared memory), then the
// cluster's blocks read each other's block sums through DSMEM in rank order.
// `slot` alternates between calls so that one cluster barrier per call suffices.
template <int NV>
__device__ __forceinline__ void cluster_sum(cg::cluster_group& cl, double (&v)[NV], double (*part)[4], int slot,
                                            double (&tot)[NV]) {
  __shared__ double sh[kWarps][4];
  __shared__ double bc[4];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = warp_sum(v[q]);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) sh[wid][q] = v[q];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double a = 0.0;
      for (int k = 0; k < kWarps; ++k) a += sh[k][q];
      part[slot][q] = a;
    }
  }
  cl.sync();   // release/acquire at cluster scope: the partials and every global write are visible
  if (threadIdx.x == 0) {
    const unsigned C = cl.num_blocks();
    double a[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) a[q] = 0.0;
    for (unsigned rk = 0; rk < C; ++rk) {
      const double* rp = cl.map_shared_rank(&part[slot][0], rk);
#pragma unroll
      for (int q = 0; q < NV; ++q) a[q] += rp[q];
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) bc[q] = a[q];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) tot[q] = bc[q];
  __syncthreads();
}

// Algorithm 3 (M = I, binary64, x_0 = 0) for one system on the calling cluster; the
// result is returned in `res` (identical in every block of the cluster).  `slot`
// alternates the DSMEM partial slots between reductions (see cluster_sum).
template <int F>
__device__ __forceinline__ void cluster_solve(cg::cluster_group& cl, double (*part)[4], int& slot, const BatchSys& d,
                                              const BatchVecs& V, double tol, int maxit, BatchOut& res) {
  using Op = typename FamilyOp<F>::T;
  const unsigned rank = cl.block_rank(), C = cl.num_blocks();
  const Op op = make_op<F>(d);
  const double sigma = d.sigma;
  const long long off = d.off;
  const double* b = V.b + off;
  double *x = V.x + off, *r = V.r + off, *w0 = V.w0 + off, *w1 = V.w1 + off, *z = V.z + off, *s = V.s + off,
         *p = V.p + off;
  const unsigned nc = (unsigned)d.n;
  const auto stp = op.step(C * kBlock);
  const int first = (int)(rank * kBlock + threadIdx.x);

  scalar_log_clear(d, rank);
  // r_0 = b (x_0 = 0), ||b||
  double bb = 0.0;
  for (unsigned i = first; i < nc; i += C * kBlock) {
    const double bv = b[i];
    r[i] = bv;
    x[i] = 0.0;
    bb = fma(bv, bv, bb);
  }
  double t1[1] = {bb}, o1[1];
  cluster_sum<1>(cl, t1, part, slot, o1);
  slot ^= 1;
  const double bnorm = sqrt(o1[0]);
  const double tol_abs = tol * bnorm;

  // w_0 = A r_0 - sigma r_0; z = s = p = 0; gamma_0, (w_0, r_0)
  double g = 0.0, o = 0.0;
  for (auto q = op.cursor(first); q.c0 < nc; op.advance(q, stp)) {
    double rc[1], ar[1];
    op.apply(r, q, rc, ar);
    const double wv = fma(-sigma, rc[0], ar[0]);
    w0[q.c0] = wv;
    z[q.c0] = 0.0;
    s[q.c0] = 0.0;
    p[q.c0] = 0.0;
    g = fma(rc[0], rc[0], g);
    o = fma(wv, rc[0], o);
  }
  double t2[2] = {g, o}, o2[2];
  cluster_sum<2>(cl, t2, part, slot, o2);
  slot ^= 1;
  double gamma = o2[0], delta = o2[1] + sigma * o2[0];
  int status = ST_RUNNING, it = 0;
  double alpha = 0.0, beta = 0.0;
  if (tol_abs > 0.0 && sqrt(gamma) <= tol_abs) {
    status = ST_CONVERGED;
  } else if (maxit <= 0) {
    status = ST_MAXIT;
  } else if (gamma == 0.0) {
    status = ST_CONVERGED;
  } else if (!(delta > 0.0) || !isfinite(delta)) {
    status = ST_BREAKDOWN;
  } else {
    alpha = gamma / delta;
    scalar_log(d, rank, 0, alpha, 0.0);
  }
  while (status == ST_RUNNING) {
    const double asg = alpha * sigma;
    const double* __restrict__ w = (it & 1) ? w1 : w0;
    double* __restrict__ wn = (it & 1) ? w0 : w1;
    g = 0.0;
    o = 0.0;
    for (auto q = op.cursor(first); q.c0 < nc; op.advance(q, stp)) {
      const unsigned c = q.c0;
      double wc[1], nv[1];
      op.apply(w, q, wc, nv);
      const double zz = fma(beta, z[c], nv[0]);
      const double ss = fma(beta, s[c], wc[0]);
      const double rr = r[c];
      const double pp = fma(beta, p[c], rr);
      x[c] = fma(alpha, pp, x[c]);
      const double rn = fma(-alpha, ss, fma(-asg, pp, rr));
      const double wv = fma(-alpha, zz, wc[0]);
      z[c] = zz;
      s[c] = ss;
      p[c] = pp;
      r[c] = rn;
      wn[c] = wv;
      g = fma(rn, rn, g);
      o = fma(wv, rn, o);
    }
    double t[2] = {g, o}, tt[2];
    cluster_sum<2>(cl, t, part, slot, tt);
    slot ^= 1;
    ++it;
    const double gn = tt[0], dn = tt[1] + sigma * tt[0];
    if (tol_abs > 0.0 && sqrt(gn) <= tol_abs) {
      status = ST_CONVERGED;
    } else if (it >= maxit) {
      status = ST_MAXIT;
    } else if (gn == 0.0) {
      status = ST_CONVERGED;
    } else {
      const double bt = gn / gamma;
      const double den = dn / gn - bt / alpha;
      if (!(den > 0.0) || !isfinite(den)) {
        status = ST_BREAKDOWN;
      } else {
        alpha = 1.0 / den;
        beta = bt;
        scalar_log(d, rank, it, alpha, beta);
      }
    }
    gamma = gn;
  }

  // true residual ||b - A x||
  double tr = 0.0;
  for (auto q = op.cursor(first); q.c0 < nc; op.advance(q, stp)) {
    double xc[1], ax[1];
    op.apply(x, q, xc, ax);
    const double e = b[q.c0] - ax[0];
    tr = fma(e, e, tr);
  }
  double t3[1] = {tr}, o3[1];
  cluster_sum<1>(cl, t3, part, slot, o3);
  slot ^= 1;
  res.iters = it;
  res.status = status;
  res.bnorm = bnorm;
  res.true_res = sqrt(o3[0]);
}

}  // namespace pcgk
