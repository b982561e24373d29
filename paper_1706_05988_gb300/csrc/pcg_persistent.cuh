// Persistent form of Algorithm 3 (M = I): one cooperative launch runs every
// iteration.  Between iterations a grid barrier stands in for the paper's global
// reduction.  After the barrier each block first issues the SpMV of its first unit
// of the next iteration (it does not need the new scalars) and only then sums the
// block partials of (r, r) and (w, r) -- the global reduction overlapped with the
// SpMV, as in the paper's Section 1 -- and derives alpha, beta itself.  Every block
// sums the same partials in the same order, so all blocks hold identical scalars
// and take the same stop decision.
//
// The grid barrier waits with a time limit (%globaltimer): a block that waits
// longer than timeout_ns gives up, the kernel ends with status ST_TIMEOUT and the
// host reports PCG_ETIMEOUT.  The launch is cooperative, so all blocks are resident.
#pragma once
#include <cuda/atomic>

#include "pcg_kernels.cuh"

namespace pcgk {

template <class Op>
struct PersistentKernels {
  static cudaError_t spcg(const Op& op, int grid, cudaStream_t stream, Vecs v, State* st, Hist h, double* partials,
                          unsigned long long timeout_ns, unsigned phantoms);
  static int blocks_per_sm();
};

#ifdef PCG_KERNELS_IMPL

// Sense-counting grid barrier on (st->bar_count, st->bar_gen).  `expected` is the
// number of arrivals that completes a phase.  Returns false after a timeout.
__device__ __forceinline__ bool grid_barrier(State* st, unsigned expected, unsigned long long timeout_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    cuda::atomic_ref<unsigned, cuda::thread_scope_device> gen(st->bar_gen), cnt(st->bar_count);
    const unsigned g = gen.load(cuda::memory_order_acquire);   // this phase cannot end before we arrive
    int ok = 1;
    __threadfence();
    if (cnt.fetch_add(1u, cuda::memory_order_acq_rel) == expected - 1) {
      cnt.store(0u, cuda::memory_order_relaxed);
      gen.store(g + 1u, cuda::memory_order_release);
    } else {
      const unsigned long long t0 = global_ns();
      while (gen.load(cuda::memory_order_acquire) == g) {
        if (global_ns() - t0 > timeout_ns) {
          ok = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <class Op>
__global__ void __launch_bounds__(kBlock, PCG_ITER_MIN_BLOCKS)
    k_spcg_persistent(Op op, Vecs v, State* st, Hist h, double* partials, unsigned long long timeout_ns,
                      unsigned phantoms) {
  constexpr int VEC = Op::VEC;
  __shared__ double sh[kWarps][2];
  __shared__ double s_scal[4];          // alpha, beta, gamma (of the current iteration), status
  if (st->status != ST_RUNNING) return;
  const unsigned G = gridDim.x;
  const double sigma = st->sigma, tol_abs = st->tol_abs;
  const int maxit = st->maxit;
  int it = st->iter;
  double alpha = h.alpha[it], beta = h.beta[it], gamma_prev = h.gamma[it];
  const unsigned nc = (unsigned)op.units() * VEC;
  const auto stp = op.step(G * kBlock);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;

  // the row of the first unit is computed before the scalars it does not need
  auto q = op.cursor(blockIdx.x * kBlock + threadIdx.x);
  double wc[VEC], nv[VEC];
  if (q.c0 < nc) op.apply((it & 1) ? v.w1 : v.w0, q, wc, nv);

  for (;;) {
    const double asg = alpha * sigma;
    const double* __restrict__ w = (it & 1) ? v.w1 : v.w0;
    double* __restrict__ wn = (it & 1) ? v.w0 : v.w1;
    double g = 0.0, o = 0.0;
    for (; q.c0 < nc; op.advance(q, stp)) {
      const int c0 = (int)q.c0;
      double z[VEC], s[VEC], p[VEC], x[VEC], r[VEC], w1[VEC];
      ld_stream<VEC>(v.z + c0, z);
      ld_stream<VEC>(v.s + c0, s);
      ld_stream<VEC>(v.p + c0, p);
      ld_stream<VEC>(v.x + c0, x);
      ld_stream<VEC>(v.r + c0, r);
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        z[e] = fma(beta, z[e], nv[e]);
        s[e] = fma(beta, s[e], wc[e]);
        p[e] = fma(beta, p[e], r[e]);
        x[e] = fma(alpha, p[e], x[e]);
        const double rn = fma(-alpha, s[e], fma(-asg, p[e], r[e]));
        const double wv = fma(-alpha, z[e], wc[e]);
        r[e] = rn;
        w1[e] = wv;
        g = fma(rn, rn, g);
        o = fma(wv, rn, o);
      }
      st_stream<VEC>(v.z + c0, z);
      st_stream<VEC>(v.s + c0, s);
      st_stream<VEC>(v.p + c0, p);
      st_stream<VEC>(v.x + c0, x);
      st_stream<VEC>(v.r + c0, r);
      st_plain<VEC>(wn + c0, w1);
      // row of the next unit of this sweep
      auto qn = q;
      op.advance(qn, stp);
      if (qn.c0 < nc) op.apply(w, qn, wc, nv);
    }
    // block partials of gamma_{i+1}, omega_{i+1} -> slot it & 1
    g = warp_sum(g);
    o = warp_sum(o);
    if (lane == 0) {
      sh[wid][0] = g;
      sh[wid][1] = o;
    }
    __syncthreads();
    double* slot = partials + (size_t)(it & 1) * 2 * G;
    if (threadIdx.x == 0) {
      double a = 0.0, c = 0.0;
      for (int k = 0; k < kWarps; ++k) {
        a += sh[k][0];
        c += sh[k][1];
      }
      slot[2 * blockIdx.x] = a;
      slot[2 * blockIdx.x + 1] = c;
    }
    if (!grid_barrier(st, G + phantoms, timeout_ns)) {
      if (threadIdx.x == 0) st->status = ST_TIMEOUT;
      return;
    }
    // next iteration's first row, issued before the global sum it does not depend on
    q = op.cursor(blockIdx.x * kBlock + threadIdx.x);
    if (q.c0 < nc) op.apply(wn, q, wc, nv);
    // global sum of the partials, same order in every block
    double a = 0.0, c = 0.0;
    for (unsigned b = threadIdx.x; b < G; b += kBlock) {
      a += __ldcg(slot + 2 * b);
      c += __ldcg(slot + 2 * b + 1);
    }
    a = warp_sum(a);
    c = warp_sum(c);
    __syncthreads();
    if (lane == 0) {
      sh[wid][0] = a;
      sh[wid][1] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double gamma = 0.0, omega = 0.0;
      for (int k = 0; k < kWarps; ++k) {
        gamma += sh[k][0];
        omega += sh[k][1];
      }
      // the scalar step of finish_spcg, evaluated identically in every block
      const int i = it + 1;
      const double delta = omega + sigma * gamma;
      const double rn = sqrt(gamma);
      int status = ST_RUNNING;
      double na = alpha, nb = 0.0;
      if (tol_abs > 0.0 && rn <= tol_abs) {
        status = ST_CONVERGED;
      } else if (i >= maxit) {
        status = ST_MAXIT;
      } else if (gamma == 0.0) {
        status = ST_CONVERGED;
      } else {
        nb = gamma / gamma_prev;
        const double den = delta / gamma - nb / alpha;
        if (!(den > 0.0) || !isfinite(den)) {
          status = ST_BREAKDOWN;
        } else {
          na = 1.0 / den;
        }
      }
      if (blockIdx.x == 0) {
        h.gamma[i] = gamma;
        h.delta[i] = delta;
        h.rec[i] = rn;
        if (status == ST_RUNNING) {
          h.alpha[i] = na;
          h.beta[i] = nb;
        }
        st->iter = i;
        st->status = status;
      }
      s_scal[0] = na;
      s_scal[1] = nb;
      s_scal[2] = gamma;
      s_scal[3] = (double)status;
    }
    __syncthreads();
    if ((int)s_scal[3] != ST_RUNNING) return;
    alpha = s_scal[0];
    beta = s_scal[1];
    gamma_prev = s_scal[2];
    ++it;
  }
}

template <class Op>
cudaError_t PersistentKernels<Op>::spcg(const Op& op, int grid, cudaStream_t stream, Vecs v, State* st, Hist h,
                                        double* partials, unsigned long long timeout_ns, unsigned phantoms) {
  Op o = op;
  void* args[] = {&o, &v, &st, &h, &partials, &timeout_ns, &phantoms};
  return cudaLaunchCooperativeKernel((const void*)k_spcg_persistent<Op>, dim3(grid), dim3(kBlock), args, 0, stream);
}
template <class Op>
int PersistentKernels<Op>::blocks_per_sm() {
  int nb = 0;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_spcg_persistent<Op>, kBlock, 0) == cudaSuccess ? nb
                                                                                                            : 0;
}

#endif  // PCG_KERNELS_IMPL

}  // namespace pcgk
