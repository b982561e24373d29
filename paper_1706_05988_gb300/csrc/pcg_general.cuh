// General form of the pipelined iteration: a diagonal preconditioner M^{-1} = D^{-1}
// (Jacobi) and/or a variable shift sigma_i (Algorithm 4, Section 4.1; Algorithm 3 is
// the constant-shift case).  Binary64.
//
// Three variants of one fused sweep, chosen on the host:
//   JAC, constant shift   Algorithm 3 with its preconditioned recurrences
//   JAC, variable shift   Algorithm 4
//   M = I, variable shift Algorithm 4 with the M = I aliases u = r, q = s, p = t, m = w
// (M = I with a constant shift is the main p-CG-sh kernel.)  Each sweep does the SpMV
// n = A m, the recurrences in the order of Algorithm 4, m_{i+1} = D^{-1} w_{i+1} for
// the next sweep (so one launch per iteration) and the partial sums of (r, u), (w, u)
// and (r, r); the last block turns them into beta, alpha with
// delta = (w, u) + sigma_{i-1} (r, u).  shifts[0] = sigma_{-1}, shifts[k + 1] = sigma_k.
// With VAR = false the correction terms (sigma_i - sigma_{i-1}) ... are dropped at
// compile time rather than multiplied by zero: the FP64 pipe, not HBM, is the tighter
// bound on GB300.
#pragma once
#include "pcg_kernels.cuh"

// Resident blocks per SM the general sweep is compiled for (register cap 65536 / (256 * this)).
#ifndef PCG_GEN_MIN_BLOCKS
#define PCG_GEN_MIN_BLOCKS 2
#endif
// Most unknowns per thread of the Jacobi sweeps (nine vectors per unknown).
#ifndef PCG_GEN_JAC_MAX_VEC
#define PCG_GEN_JAC_MAX_VEC 2
#endif

namespace pcgk {

struct GenVecs {
  const double* b;
  double *x, *r, *w0, *w1, *z, *s, *t;   // t doubles as p when M = I
  double *u, *q, *p, *m0, *m1;           // JAC only
  const double* dinv;                    // JAC only
  const float* dinv32;                   // JAC, mixed precision only
  const double* shifts;                  // maxit + 1 shifts
};

template <class Op, bool JAC, bool VAR>
struct GeneralKernels {
  static cudaError_t w0(const Op& op, const Launch& L, GenVecs v, State* st, Hist h, double* partials);
  static cudaError_t iter(const Op& op, const Launch& L, GenVecs v, State* st, Hist h, double* partials);
  static int blocks_per_sm();
};

// y = d * x element-wise (u_0 = D^{-1} r_0); a no-op once the solve has stopped.
cudaError_t launch_diag_scale(const double* d, const double* x, double* y, int n, const State* st,
                              cudaStream_t stream);

#ifdef PCG_KERNELS_IMPL

// Stop tests and scalars after the partials (r,u), (w,u), (r,r) of iterate i.
__device__ __forceinline__ void finish_general(State* st, Hist h, const double* shifts, double ru, double wu,
                                               double rr, bool init) {
  const int i = init ? 0 : st->iter + 1;
  const double sprev = shifts[i];                  // sigma_{i-1}
  const double delta = wu + sprev * ru;
  const double rn = sqrt(rr);
  h.gamma[i] = ru;
  h.delta[i] = delta;
  h.rec[i] = rn;
  int status = ST_RUNNING;
  if (st->tol_abs > 0.0 && rn <= st->tol_abs) {
    status = ST_CONVERGED;
  } else if (i >= st->maxit) {
    status = ST_MAXIT;
  } else if (ru == 0.0) {
    status = ST_CONVERGED;
  } else if (init) {
    if (!(delta > 0.0) || !isfinite(delta)) {
      status = ST_BREAKDOWN;
    } else {
      h.alpha[0] = ru / delta;
      h.beta[0] = 0.0;
    }
  } else {
    const double beta = ru / h.gamma[i - 1];
    const double den = delta / ru - beta / h.alpha[i - 1];
    if (!(den > 0.0) || !isfinite(den)) {
      status = ST_BREAKDOWN;
    } else {
      h.alpha[i] = 1.0 / den;
      h.beta[i] = beta;
    }
  }
  st->iter = i;
  st->status = status;
  st->ticket = 0;
}

// Line 1 of Algorithm 4: u_0 = M^{-1} r_0 (JAC: already in v.u), w_0 = A u_0 - sigma_{-1} r_0,
// m_0 = M^{-1} w_0, auxiliary vectors zero.
template <class Op, bool JAC>
__global__ void __launch_bounds__(kBlock) k_gen_w0(Op op, GenVecs v, State* st, Hist h, double* partials) {
  constexpr int VEC = Op::VEC;
  if (st->status != ST_RUNNING) return;
  const double s0 = v.shifts[0];
  double ru = 0.0, wu = 0.0, rr = 0.0;
  const unsigned nc = (unsigned)op.units() * VEC;
  const auto stp = op.step(gridDim.x * kBlock);
  for (auto q = op.cursor(blockIdx.x * kBlock + threadIdx.x); q.c0 < nc; op.advance(q, stp)) {
    const int c0 = (int)q.c0;
    double uc[VEC], au[VEC], rv[VEC], w[VEC], zero[VEC];
    op.apply(JAC ? v.u : v.r, q, uc, au);
    if (JAC) {
      ld_stream<VEC>(v.r + c0, rv);
    } else {
#pragma unroll
      for (int e = 0; e < VEC; ++e) rv[e] = uc[e];
    }
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      w[e] = fma(-s0, rv[e], au[e]);
      zero[e] = 0.0;
      ru = fma(rv[e], uc[e], ru);
      wu = fma(w[e], uc[e], wu);
    }
    st_plain<VEC>(v.w0 + c0, w);
    st_plain<VEC>(v.z + c0, zero);
    st_plain<VEC>(v.s + c0, zero);
    st_plain<VEC>(v.t + c0, zero);
    if (JAC) {
      double d[VEC], m[VEC];
      ld_stream<VEC>(v.dinv + c0, d);
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        m[e] = d[e] * w[e];
        rr = fma(rv[e], rv[e], rr);
      }
      st_plain<VEC>(v.m0 + c0, m);
      st_plain<VEC>(v.q + c0, zero);
      st_plain<VEC>(v.p + c0, zero);
    }
  }
  if (JAC) {
    double vals[3] = {ru, wu, rr}, tot[3];
    if (!reduce_last_block<3>(vals, partials, &st->ticket, tot)) return;
    if (threadIdx.x == 0) finish_general(st, h, v.shifts, tot[0], tot[1], tot[2], true);
  } else {
    double vals[2] = {ru, wu}, tot[2];
    if (!reduce_last_block<2>(vals, partials, &st->ticket, tot)) return;
    if (threadIdx.x == 0) finish_general(st, h, v.shifts, tot[0], tot[1], tot[0], true);
  }
}

// One iteration of Algorithm 4 (order of its statement), n = A m fused.
template <class Op, bool JAC, bool VAR>
__global__ void __launch_bounds__(kBlock, PCG_GEN_MIN_BLOCKS) k_gen_iter(Op op, GenVecs v, State* st, Hist h,
                                                                        double* partials) {
  constexpr int VEC = Op::VEC;
  if (st->status != ST_RUNNING) return;
  const int it = st->iter;
  const double alpha = h.alpha[it], beta = h.beta[it];
  const double scur = v.shifts[it + 1];
  const double ds = VAR ? scur - v.shifts[it] : 0.0;
  const double asg = alpha * scur;
  const double* __restrict__ w = (it & 1) ? v.w1 : v.w0;
  double* __restrict__ wn = (it & 1) ? v.w0 : v.w1;
  const double* __restrict__ m = JAC ? ((it & 1) ? v.m1 : v.m0) : w;
  double* __restrict__ mn = (it & 1) ? v.m0 : v.m1;
  double ru = 0.0, wu = 0.0, rr = 0.0;
  const unsigned nc = (unsigned)op.units() * VEC;
  const auto stp = op.step(gridDim.x * kBlock);
  for (auto q = op.cursor(blockIdx.x * kBlock + threadIdx.x); q.c0 < nc; op.advance(q, stp)) {
    const int c0 = (int)q.c0;
    double mc[VEC], nv[VEC], wc[VEC], x[VEC], r[VEC], z[VEC], s[VEC], t[VEC];
    op.apply(m, q, mc, nv);
    if (JAC) {
      ld_stream<VEC>(w + c0, wc);
    } else {
#pragma unroll
      for (int e = 0; e < VEC; ++e) wc[e] = mc[e];
    }
    ld_stream<VEC>(v.x + c0, x);
    ld_stream<VEC>(v.r + c0, r);
    ld_stream<VEC>(v.z + c0, z);
    ld_stream<VEC>(v.s + c0, s);
    ld_stream<VEC>(v.t + c0, t);
    double u[VEC], qq[VEC], p[VEC], d[VEC];
    if (JAC) {
      ld_stream<VEC>(v.u + c0, u);
      ld_stream<VEC>(v.q + c0, qq);
      ld_stream<VEC>(v.p + c0, p);
      ld_stream<VEC>(v.dinv + c0, d);
    }
    double w1[VEC], m1[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      t[e] = fma(beta, t[e], r[e]);
      s[e] = fma(beta, s[e], wc[e]);
      z[e] = fma(beta, z[e], nv[e]);
      if (VAR) {
        s[e] = fma(-ds, t[e], s[e]);
        z[e] = fma(-ds, fma(scur, t[e], s[e]), z[e]);
      }
      const double rn = fma(-alpha, s[e], fma(-asg, t[e], r[e]));
      w1[e] = fma(-alpha, z[e], wc[e]);
      if (VAR) w1[e] = fma(-ds, r[e], w1[e]);
      if (JAC) {
        p[e] = fma(beta, p[e], u[e]);
        qq[e] = fma(beta, qq[e], mc[e]);
        if (VAR) qq[e] = fma(-ds, p[e], qq[e]);
        x[e] = fma(alpha, p[e], x[e]);
        const double un = fma(-alpha, qq[e], fma(-asg, p[e], u[e]));
        u[e] = un;
        m1[e] = d[e] * w1[e];
        ru = fma(rn, un, ru);
        wu = fma(w1[e], un, wu);
      } else {
        x[e] = fma(alpha, t[e], x[e]);
        wu = fma(w1[e], rn, wu);
      }
      rr = fma(rn, rn, rr);
      r[e] = rn;
    }
    st_stream<VEC>(v.x + c0, x);
    st_stream<VEC>(v.r + c0, r);
    st_stream<VEC>(v.z + c0, z);
    st_stream<VEC>(v.s + c0, s);
    st_stream<VEC>(v.t + c0, t);
    st_plain<VEC>(wn + c0, w1);
    if (JAC) {
      st_stream<VEC>(v.u + c0, u);
      st_stream<VEC>(v.q + c0, qq);
      st_stream<VEC>(v.p + c0, p);
      st_plain<VEC>(mn + c0, m1);
    }
  }
  if (JAC) {
    double vals[3] = {ru, wu, rr}, tot[3];
    if (!reduce_last_block<3>(vals, partials, &st->ticket, tot)) return;
    if (threadIdx.x == 0) finish_general(st, h, v.shifts, tot[0], tot[1], tot[2], false);
  } else {
    double vals[2] = {rr, wu}, tot[2];
    if (!reduce_last_block<2>(vals, partials, &st->ticket, tot)) return;
    if (threadIdx.x == 0) finish_general(st, h, v.shifts, tot[0], tot[1], tot[0], false);
  }
}

template <class Op, bool JAC, bool VAR>
cudaError_t GeneralKernels<Op, JAC, VAR>::w0(const Op& op, const Launch& L, GenVecs v, State* st, Hist h,
                                             double* partials) {
  k_gen_w0<Op, JAC><<<L.grid, L.block, 0, L.stream>>>(op, v, st, h, partials);
  return cudaGetLastError();
}
template <class Op, bool JAC, bool VAR>
cudaError_t GeneralKernels<Op, JAC, VAR>::iter(const Op& op, const Launch& L, GenVecs v, State* st, Hist h,
                                               double* partials) {
  k_gen_iter<Op, JAC, VAR><<<L.grid, L.block, 0, L.stream>>>(op, v, st, h, partials);
  return cudaGetLastError();
}
template <class Op, bool JAC, bool VAR>
int GeneralKernels<Op, JAC, VAR>::blocks_per_sm() {
  int nb = 0;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_gen_iter<Op, JAC, VAR>, kBlock, 0) == cudaSuccess
             ? nb
             : 0;
}

#define PCG_INSTANTIATE_GENERAL(OP)                \
  template struct GeneralKernels<OP, true, false>; \
  template struct GeneralKernels<OP, true, true>;  \
  template struct GeneralKernels<OP, false, true>;

#endif  // PCG_KERNELS_IMPL

}  // namespace pcgk
