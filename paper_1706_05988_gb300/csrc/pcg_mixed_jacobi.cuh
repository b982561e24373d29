// Mixed-precision shifted pipelined CG with the Jacobi preconditioner M^{-1} = D^{-1}
// (Algorithm 3 with its preconditioned recurrences) and restarts (iterative refinement).
//
// Storage: x and r in binary64; u, w (two buffers), m = D^{-1} w (two buffers), z, q,
// s, t and p in binary32, each inside the first half of a binary64-sized buffer.
// Arithmetic: the auxiliary recurrences and the SpMV n = A m run in binary32; x and r
// in binary64 (binary32 operands widen exactly); (r, u), (w, u) and (r, r) accumulate
// in binary64; alpha, beta and sigma stay binary64.  m_{i+1} = D^{-1} w_{i+1} is formed
// as w_{i+1} is written, so an iteration is one launch.
// Restart (Algorithm 3, line 1, from the current x): r = b - A x in binary64 (the
// shared restart kernel), u_0 = D^{-1} r rounded to binary32 and kept also widened in a
// binary64 scratch vector, w_0 = A u_0 - sigma r with the binary64 operator applied to
// that scratch (so w_0 belongs to the stored u_0), rounded to binary32.
#pragma once
#include "pcg_general.cuh"
#include "pcg_mixed.cuh"

namespace pcgk {

template <class Op64>
struct MixedJacRestartKernels {
  static cudaError_t w0(const Op64& op, const Launch& L, GenVecs v, double* u64, State* st, Hist h,
                        double* partials);
  static int blocks_per_sm();
};

template <class Op32>
struct MixedJacIterKernels {
  static cudaError_t iter(const Op32& op, const Launch& L, GenVecs v, State* st, Hist h, double* partials);
  static int blocks_per_sm();
};

// u_0 = D^{-1} r rounded to binary32 (v.u) and widened back (u64); runs only on a restart.
cudaError_t launch_mxj_u0(const GenVecs& v, double* u64, int n, const State* st, cudaStream_t stream);

#ifdef PCG_KERNELS_IMPL

// Inner finisher with M^{-1}: gamma = (r, u), delta = (w, u) + sigma gamma, ||r|| for the
// inner tolerance; reaching it, an exact zero or a breakdown asks for a restart.
__device__ __forceinline__ void finish_mixed_jac(State* st, Hist h, double ru, double wu, double rr) {
  const int i = st->iter + 1;
  const double delta = wu + st->sigma * ru;
  const double rn = sqrt(rr);
  h.gamma[i] = ru;
  h.delta[i] = delta;
  h.rec[i] = rn;
  int status = ST_RUNNING;
  if (i >= st->maxit) {
    status = ST_MAXIT;
  } else if (rn <= st->tol_abs || ru == 0.0) {
    status = ST_RESTART;
  } else {
    const double beta = ru / h.gamma[i - 1];
    const double den = delta / ru - beta / h.alpha[i - 1];
    if (!(den > 0.0) || !isfinite(den)) {
      status = ST_RESTART;
    } else {
      h.alpha[i] = 1.0 / den;
      h.beta[i] = beta;
    }
  }
  st->iter = i;
  st->status = status;
  st->ticket = 0;
}

// Restart, part 3: w_0 = A u_0 - sigma r (binary64 operator on the widened u_0, stored
// rounded to binary32), m_0 = D^{-1} w_0 in binary32, z = q = s = t = p = 0,
// gamma = (r, u_0), delta = (w_0, u_0) + sigma gamma, alpha = gamma / delta, beta = 0.
template <class Op64>
__global__ void __launch_bounds__(kBlock) k_mxj_w0(Op64 op, GenVecs v, const double* __restrict__ u64, State* st,
                                                   Hist h, double* partials) {
  constexpr int VEC = Op64::VEC;
  if (st->status != ST_RESTART) return;
  const double sigma = st->sigma;
  const bool odd = st->iter & 1;
  float* __restrict__ w = reinterpret_cast<float*>(odd ? v.w1 : v.w0);
  float* __restrict__ m = reinterpret_cast<float*>(odd ? v.m1 : v.m0);
  float* __restrict__ zf = reinterpret_cast<float*>(v.z);
  float* __restrict__ qf = reinterpret_cast<float*>(v.q);
  float* __restrict__ sf = reinterpret_cast<float*>(v.s);
  float* __restrict__ tf = reinterpret_cast<float*>(v.t);
  float* __restrict__ pf = reinterpret_cast<float*>(v.p);
  double ru = 0.0, wu = 0.0, rr = 0.0;
  const unsigned nc = (unsigned)op.units() * VEC;
  const auto stp = op.step(gridDim.x * kBlock);
  for (auto q = op.cursor(blockIdx.x * kBlock + threadIdx.x); q.c0 < nc; op.advance(q, stp)) {
    const int c0 = (int)q.c0;
    double uc[VEC], au[VEC], rv[VEC];
    op.apply(u64, q, uc, au);
    ld_stream<VEC>(v.r + c0, rv);
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      const float w32 = f32_of(fma(-sigma, rv[e], au[e]));
      w[c0 + e] = w32;
      m[c0 + e] = v.dinv32[c0 + e] * w32;
      zf[c0 + e] = 0.f;
      qf[c0 + e] = 0.f;
      sf[c0 + e] = 0.f;
      tf[c0 + e] = 0.f;
      pf[c0 + e] = 0.f;
      ru = fma(rv[e], uc[e], ru);
      wu = fma(f64_of(w32), uc[e], wu);
      rr = fma(rv[e], rv[e], rr);
    }
  }
  double vals[3] = {ru, wu, rr}, tot[3];
  if (!reduce_last_block<3>(vals, partials, &st->ticket, tot)) return;
  if (threadIdx.x == 0) {
    const int i = st->iter;
    const double gamma = tot[0], delta = tot[1] + sigma * gamma;
    h.gamma[i] = gamma;
    h.delta[i] = delta;
    h.rec[i] = sqrt(tot[2]);
    if (!(delta > 0.0) || !isfinite(delta)) {
      st->status = ST_BREAKDOWN;
    } else {
      h.alpha[i] = gamma / delta;
      h.beta[i] = 0.0;
      st->status = ST_RUNNING;
    }
    st->ticket = 0;
  }
}

// One inner iteration with M^{-1} = D^{-1}: binary32 auxiliary recurrences, binary64 x, r, dots.
template <class Op32>
__global__ void __launch_bounds__(kBlock, PCG_MIXED_MIN_BLOCKS) k_mxj_iter(Op32 op, GenVecs v, State* st, Hist h, double* partials) {
  constexpr int VEC = Op32::VEC;
  if (st->status != ST_RUNNING) return;
  const int it = st->iter;
  const double alpha = h.alpha[it], beta = h.beta[it];
  const double asg = alpha * st->sigma;
  const float alpha32 = f32_of(alpha), beta32 = f32_of(beta), asg32 = f32_of(asg);
  const bool odd = it & 1;
  const float* __restrict__ w = reinterpret_cast<const float*>(odd ? v.w1 : v.w0);
  float* __restrict__ wn = reinterpret_cast<float*>(odd ? v.w0 : v.w1);
  const float* __restrict__ m = reinterpret_cast<const float*>(odd ? v.m1 : v.m0);
  float* __restrict__ mn = reinterpret_cast<float*>(odd ? v.m0 : v.m1);
  float* __restrict__ zf = reinterpret_cast<float*>(v.z);
  float* __restrict__ qf = reinterpret_cast<float*>(v.q);
  float* __restrict__ sf = reinterpret_cast<float*>(v.s);
  float* __restrict__ tf = reinterpret_cast<float*>(v.t);
  float* __restrict__ pf = reinterpret_cast<float*>(v.p);
  float* __restrict__ uf = reinterpret_cast<float*>(v.u);
  double ru = 0.0, wu = 0.0, rr = 0.0;
  const unsigned nc = (unsigned)op.units() * VEC;
  const auto stp = op.step(gridDim.x * kBlock);
  for (auto q = op.cursor(blockIdx.x * kBlock + threadIdx.x); q.c0 < nc; op.advance(q, stp)) {
    const int c0 = (int)q.c0;
    float mc[VEC], nv[VEC], wc[VEC], z[VEC], qq[VEC], s[VEC], t[VEC], p[VEC], u[VEC], d[VEC], w1[VEC], m1[VEC];
    double x[VEC], r[VEC];
    op.apply(m, q, mc, nv);
    ldf<VEC>(w + c0, wc);
    ldf<VEC>(zf + c0, z);
    ldf<VEC>(qf + c0, qq);
    ldf<VEC>(sf + c0, s);
    ldf<VEC>(tf + c0, t);
    ldf<VEC>(pf + c0, p);
    ldf<VEC>(uf + c0, u);
    ldf<VEC>(v.dinv32 + c0, d);
    ldd<VEC>(v.x + c0, x);
    ldd<VEC>(v.r + c0, r);
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      z[e] = fmaf(beta32, z[e], nv[e]);
      qq[e] = fmaf(beta32, qq[e], mc[e]);
      s[e] = fmaf(beta32, s[e], wc[e]);
      t[e] = fmaf(beta32, t[e], f32_of(r[e]));
      p[e] = fmaf(beta32, p[e], u[e]);
      x[e] = fma(alpha, f64_of(p[e]), x[e]);
      const double rn = fma(-alpha, f64_of(s[e]), fma(-asg, f64_of(t[e]), r[e]));
      u[e] = fmaf(-alpha32, qq[e], fmaf(-asg32, p[e], u[e]));
      w1[e] = fmaf(-alpha32, z[e], wc[e]);
      m1[e] = d[e] * w1[e];
      r[e] = rn;
      const double ud = f64_of(u[e]);
      ru = fma(rn, ud, ru);
      wu = fma(f64_of(w1[e]), ud, wu);
      rr = fma(rn, rn, rr);
    }
    stf<VEC>(zf + c0, z);
    stf<VEC>(qf + c0, qq);
    stf<VEC>(sf + c0, s);
    stf<VEC>(tf + c0, t);
    stf<VEC>(pf + c0, p);
    stf<VEC>(uf + c0, u);
    std_<VEC>(v.x + c0, x);
    std_<VEC>(v.r + c0, r);
    stf<VEC>(wn + c0, w1, false);
    stf<VEC>(mn + c0, m1, false);
  }
  double vals[3] = {ru, wu, rr}, tot[3];
  if (!reduce_last_block<3>(vals, partials, &st->ticket, tot)) return;
  if (threadIdx.x == 0) finish_mixed_jac(st, h, tot[0], tot[1], tot[2]);
}

template <class Op64>
cudaError_t MixedJacRestartKernels<Op64>::w0(const Op64& op, const Launch& L, GenVecs v, double* u64, State* st,
                                             Hist h, double* partials) {
  k_mxj_w0<Op64><<<L.grid, L.block, 0, L.stream>>>(op, v, u64, st, h, partials);
  return cudaGetLastError();
}
template <class Op64>
int MixedJacRestartKernels<Op64>::blocks_per_sm() {
  int nb = 0;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_mxj_w0<Op64>, kBlock, 0) == cudaSuccess ? nb : 0;
}
template <class Op32>
cudaError_t MixedJacIterKernels<Op32>::iter(const Op32& op, const Launch& L, GenVecs v, State* st, Hist h,
                                            double* partials) {
  k_mxj_iter<Op32><<<L.grid, L.block, 0, L.stream>>>(op, v, st, h, partials);
  return cudaGetLastError();
}
template <class Op32>
int MixedJacIterKernels<Op32>::blocks_per_sm() {
  int nb = 0;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_mxj_iter<Op32>, kBlock, 0) == cudaSuccess ? nb : 0;
}

#endif  // PCG_KERNELS_IMPL

}  // namespace pcgk
