// Mixed-precision shifted pipelined CG with restarts (iterative refinement).
//
// Storage: x and r in binary64; w (double-buffered), z, s and p in binary32.
// Arithmetic: the auxiliary recurrences z, s, p, w and the SpMV n = A w run in
// binary32; x_{i+1} = x_i + alpha p_i and r_{i+1} = r_i - alpha s_i - alpha sigma p_i
// run in binary64 (binary32 operands widen exactly); the dot products (r, r)
// and (w, r) accumulate exact binary64 products in binary64; alpha, beta and
// sigma stay binary64 (rounded once to binary32 for the binary32 recurrences).
// Restart (Algorithm 3, line 1, from the current x): r = b - A x with the
// binary64 operator, w_0 = A r - sigma r rounded to binary32, z = s = p = 0,
// beta = 0.  A restart happens when the inner recursive residual reaches eta
// times the true residual of the previous restart; the solve ends when the
// true residual reaches tol ||b||, or stalls, or after maxit iterations.
#pragma once
#include "pcg_convert.cuh"
#include "pcg_kernels.cuh"

// Resident blocks per SM the inner-iteration kernels are compiled for (register cap
// 65536 / (256 * this)): they stream memory with little arithmetic, so occupancy
// hides latency better than the registers that a wider cap would give.
#ifndef PCG_MIXED_MIN_BLOCKS
#define PCG_MIXED_MIN_BLOCKS 3
#endif
// Most unknowns per thread of the Jacobi inner iteration.
#ifndef PCG_MIXED_JAC_MAX_VEC
#define PCG_MIXED_JAC_MAX_VEC 2
#endif

namespace pcgk {

// ---------------------------------------------------------------- binary32 operators

template <int DIM, bool VAR, int VEC_>
struct StencilOp32 {
  static constexpr int VEC = VEC_;
  int n, nx, ny, nz, nxny;
  const float *diag, *ax, *ay, *az;

  __host__ __device__ int units() const { return n / VEC; }

#ifdef PCG_KERNELS_IMPL
  struct Cursor {
    unsigned c0, i0, j, k;
  };
  struct Step {
    unsigned dc, di, dj, dk;
  };
  __device__ __forceinline__ Cursor cursor(int u) const {
    Cursor q;
    q.c0 = (unsigned)u * VEC;
    q.i0 = q.c0 % (unsigned)nx;
    const unsigned t = q.c0 / (unsigned)nx;
    q.j = t % (unsigned)ny;
    q.k = t / (unsigned)ny;
    return q;
  }
  __device__ __forceinline__ Step step(unsigned stride_units) const {
    Step s;
    s.dc = stride_units * VEC;
    s.di = s.dc % (unsigned)nx;
    const unsigned rows = s.dc / (unsigned)nx;
    s.dj = rows % (unsigned)ny;
    s.dk = rows / (unsigned)ny;
    return s;
  }
  __device__ __forceinline__ void advance(Cursor& q, const Step& s) const {
    q.c0 += s.dc;
    q.i0 += s.di;
    const unsigned cx = q.i0 >= (unsigned)nx;
    q.i0 -= cx ? (unsigned)nx : 0u;
    q.j += s.dj + cx;
    const unsigned cy = q.j >= (unsigned)ny;
    q.j -= cy ? (unsigned)ny : 0u;
    q.k += s.dk + cy;
  }

  template <int V>
  __device__ __forceinline__ static void ldg(const float* p, float (&o)[V]) {
    if constexpr (V == 4) {
      const float4 t = __ldg(reinterpret_cast<const float4*>(p));
      o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
    } else if constexpr (V == 2) {
      const float2 t = __ldg(reinterpret_cast<const float2*>(p));
      o[0] = t.x; o[1] = t.y;
    } else {
      o[0] = __ldg(p);
    }
  }
  template <int V>
  __device__ __forceinline__ static void ldg_if(bool ok, const float* p, float (&o)[V]) {
    if (ok) {
      ldg<V>(p, o);
    } else {
#pragma unroll
      for (int e = 0; e < V; ++e) o[e] = 0.f;
    }
  }

  // wc = w at the unit's unknowns, aw = (A w) there, in binary32.
  __device__ __forceinline__ void apply(const float* __restrict__ w, const Cursor& q, float (&wc)[VEC],
                                        float (&aw)[VEC]) const {
    const unsigned c0 = q.c0, i0 = q.i0, j = q.j, k = q.k;
    const bool has_ym = j > 0, has_yp = j + 1 < (unsigned)ny;
    const bool has_zm = DIM == 3 && k > 0, has_zp = DIM == 3 && k + 1 < (unsigned)nz;
    float c[VEC], ym[VEC], yp[VEC], zm[VEC], zp[VEC];
    ldg<VEC>(w + c0, c);
    ldg_if<VEC>(has_ym, w + c0 - nx, ym);
    ldg_if<VEC>(has_yp, w + c0 + nx, yp);
    if (DIM == 3) {
      ldg_if<VEC>(has_zm, w + c0 - nxny, zm);
      ldg_if<VEC>(has_zp, w + c0 + nxny, zp);
    }
    const float xl = i0 > 0 ? __ldg(w + c0 - 1) : 0.f;
    const float xr = i0 + VEC < (unsigned)nx ? __ldg(w + c0 + VEC) : 0.f;
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      const float xm = e == 0 ? xl : c[e - 1];
      const float xp = e == VEC - 1 ? xr : c[e + 1];
      wc[e] = c[e];
      if (!VAR) {
        float s = (xm + xp) + (ym[e] + yp[e]);
        if (DIM == 3) s += zm[e] + zp[e];
        aw[e] = fmaf(DIM == 3 ? 6.f : 4.f, c[e], -s);
      } else {
        aw[e] = 0.f;   // variable coefficients: below
      }
    }
    if (VAR) {
      float d[VEC], fx[VEC], fy[VEC], fyp[VEC], fz[VEC], fzp[VEC];
      ldg<VEC>(diag + c0, d);
      ldg<VEC>(ax + c0, fx);
      ldg<VEC>(ay + c0, fy);
      ldg_if<VEC>(has_yp, ay + c0 + nx, fyp);
      if (DIM == 3) {
        ldg<VEC>(az + c0, fz);
        ldg_if<VEC>(has_zp, az + c0 + nxny, fzp);
      }
      const float fxr = i0 + VEC < (unsigned)nx ? __ldg(ax + c0 + VEC) : 0.f;
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        const float xm = e == 0 ? xl : c[e - 1];
        const float xp = e == VEC - 1 ? xr : c[e + 1];
        const float fxp = e == VEC - 1 ? fxr : fx[e + 1];
        float a = d[e] * c[e];
        a = fmaf(-fx[e], xm, a);
        a = fmaf(-fxp, xp, a);
        a = fmaf(-fy[e], ym[e], a);
        a = fmaf(-fyp[e], yp[e], a);
        if (DIM == 3) {
          a = fmaf(-fz[e], zm[e], a);
          a = fmaf(-fzp[e], zp[e], a);
        }
        aw[e] = a;
      }
    }
  }
#endif
};

struct CsrOp32 {
  static constexpr int VEC = 1;
  int n;
  const int *row_ptr, *col;
  const float* val;

  __host__ __device__ int units() const { return n; }

#ifdef PCG_KERNELS_IMPL
  struct Cursor {
    unsigned c0;
  };
  struct Step {
    unsigned dc;
  };
  __device__ __forceinline__ Cursor cursor(int u) const { return Cursor{(unsigned)u}; }
  __device__ __forceinline__ Step step(unsigned stride_units) const { return Step{stride_units}; }
  __device__ __forceinline__ void advance(Cursor& q, const Step& s) const { q.c0 += s.dc; }
  __device__ __forceinline__ void apply(const float* __restrict__ w, const Cursor& q, float (&wc)[1],
                                        float (&aw)[1]) const {
    const int u = (int)q.c0;
    const int beg = __ldg(row_ptr + u), end = __ldg(row_ptr + u + 1);
    float a = 0.f;
    for (int k = beg; k < end; ++k) a = fmaf(__ldg(val + k), __ldg(w + __ldg(col + k)), a);
    aw[0] = a;
    wc[0] = __ldg(w + u);
  }
#endif
};

template <class Op64>
struct MixedRestartKernels {
  static cudaError_t restart(const Op64& op, const Launch& L, Vecs v, State* st, Hist h, double* partials);
  static cudaError_t w0(const Op64& op, const Launch& L, Vecs v, State* st, Hist h, double* partials);
  static int blocks_per_sm(int kind);
};

template <class Op32>
struct MixedIterKernels {
  static cudaError_t iter(const Op32& op, const Launch& L, Vecs v, State* st, Hist h, double* partials);
  static int blocks_per_sm();
};

#ifdef PCG_KERNELS_IMPL

template <int V>
__device__ __forceinline__ void ldf(const float* p, float (&o)[V]) {
  if constexpr (V == 4) {
    const float4 t = __ldcs(reinterpret_cast<const float4*>(p));
    o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
  } else if constexpr (V == 2) {
    const float2 t = __ldcs(reinterpret_cast<const float2*>(p));
    o[0] = t.x; o[1] = t.y;
  } else {
    o[0] = __ldcs(p);
  }
}
template <int V>
__device__ __forceinline__ void stf(float* p, const float (&o)[V], bool stream = true) {
  if constexpr (V == 4) {
    const float4 t = make_float4(o[0], o[1], o[2], o[3]);
    if (stream) __stcs(reinterpret_cast<float4*>(p), t); else *reinterpret_cast<float4*>(p) = t;
  } else if constexpr (V == 2) {
    const float2 t = make_float2(o[0], o[1]);
    if (stream) __stcs(reinterpret_cast<float2*>(p), t); else *reinterpret_cast<float2*>(p) = t;
  } else {
    if (stream) __stcs(p, o[0]); else *p = o[0];
  }
}
// binary64 vectors with V = 4 use two 128-bit accesses
template <int V>
__device__ __forceinline__ void ldd(const double* p, double (&o)[V]) {
  if constexpr (V >= 2) {
#pragma unroll
    for (int h = 0; h < V; h += 2) {
      const double2 t = __ldcs(reinterpret_cast<const double2*>(p + h));
      o[h] = t.x;
      o[h + 1] = t.y;
    }
  } else {
    o[0] = __ldcs(p);
  }
}
template <int V>
__device__ __forceinline__ void std_(double* p, const double (&o)[V]) {
  if constexpr (V >= 2) {
#pragma unroll
    for (int h = 0; h < V; h += 2) __stcs(reinterpret_cast<double2*>(p + h), make_double2(o[h], o[h + 1]));
  } else {
    __stcs(p, o[0]);
  }
}

// Finisher of the inner iteration: like finish_spcg, but reaching the inner
// tolerance, an exact zero or a breakdown asks for a restart.
__device__ __forceinline__ void finish_mixed(State* st, Hist h, double gamma, double omega) {
  const int i = st->iter + 1;
  const double delta = omega + st->sigma * gamma;
  const double rn = sqrt(gamma);
  h.gamma[i] = gamma;
  h.delta[i] = delta;
  h.rec[i] = rn;
  int status = ST_RUNNING;
  if (i >= st->maxit) {
    status = ST_MAXIT;
  } else if (rn <= st->tol_abs || gamma == 0.0) {
    status = ST_RESTART;
  } else {
    const double beta = gamma / h.gamma[i - 1];
    const double den = delta / gamma - beta / h.alpha[i - 1];
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

// One inner iteration (M = I): binary32 auxiliary recurrences, binary64 x, r and dots.
template <class Op32>
__global__ void __launch_bounds__(kBlock, PCG_MIXED_MIN_BLOCKS) k_mx_iter(Op32 op, Vecs v, State* st, Hist h, double* partials) {
  constexpr int VEC = Op32::VEC;
  if (st->status != ST_RUNNING) return;
  const int it = st->iter;
  const double alpha = h.alpha[it], beta = h.beta[it];
  const double asg = alpha * st->sigma;
  const float alpha32 = f32_of(alpha), beta32 = f32_of(beta);
  const float* __restrict__ w = reinterpret_cast<const float*>((it & 1) ? v.w1 : v.w0);
  float* __restrict__ wn = reinterpret_cast<float*>((it & 1) ? v.w0 : v.w1);
  float* __restrict__ zf = reinterpret_cast<float*>(v.z);
  float* __restrict__ sf = reinterpret_cast<float*>(v.s);
  float* __restrict__ pf = reinterpret_cast<float*>(v.p);
  double g = 0.0, o = 0.0;
  const unsigned nc = (unsigned)op.units() * VEC;
  const auto stp = op.step(gridDim.x * kBlock);
  for (auto q = op.cursor(blockIdx.x * kBlock + threadIdx.x); q.c0 < nc; op.advance(q, stp)) {
    const int c0 = (int)q.c0;
    float wc[VEC], nv[VEC], z[VEC], s[VEC], p[VEC], w1[VEC];
    double x[VEC], r[VEC];
    op.apply(w, q, wc, nv);
    ldf<VEC>(zf + c0, z);
    ldf<VEC>(sf + c0, s);
    ldf<VEC>(pf + c0, p);
    ldd<VEC>(v.x + c0, x);
    ldd<VEC>(v.r + c0, r);
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      z[e] = fmaf(beta32, z[e], nv[e]);
      s[e] = fmaf(beta32, s[e], wc[e]);
      p[e] = fmaf(beta32, p[e], f32_of(r[e]));
      const double pd = f64_of(p[e]), sd = f64_of(s[e]);
      x[e] = fma(alpha, pd, x[e]);
      const double rn = fma(-alpha, sd, fma(-asg, pd, r[e]));
      w1[e] = fmaf(-alpha32, z[e], wc[e]);
      r[e] = rn;
      g = fma(rn, rn, g);
      o = fma(f64_of(w1[e]), rn, o);
    }
    stf<VEC>(zf + c0, z);
    stf<VEC>(sf + c0, s);
    stf<VEC>(pf + c0, p);
    std_<VEC>(v.x + c0, x);
    std_<VEC>(v.r + c0, r);
    stf<VEC>(wn + c0, w1, false);
  }
  double vals[2] = {g, o}, tot[2];
  if (!reduce_last_block<2>(vals, partials, &st->ticket, tot)) return;
  if (threadIdx.x == 0) finish_mixed(st, h, tot[0], tot[1]);
}

// Restart, part 1: r = b - A x in binary64, ||r||, ||b|| -> convergence / stall tests.
template <class Op64>
__global__ void __launch_bounds__(kBlock) k_mx_restart(Op64 op, Vecs v, State* st, Hist h, double* partials) {
  constexpr int VEC = Op64::VEC;
  if (st->status != ST_RESTART) return;
  double rr = 0.0, bb = 0.0;
  const unsigned nc = (unsigned)op.units() * VEC;
  const auto stp = op.step(gridDim.x * kBlock);
  for (auto q = op.cursor(blockIdx.x * kBlock + threadIdx.x); q.c0 < nc; op.advance(q, stp)) {
    const int c0 = (int)q.c0;
    double xc[VEC], ax[VEC], bv[VEC], rv[VEC];
    op.apply(v.x, q, xc, ax);
    ld_stream<VEC>(v.b + c0, bv);
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      rv[e] = bv[e] - ax[e];
      rr = fma(rv[e], rv[e], rr);
      bb = fma(bv[e], bv[e], bb);
    }
    st_plain<VEC>(v.r + c0, rv);
  }
  double vals[2] = {rr, bb}, tot[2];
  if (!reduce_last_block<2>(vals, partials, &st->ticket, tot)) return;
  if (threadIdx.x == 0) {
    const int i = st->iter;
    const double rt = sqrt(tot[0]);
    st->bnorm = sqrt(tot[1]);
    h.tru[i] = rt;
    h.gap[i] = 0.0;                       // r was just set to the true residual
    if (rt <= st->tol_rel * st->bnorm || tot[0] == 0.0) {
      st->status = ST_CONVERGED;
    } else if (st->restarts > 0 && !(rt < st->rprev)) {
      st->status = ST_STALLED;
    } else if (st->restarts >= st->max_restarts) {
      st->status = ST_STALLED;
    } else {
      // inner target: eta times this true residual, but not below half the outer target
      st->tol_abs = fmax(st->eta * rt, 0.5 * st->tol_rel * st->bnorm);
      st->rprev = rt;
      st->restarts += 1;
    }
    st->ticket = 0;
  }
}

// Restart, part 2: w_0 = A r - sigma r (binary64, stored rounded to binary32), z = s = p = 0,
// gamma = (r, r), delta = (w_0, r) + sigma gamma, alpha = gamma / delta, beta = 0.
template <class Op64>
__global__ void __launch_bounds__(kBlock) k_mx_w0(Op64 op, Vecs v, State* st, Hist h, double* partials) {
  constexpr int VEC = Op64::VEC;
  if (st->status != ST_RESTART) return;
  const double sigma = st->sigma;
  float* __restrict__ w = reinterpret_cast<float*>((st->iter & 1) ? v.w1 : v.w0);
  float* __restrict__ zf = reinterpret_cast<float*>(v.z);
  float* __restrict__ sf = reinterpret_cast<float*>(v.s);
  float* __restrict__ pf = reinterpret_cast<float*>(v.p);
  double g = 0.0, o = 0.0;
  const unsigned nc = (unsigned)op.units() * VEC;
  const auto stp = op.step(gridDim.x * kBlock);
  for (auto q = op.cursor(blockIdx.x * kBlock + threadIdx.x); q.c0 < nc; op.advance(q, stp)) {
    const int c0 = (int)q.c0;
    double rc[VEC], ar[VEC];
    op.apply(v.r, q, rc, ar);
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      const float w32 = f32_of(fma(-sigma, rc[e], ar[e]));
      w[c0 + e] = w32;
      zf[c0 + e] = 0.f;
      sf[c0 + e] = 0.f;
      pf[c0 + e] = 0.f;
      g = fma(rc[e], rc[e], g);
      o = fma(f64_of(w32), rc[e], o);
    }
  }
  double vals[2] = {g, o}, tot[2];
  if (!reduce_last_block<2>(vals, partials, &st->ticket, tot)) return;
  if (threadIdx.x == 0) {
    const int i = st->iter;
    const double gamma = tot[0], delta = tot[1] + sigma * gamma;
    h.gamma[i] = gamma;
    h.delta[i] = delta;
    h.rec[i] = sqrt(gamma);
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

template <class Op64>
cudaError_t MixedRestartKernels<Op64>::restart(const Op64& op, const Launch& L, Vecs v, State* st, Hist h,
                                               double* partials) {
  k_mx_restart<Op64><<<L.grid, L.block, 0, L.stream>>>(op, v, st, h, partials);
  return cudaGetLastError();
}
template <class Op64>
cudaError_t MixedRestartKernels<Op64>::w0(const Op64& op, const Launch& L, Vecs v, State* st, Hist h,
                                          double* partials) {
  k_mx_w0<Op64><<<L.grid, L.block, 0, L.stream>>>(op, v, st, h, partials);
  return cudaGetLastError();
}
template <class Op64>
int MixedRestartKernels<Op64>::blocks_per_sm(int kind) {
  int nb = 0;
  const cudaError_t e = kind == KM_RESTART
                            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_mx_restart<Op64>, kBlock, 0)
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_mx_w0<Op64>, kBlock, 0);
  return e == cudaSuccess ? nb : 0;
}
template <class Op32>
cudaError_t MixedIterKernels<Op32>::iter(const Op32& op, const Launch& L, Vecs v, State* st, Hist h,
                                         double* partials) {
  k_mx_iter<Op32><<<L.grid, L.block, 0, L.stream>>>(op, v, st, h, partials);
  return cudaGetLastError();
}
template <class Op32>
int MixedIterKernels<Op32>::blocks_per_sm() {
  int nb = 0;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_mx_iter<Op32>, kBlock, 0) == cudaSuccess ? nb : 0;
}

#endif  // PCG_KERNELS_IMPL

}  // namespace pcgk
