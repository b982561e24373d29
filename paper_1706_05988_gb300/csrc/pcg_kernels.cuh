// Device code of the solver: operators, the two-level reduction with its
// finishers, and the kernels of Algorithms 1 and 3 (arXiv 1706.05988).
//
// Layout: every vector is a contiguous binary64 array; a thread handles VEC
// consecutive unknowns (VEC = 2 -> 128-bit loads/stores) of a grid-stride loop
// over "units" of VEC unknowns.  The grid is sized to the resident capacity of
// the GPU so that each block accumulates its dot-product partials over many
// units and the global reduction reads only one partial per block.
//
// Definitions are compiled only where PCG_KERNELS_IMPL is defined (one
// translation unit per operator family); other units see declarations.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "pcg_check.cuh"
#include "pcg_ffdot.cuh"
#include "pcg_tma.cuh"
#include "pcg_fixedsum.cuh"
#include "pcg_internal.h"

namespace pcgk {

constexpr int kBlock = kBlockThreads;

// Resident blocks per SM the fused iteration kernel is compiled for (register cap).
#ifndef PCG_ITER_MIN_BLOCKS
#define PCG_ITER_MIN_BLOCKS 4
#endif
constexpr int kWarps = kBlock / 32;

// ---------------------------------------------------------------- operators

// Cell-centred stencil on an nx x ny (x nz) grid with Dirichlet boundary.
// Constant coefficients: (A w)_c = C w_c - sum of the in-grid neighbours,
// C = 4 (2D) / 6 (3D).  Variable coefficients: see pcg_matrix in pcg.h.
// MODE: how a row is evaluated (see StencilMode).
enum StencilMode { ST_LAP_FP64 = 0, ST_LAP_FIXED = 1, ST_VAR = 2 };

template <int DIM, int MODE, int VEC_>
struct StencilOp {
  static constexpr int VEC = VEC_;
  static constexpr bool VAR = MODE == ST_VAR;
  // the staged fused iteration (k_spcg_iter_tma) copies w's rows with 16-byte bulk copies
  static constexpr bool STAGED = MODE != ST_VAR && VEC == 2;
  static constexpr int DIMS = DIM;
  int n, nx, ny, nz, nxny;
  const double *diag, *ax, *ay, *az;

  __host__ __device__ int units() const { return n / VEC; }

#ifdef PCG_KERNELS_IMPL
  // Position of a unit: first unknown c0 and its grid coordinates.  The
  // grid-stride loops advance it by a fixed step with carries instead of
  // dividing by nx and ny for every unit.
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

  // wc[e] = w at the unit's own unknowns, aw[e] = (A w) there.
  __device__ __forceinline__ void apply(const double* __restrict__ w, const Cursor& q, double (&wc)[VEC],
                                        double (&aw)[VEC]) const {
    const unsigned c0 = q.c0, i0 = q.i0, j = q.j, k = q.k;
    const bool has_ym = j > 0, has_yp = j + 1 < (unsigned)ny;
    const bool has_zm = DIM == 3 && k > 0, has_zp = DIM == 3 && k + 1 < (unsigned)nz;
    double c[VEC], ym[VEC], yp[VEC], zm[VEC], zp[VEC];
    const unsigned un = (unsigned)n;
    const bool in = pcg_check(c0 + VEC <= un, CHK_STENCIL_CENTRE);
    ldg_if<VEC>(in, w + c0, c);
    ldg_if<VEC>(has_ym && pcg_check(in && c0 >= (unsigned)nx, CHK_STENCIL_Y), w + c0 - nx, ym);
    ldg_if<VEC>(has_yp && pcg_check(c0 + VEC + nx <= un, CHK_STENCIL_Y), w + c0 + nx, yp);
    if (DIM == 3) {
      ldg_if<VEC>(has_zm && pcg_check(in && c0 >= (unsigned)nxny, CHK_STENCIL_Z), w + c0 - nxny, zm);
      ldg_if<VEC>(has_zp && pcg_check(c0 + VEC + nxny <= un, CHK_STENCIL_Z), w + c0 + nxny, zp);
    }
    // x neighbours of the unit: left of the first, right of the last unknown
    const double xl = i0 > 0 && pcg_check(in && c0 >= 1, CHK_STENCIL_X) ? __ldg(w + c0 - 1) : 0.0;
    const double xr = i0 + VEC < (unsigned)nx && pcg_check(c0 + VEC < un, CHK_STENCIL_X) ? __ldg(w + c0 + VEC) : 0.0;
    row(q, c, xl, xr, ym, yp, zm, zp, wc, aw);
  }

  // The same row from staged copies of w in shared memory (constant coefficients):
  // `ctr` holds w from the unit's row minus nx (ctr[nx] = w[c0]), `zlo`/`zhi` w one
  // plane below/above (zlo[0] = w[c0 - nxny], zhi[0] = w[c0 + nxny]).  Neighbours outside
  // the grid read as 0, as in apply().
  __device__ __forceinline__ void apply_staged(const double* ctr, const double* zlo, const double* zhi,
                                               const Cursor& q, double (&wc)[VEC], double (&aw)[VEC]) const {
    const unsigned i0 = q.i0, j = q.j, k = q.k;
    const bool has_ym = j > 0, has_yp = j + 1 < (unsigned)ny;
    const bool has_zm = DIM == 3 && k > 0, has_zp = DIM == 3 && k + 1 < (unsigned)nz;
    double c[VEC], ym[VEC], yp[VEC], zm[VEC], zp[VEC];
    lds<VEC>(ctr + nx, c);
    lds_if<VEC>(has_ym, ctr, ym);
    lds_if<VEC>(has_yp, ctr + 2 * nx, yp);
    if (DIM == 3) {
      lds_if<VEC>(has_zm, zlo, zm);
      lds_if<VEC>(has_zp, zhi, zp);
    }
    const double xl = i0 > 0 ? ctr[nx - 1] : 0.0;
    const double xr = i0 + VEC < (unsigned)nx ? ctr[nx + VEC] : 0.0;
    row(q, c, xl, xr, ym, yp, zm, zp, wc, aw);
  }

  // (A w) at the unit from w there (c) and at its neighbours (0 outside the grid).
  __device__ __forceinline__ void row(const Cursor& q, const double (&c)[VEC], double xl, double xr,
                                      const double (&ym)[VEC], const double (&yp)[VEC], const double (&zm)[VEC],
                                      const double (&zp)[VEC], double (&wc)[VEC], double (&aw)[VEC]) const {
    double xm[VEC], xp[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      xm[e] = e == 0 ? xl : c[e - 1];
      xp[e] = e == VEC - 1 ? xr : c[e + 1];
      wc[e] = c[e];
    }
    if (MODE == ST_LAP_FIXED && !(DIM == 3 && VEC == 2)) {
      // integer-pipe fixed-point rows, full form (pcg_fixedsum.cuh): no FP64 instruction,
      // for any input; one row at a time, each unpacking its own terms
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        FxTerm t[DIM == 3 ? 7 : 5];
        t[0] = fx_centre_full<DIM>(c[e]);
        t[1] = fx_raw_full(xm[e], 1);
        t[2] = fx_raw_full(xp[e], 1);
        t[3] = fx_raw_full(ym[e], 1);
        t[4] = fx_raw_full(yp[e], 1);
        if constexpr (DIM == 3) {
          t[5] = fx_raw_full(zm[e], 1);
          t[6] = fx_raw_full(zp[e], 1);
        }
        aw[e] = fx_sum_full(t);
      }
    } else if (MODE == ST_LAP_FIXED) {
      // integer-pipe fixed-point rows, fast form (pcg_fixedsum.cuh); FP64 additions for a
      // unit with an Inf/NaN term or a row outside the normal range
      FxRaw rc[VEC], rym[VEC], ryp[VEC], rzm[VEC], rzp[VEC];
      const FxRaw rxl = fx_raw(xl), rxr = fx_raw(xr);
      int special = rxl.special | rxr.special;
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        rc[e] = fx_raw(c[e]);
        rym[e] = fx_raw(ym[e]);
        ryp[e] = fx_raw(yp[e]);
        special |= rc[e].special | rym[e].special | ryp[e].special;
        if (DIM == 3) {
          rzm[e] = fx_raw(zm[e]);
          rzp[e] = fx_raw(zp[e]);
          special |= rzm[e].special | rzp[e].special;
        }
      }
      bool ok = !special;
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        FxTerm t[DIM == 3 ? 7 : 5];
        t[0] = fx_centre<DIM>(rc[e]);
        t[1] = fx_minus(e == 0 ? rxl : rc[e - 1]);
        t[2] = fx_minus(e == VEC - 1 ? rxr : rc[e + 1]);
        t[3] = fx_minus(rym[e]);
        t[4] = fx_minus(ryp[e]);
        if constexpr (DIM == 3) {
          t[5] = fx_minus(rzm[e]);
          t[6] = fx_minus(rzp[e]);
        }
        aw[e] = fx_sum(t, ok);
      }
      if (!ok) {
        constexpr double C = DIM == 3 ? 6.0 : 4.0;
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
          double s = (xm[e] + xp[e]) + (ym[e] + yp[e]);
          if (DIM == 3) s += zm[e] + zp[e];
          aw[e] = fma(C, c[e], -s);
        }
      }
    } else if (MODE == ST_LAP_FP64) {
      constexpr double C = DIM == 3 ? 6.0 : 4.0;
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        double s = (xm[e] + xp[e]) + (ym[e] + yp[e]);
        if (DIM == 3) s += zm[e] + zp[e];
        aw[e] = fma(C, c[e], -s);
      }
    } else {
      const unsigned c0 = q.c0, i0 = q.i0, un = (unsigned)n;
      const bool has_yp = q.j + 1 < (unsigned)ny, has_zp = DIM == 3 && q.k + 1 < (unsigned)nz;
      const bool in = pcg_check(c0 + VEC <= un, CHK_COEFF);
      double d[VEC], fx[VEC], fy[VEC], fyp[VEC], fz[VEC], fzp[VEC];
      ldg_if<VEC>(in, diag + c0, d);
      ldg_if<VEC>(in, ax + c0, fx);
      ldg_if<VEC>(in, ay + c0, fy);
      ldg_if<VEC>(has_yp && pcg_check(c0 + VEC + nx <= un, CHK_COEFF), ay + c0 + nx, fyp);
      if (DIM == 3) {
        ldg_if<VEC>(in, az + c0, fz);
        ldg_if<VEC>(has_zp && pcg_check(c0 + VEC + nxny <= un, CHK_COEFF), az + c0 + nxny, fzp);
      }
      const double fxr = i0 + VEC < (unsigned)nx && pcg_check(c0 + VEC < un, CHK_COEFF) ? __ldg(ax + c0 + VEC) : 0.0;
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        const double fxp = e == VEC - 1 ? fxr : fx[e + 1];
        double a = d[e] * c[e];
        a = fma(-fx[e], xm[e], a);
        a = fma(-fxp, xp[e], a);
        a = fma(-fy[e], ym[e], a);
        a = fma(-fyp[e], yp[e], a);
        if (DIM == 3) {
          a = fma(-fz[e], zm[e], a);
          a = fma(-fzp[e], zp[e], a);
        }
        aw[e] = a;
      }
    }
  }

  template <int V>
  __device__ __forceinline__ static void lds(const double* p, double (&o)[V]) {
    if constexpr (V == 2) {
      const double2 t = *reinterpret_cast<const double2*>(p);
      o[0] = t.x;
      o[1] = t.y;
    } else {
      o[0] = *p;
    }
  }
  template <int V>
  __device__ __forceinline__ static void lds_if(bool ok, const double* p, double (&o)[V]) {
    if (ok) {
      lds<V>(p, o);
    } else {
#pragma unroll
      for (int e = 0; e < V; ++e) o[e] = 0.0;
    }
  }

  template <int V>
  __device__ __forceinline__ static void ldg(const double* p, double (&o)[V]) {
    if constexpr (V == 2) {
      const double2 t = __ldg(reinterpret_cast<const double2*>(p));
      o[0] = t.x;
      o[1] = t.y;
    } else {
      o[0] = __ldg(p);
    }
  }
  template <int V>
  __device__ __forceinline__ static void ldg_if(bool ok, const double* p, double (&o)[V]) {
    if (ok) {
      ldg<V>(p, o);
    } else {
#pragma unroll
      for (int e = 0; e < V; ++e) o[e] = 0.0;
    }
  }
#endif
};

// CSR matrix, one row per unit.
struct CsrOp {
  static constexpr int VEC = 1;
  static constexpr bool STAGED = false;
  int n;
  const int *row_ptr, *col;
  const double* val;

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

  __device__ __forceinline__ void apply(const double* __restrict__ w, const Cursor& q, double (&wc)[1],
                                        double (&aw)[1]) const {
    const int u = (int)q.c0;
    const bool in = pcg_check(u >= 0 && u < n, CHK_CSR_ROW);
    const int beg = in ? __ldg(row_ptr + u) : 0;
    int end = in ? __ldg(row_ptr + u + 1) : 0;
#ifdef PCG_CHECKED
    if (!pcg_check(beg >= 0 && beg <= end && end <= __ldg(row_ptr + n), CHK_CSR_ROW)) end = beg;
#endif
    double a = 0.0;
    for (int k = beg; k < end; ++k) {
      const int c = __ldg(col + k);
      if (pcg_check(c >= 0 && c < n, CHK_CSR_COL)) a = fma(__ldg(val + k), __ldg(w + c), a);
    }
    aw[0] = a;
    wc[0] = in ? __ldg(w + u) : 0.0;
  }
#endif
};

// ---------------------------------------------------------------- launch table

template <class Op>
struct Kernels {
  static cudaError_t residual(const Op& op, const Launch& L, const double* b, const double* x0, double* x,
                              double* r, State* st, double* partials);
  static cudaError_t spcg_w0(const Op& op, const Launch& L, Vecs v, State* st, Hist h, double* partials);
  static cudaError_t spcg_iter(const Op& op, const Launch& L, Vecs v, State* st, Hist h, double* partials,
                               bool ff_dots, int stages);
  static cudaError_t true_res(const Op& op, const Launch& L, Vecs v, State* st, Hist h, double* partials);
  static cudaError_t cg_p0(const Op& op, const Launch& L, Vecs v, State* st, Hist h, double* partials);
  static cudaError_t cg_spmv(const Op& op, const Launch& L, Vecs v, State* st, Hist h, double* partials);
  static cudaError_t cg_update(const Op& op, const Launch& L, Vecs v, State* st, Hist h, double* partials);
  static cudaError_t cg_p(const Op& op, const Launch& L, Vecs v, State* st, Hist h);
  static cudaError_t apply(const Op& op, const Launch& L, const double* x, double* y);
  static int blocks_per_sm(const Op& op, int kind, int stages);
  static int iter_stages(const Op& op, int stages);
};

#ifdef PCG_KERNELS_IMPL

// ---------------------------------------------------------------- vector access

template <int V>
__device__ __forceinline__ void ld_stream(const double* p, double (&o)[V]) {
  if constexpr (V == 2) {
    const double2 t = __ldcs(reinterpret_cast<const double2*>(p));
    o[0] = t.x;
    o[1] = t.y;
  } else {
    o[0] = __ldcs(p);
  }
}
template <int V>
__device__ __forceinline__ void st_stream(double* p, const double (&o)[V]) {
  if constexpr (V == 2) {
    __stcs(reinterpret_cast<double2*>(p), make_double2(o[0], o[1]));
  } else {
    __stcs(p, o[0]);
  }
}
template <int V>
__device__ __forceinline__ void st_plain(double* p, const double (&o)[V]) {
  if constexpr (V == 2) {
    *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
  } else {
    *p = o[0];
  }
}

// ---------------------------------------------------------------- reductions

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sums of NV values -> one partial per block; the last block to arrive
// (atomic ticket) sums all partials in block order and returns true with the
// totals in thread 0's `tot`.  Deterministic: the summation order depends only
// on the grid size.  No block waits for another.
template <int NV>
__device__ __forceinline__ bool reduce_last_block(double (&v)[NV], double* __restrict__ partials,
                                                  unsigned* ticket, double (&tot)[NV]) {
  __shared__ double sh[kWarps][NV];
  __shared__ int s_last;
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
      partials[blockIdx.x * NV + q] = a;
    }
    __threadfence();
    const unsigned t = atomicAdd(ticket, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  double a[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) a[q] = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += kBlock) {
#pragma unroll
    for (int q = 0; q < NV; ++q) a[q] += __ldcg(partials + b * NV + q);
  }
#pragma unroll
  for (int q = 0; q < NV; ++q) a[q] = warp_sum(a[q]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) sh[wid][q] = a[q];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double s = 0.0;
      for (int k = 0; k < kWarps; ++k) s += sh[k][q];
      tot[q] = s;
    }
  }
  return true;
}

// ---------------------------------------------------------------- finishers (one thread)

// Scalars of Algorithm 3 for iteration i from gamma_i = (r_i, r_i) and
// omega_i = (w_i, r_i); delta = (w_i + sigma r_i, r_i) = omega_i + sigma gamma_i.
// i = 0: beta_0 = 0, alpha_0 = gamma_0 / delta.  i > 0: beta_i = gamma_i / gamma_{i-1},
// alpha_i = 1 / (delta / gamma_i - beta_i / alpha_{i-1}).
// Stop tests in the oracle's order: tolerance, maxit, exact zero, breakdown.
__device__ __forceinline__ void finish_spcg(State* st, Hist h, double gamma, double omega, bool init) {
  const int i = init ? 0 : st->iter + 1;
  const double delta = omega + st->sigma * gamma;
  const double rn = sqrt(gamma);
  h.gamma[i] = gamma;
  h.delta[i] = delta;
  h.rec[i] = rn;
  int status = ST_RUNNING;
  if (st->tol_abs > 0.0 && rn <= st->tol_abs) {
    status = ST_CONVERGED;
  } else if (i >= st->maxit) {
    status = ST_MAXIT;
  } else if (gamma == 0.0) {
    status = ST_CONVERGED;
  } else if (init) {
    if (!(delta > 0.0) || !isfinite(delta)) {
      status = ST_BREAKDOWN;
    } else {
      h.alpha[0] = gamma / delta;
      h.beta[0] = 0.0;
    }
  } else {
    const double beta = gamma / h.gamma[i - 1];
    const double den = delta / gamma - beta / h.alpha[i - 1];
    if (!(den > 0.0) || !isfinite(den)) {
      status = ST_BREAKDOWN;
    } else {
      h.alpha[i] = 1.0 / den;
      h.beta[i] = beta;
    }
  }
  ff_scales(gamma, delta, st->sigma, st->ff_sr, st->ff_sw);
  st->iter = i;
  st->status = status;
  st->ticket = 0;
}

// Algorithm 1 after gamma_i = (r_i, u_i) and (r_i, r_i): stop tests, beta_i = gamma_i / gamma_{i-1}.
__device__ __forceinline__ void finish_cg_gamma(State* st, Hist h, double gamma, double rr, bool init) {
  const int i = init ? 0 : st->iter + 1;
  const double rn = sqrt(rr);
  h.gamma[i] = gamma;
  h.rec[i] = rn;
  int status = ST_RUNNING;
  if (st->tol_abs > 0.0 && rn <= st->tol_abs) {
    status = ST_CONVERGED;
  } else if (i >= st->maxit) {
    status = ST_MAXIT;
  } else if (gamma == 0.0) {
    status = ST_CONVERGED;
  } else {
    h.beta[i] = init ? 0.0 : gamma / h.gamma[i - 1];
  }
  st->iter = i;
  st->status = status;
  st->ticket = 0;
}

// ---------------------------------------------------------------- kernels

// r = b - A x0 (x0 given) or r = b, x = 0; ||b|| -> bnorm, tol_abs = tol_rel * ||b||.
template <class Op>
__global__ void __launch_bounds__(kBlock) k_residual(Op op, const double* __restrict__ b, int has_x0,
                                                     double* __restrict__ x, double* __restrict__ r, State* st,
                                                     double* partials) {
  constexpr int VEC = Op::VEC;
  double bb = 0.0;
  const unsigned nc = (unsigned)op.units() * VEC;
  const auto stp = op.step(gridDim.x * kBlock);
  for (auto q = op.cursor(blockIdx.x * kBlock + threadIdx.x); q.c0 < nc; op.advance(q, stp)) {
    const int c0 = (int)q.c0;
    double bv[VEC], rv[VEC];
    ld_stream<VEC>(b + c0, bv);
    if (has_x0) {
      double xc[VEC], ax[VEC];
      op.apply(x, q, xc, ax);
#pragma unroll
      for (int e = 0; e < VEC; ++e) rv[e] = bv[e] - ax[e];
    } else {
      double zero[VEC];
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        rv[e] = bv[e];
        zero[e] = 0.0;
      }
      st_plain<VEC>(x + c0, zero);
    }
    st_plain<VEC>(r + c0, rv);
#pragma unroll
    for (int e = 0; e < VEC; ++e) bb = fma(bv[e], bv[e], bb);
  }
  double v[1] = {bb}, tot[1];
  if (!reduce_last_block<1>(v, partials, &st->ticket, tot)) return;
  if (threadIdx.x == 0) {
    st->bnorm = sqrt(tot[0]);
    st->tol_abs = st->tol_abs * st->bnorm;   // tol_abs holds the relative tolerance until here
    st->ticket = 0;
  }
}

// Algorithm 3, line 1 (M = I): w_0 = A r_0 - sigma r_0; z, s, p := 0 (so that
// beta_0 z_{-1} etc. vanish); gamma_0, delta_0 -> alpha_0.
template <class Op>
__global__ void __launch_bounds__(kBlock) k_spcg_w0(Op op, Vecs v, State* st, Hist h, double* partials) {
  constexpr int VEC = Op::VEC;
  if (st->status != ST_RUNNING) return;
  const double sigma = st->sigma;
  double g = 0.0, o = 0.0;
  const unsigned nc = (unsigned)op.units() * VEC;
  const auto stp = op.step(gridDim.x * kBlock);
  for (auto q = op.cursor(blockIdx.x * kBlock + threadIdx.x); q.c0 < nc; op.advance(q, stp)) {
    const int c0 = (int)q.c0;
    double rc[VEC], ar[VEC], w[VEC], zero[VEC];
    op.apply(v.r, q, rc, ar);
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      w[e] = fma(-sigma, rc[e], ar[e]);
      zero[e] = 0.0;
      g = fma(rc[e], rc[e], g);
      o = fma(w[e], rc[e], o);
    }
    st_plain<VEC>(v.w0 + c0, w);
    st_plain<VEC>(v.z + c0, zero);
    st_plain<VEC>(v.s + c0, zero);
    st_plain<VEC>(v.p + c0, zero);
  }
  double vals[2] = {g, o}, tot[2];
  if (!reduce_last_block<2>(vals, partials, &st->ticket, tot)) return;
  if (threadIdx.x == 0) finish_spcg(st, h, tot[0], tot[1], true);
}

// One iteration of Algorithm 3 with M = I (u = r, q = s, t = p, m = w), fused:
//   n_i = A w_i;  z_i = n_i + beta_i z_{i-1};  s_i = w_i + beta_i s_{i-1};
//   p_i = r_i + beta_i p_{i-1};  x_{i+1} = x_i + alpha_i p_i;
//   r_{i+1} = r_i - alpha_i s_i - alpha_i sigma p_i  (two fused multiply-adds, the shift
//   term first);  w_{i+1} = w_i - alpha_i z_i;
// and, in the same sweep, the partials of gamma_{i+1} = (r_{i+1}, r_{i+1}) and
// (w_{i+1}, r_{i+1}); the last block turns them into alpha_{i+1}, beta_{i+1}.
// w is double-buffered (neighbours read w_i while w_{i+1} is written).
// FF: the two dots on the FP32 pipe (pcg_ffdot.cuh), else binary64 fused multiply-adds.

// Per-thread state of the sweep: the iteration's scalars and the dot accumulators.
struct SpcgSweep {
  double alpha, beta, asg;
  int sr, sw;
  double g = 0.0, o = 0.0;
  FfAcc G, O;
  unsigned bad = 0u;
};

// The recurrences of one unit from its loaded z, s, p, x, r, w_i and (A w_i); stores the
// updated vectors and accumulates the dots.
template <int VEC, bool FF>
__device__ __forceinline__ void spcg_unit(const Vecs& v, double* __restrict__ wn, int c0, SpcgSweep& S,
                                          const double (&wc)[VEC], const double (&nv)[VEC], double (&z)[VEC],
                                          double (&s)[VEC], double (&p)[VEC], double (&x)[VEC], double (&r)[VEC]) {
  double w1[VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) {
    z[e] = fma(S.beta, z[e], nv[e]);
    s[e] = fma(S.beta, s[e], wc[e]);
    p[e] = fma(S.beta, p[e], r[e]);
    x[e] = fma(S.alpha, p[e], x[e]);
    const double rn = fma(-S.alpha, s[e], fma(-S.asg, p[e], r[e]));
    const double wv = fma(-S.alpha, z[e], wc[e]);
    r[e] = rn;
    w1[e] = wv;
    if constexpr (FF) {
      const FfSplit fr = ff_split(rn, S.sr, S.bad), fw = ff_split(wv, S.sw, S.bad);
      ff_add_square(S.G, fr);
      ff_add_product(S.O, fw, fr);
    } else {
      S.g = fma(rn, rn, S.g);
      S.o = fma(wv, rn, S.o);
    }
  }
  st_stream<VEC>(v.z + c0, z);
  st_stream<VEC>(v.s + c0, s);
  st_stream<VEC>(v.p + c0, p);
  st_stream<VEC>(v.x + c0, x);
  st_stream<VEC>(v.r + c0, r);
  st_plain<VEC>(wn + c0, w1);
}

// One unit with its vectors loaded from global memory.
template <class Op, bool FF>
__device__ __forceinline__ void spcg_unit_global(const Op& op, const Vecs& v, const double* __restrict__ w,
                                                 double* __restrict__ wn, const typename Op::Cursor& q, SpcgSweep& S) {
  constexpr int VEC = Op::VEC;
  const int c0 = (int)q.c0;
  double wc[VEC], nv[VEC], z[VEC], s[VEC], p[VEC], x[VEC], r[VEC];
  op.apply(w, q, wc, nv);
  ld_stream<VEC>(v.z + c0, z);
  ld_stream<VEC>(v.s + c0, s);
  ld_stream<VEC>(v.p + c0, p);
  ld_stream<VEC>(v.x + c0, x);
  ld_stream<VEC>(v.r + c0, r);
  spcg_unit<VEC, FF>(v, wn, c0, S, wc, nv, z, s, p, x, r);
}

// The thread's dot partials, then the grid reduction and the finisher.  With FF and an
// out-of-range value, the thread's dots are summed again in binary64 from the r_{i+1}
// and w_{i+1} it has just written (its units are the grid-stride units from q0).
template <class Op, bool FF>
__device__ __forceinline__ void spcg_sweep_finish(const Op& op, const Vecs& v, const double* __restrict__ wn,
                                                  typename Op::Cursor q0, const typename Op::Step& stp, unsigned nc,
                                                  SpcgSweep& S, State* st, Hist h, double* partials) {
  constexpr int VEC = Op::VEC;
  if constexpr (FF) {
    if (S.bad) {
      for (auto q = q0; q.c0 < nc; op.advance(q, stp)) {
        const int c0 = (int)q.c0;
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
          const double rn = v.r[c0 + e], wv = wn[c0 + e];
          S.g = fma(rn, rn, S.g);
          S.o = fma(wv, rn, S.o);
        }
      }
    } else {
      S.g = ff_value(S.G, 2 * S.sr);
      S.o = ff_value(S.O, S.sr + S.sw);
    }
  }
  double vals[2] = {S.g, S.o}, tot[2];
  if (!reduce_last_block<2>(vals, partials, &st->ticket, tot)) return;
  if (threadIdx.x == 0) finish_spcg(st, h, tot[0], tot[1], false);
}

template <class Op, bool FF>
__global__ void __launch_bounds__(kBlock, PCG_ITER_MIN_BLOCKS) k_spcg_iter(Op op, Vecs v, State* st, Hist h, double* partials) {
  constexpr int VEC = Op::VEC;
  if (st->status != ST_RUNNING) return;
  const int it = st->iter;
  SpcgSweep S;
  S.alpha = h.alpha[it];
  S.beta = h.beta[it];
  S.asg = S.alpha * st->sigma;
  S.sr = st->ff_sr;
  S.sw = st->ff_sw;
  const double* __restrict__ w = (it & 1) ? v.w1 : v.w0;
  double* __restrict__ wn = (it & 1) ? v.w0 : v.w1;
  const unsigned nc = (unsigned)op.units() * VEC;
  const auto stp = op.step(gridDim.x * kBlock);
  const auto q0 = op.cursor(blockIdx.x * kBlock + threadIdx.x);
  for (auto q = q0; q.c0 < nc; op.advance(q, stp)) spcg_unit_global<Op, FF>(op, v, w, wn, q, S);
  spcg_sweep_finish<Op, FF>(op, v, wn, q0, stp, nc, S, st, h, partials);
}

// The same iteration with every operand of a chunk staged in shared memory by TMA bulk
// copies (constant-coefficient stencils with two unknowns per thread).  The sweep is cut
// into chunks of CH = kBlock * VEC consecutive unknowns, taken by the blocks in
// grid-stride order (chunk c by block c mod gridDim.x, so every thread owns the same
// units as in k_spcg_iter).  Per chunk, thread 0 copies into one stage of a ring of NST:
//   z, s, p, x, r over the chunk;  w_i over the chunk widened by one grid row on each
//   side (its x and y neighbours);  in 3D, w_i over the chunk one plane below and above.
// The copies of a chunk complete one phase of that stage's mbarrier; the ring keeps
// NST - 1 chunks in flight ahead of the one being computed, so no warp waits on a global
// load.  A chunk shorter than CH (n not a multiple of it) is computed from global memory.
// A wait that exceeds its time limit stops the solve with ST_TIMEOUT after the block has
// waited (again bounded) for its copies in flight.
// Measured (256^3 Laplacian, GB300): the staging removes the stalls on global loads
// (long-scoreboard stalls per issue 5.6 -> 0.6) and reads DRAM no more than the register
// sweep, but a ring of two 36 KB stages lets 3 blocks share an SM instead of 4, the FP64
// pipe is then less busy (71 % against 84 %), and the sweep takes 0.33 ms against 0.29 ms.
// It is therefore opt-in (PCG_PARAM_ITER_STAGES).
#ifndef PCG_TMA_MIN_BLOCKS
#define PCG_TMA_MIN_BLOCKS 3
#endif

// Doubles per stage: five chunk vectors, two plane rows (3D) and the widened w rows.
__host__ __device__ constexpr long long spcg_stage_doubles(int dim, int vec, long long nx) {
  return (5 + (dim == 3 ? 2 : 0)) * (long long)kBlock * vec + ((long long)kBlock * vec + 2 * nx);
}

template <class Op, bool FF, int NST>
__global__ void __launch_bounds__(kBlock, PCG_TMA_MIN_BLOCKS) k_spcg_iter_tma(Op op, Vecs v, State* st, Hist h,
                                                                                double* partials) {
  constexpr int VEC = Op::VEC;
  constexpr int DIM = Op::DIMS;
  constexpr int CH = kBlock * VEC;   // unknowns per chunk
  constexpr unsigned CHB = CH * sizeof(double);
  extern __shared__ __align__(128) double stage[];   // [NST][z s p x r | zlo zhi | ctr]
  // full[k]: the chunk's copies have landed; empty[k]: every warp is done reading it
  __shared__ unsigned long long full[NST], empty[NST];
  __shared__ volatile int s_fail;
  if (st->status != ST_RUNNING) return;
  const int it = st->iter;
  SpcgSweep S;
  S.alpha = h.alpha[it];
  S.beta = h.beta[it];
  S.asg = S.alpha * st->sigma;
  S.sr = st->ff_sr;
  S.sw = st->ff_sw;
  const double* __restrict__ w = (it & 1) ? v.w1 : v.w0;
  double* __restrict__ wn = (it & 1) ? v.w0 : v.w1;
  const unsigned nc = (unsigned)op.units() * VEC;
  const unsigned nfull = nc / CH;
  const unsigned G = gridDim.x;
  const unsigned nk = blockIdx.x < nfull ? (nfull - 1 - blockIdx.x) / G + 1 : 0u;   // staged chunks
  const long long nx = op.nx, nxny = op.nxny;
  const long long SS = spcg_stage_doubles(DIM, VEC, nx);
  const int ZLO = 5 * CH, ZHI = 6 * CH, CTR = (DIM == 3 ? 7 : 5) * CH;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NST; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], kWarps);
    }
    mbar_fence_init();
    s_fail = 0;
  }
  __syncthreads();
  const unsigned long long pol = l2_evict_first();
  auto issue = [&](unsigned k) {
    const unsigned sl = k % NST;
    const long long c0 = (long long)(blockIdx.x + k * G) * CH;
    double* dst = stage + sl * SS;
    // w rows: the chunk widened by one grid row, and (3D) the chunk one plane below/above,
    // each clipped to [0, n)
    const long long clo = c0 - nx > 0 ? c0 - nx : 0, chi = c0 + CH + nx < (long long)nc ? c0 + CH + nx : nc;
    unsigned tx = 5 * CHB + (unsigned)(chi - clo) * 8u;
    long long zlo_lo = 0, zlo_hi = 0, zhi_lo = 0, zhi_hi = 0;
    if (DIM == 3) {
      zlo_lo = c0 - nxny > 0 ? c0 - nxny : 0;
      zlo_hi = c0 - nxny + CH;
      zhi_lo = c0 + nxny;
      zhi_hi = c0 + nxny + CH < (long long)nc ? c0 + nxny + CH : nc;
      if (zlo_hi > zlo_lo) tx += (unsigned)(zlo_hi - zlo_lo) * 8u;
      if (zhi_hi > zhi_lo) tx += (unsigned)(zhi_hi - zhi_lo) * 8u;
    }
#ifdef PCG_CHECKED
    // every copy inside [0, n) with 16-byte sizes and addresses; a failing chunk is not
    // copied at all (its wait then runs out and the solve stops as timed out)
    auto ok16 = [](long long lo, long long hi) { return lo >= 0 && hi >= lo && ((hi - lo) & 1) == 0 && (lo & 1) == 0; };
    if (!pcg_check(c0 >= 0 && c0 + CH <= (long long)nc && ok16(clo, chi) && chi <= (long long)nc &&
                       (DIM != 3 || ((zlo_hi <= zlo_lo || ok16(zlo_lo, zlo_hi)) &&
                                     (zhi_hi <= zhi_lo || (ok16(zhi_lo, zhi_hi) && zhi_hi <= (long long)nc)))),
                   CHK_BULK_COPY))
      return;
#endif
    mbar_arrive_expect_tx(&full[sl], tx);
    bulk_g2s(dst + 0 * CH, v.z + c0, CHB, &full[sl], pol);
    bulk_g2s(dst + 1 * CH, v.s + c0, CHB, &full[sl], pol);
    bulk_g2s(dst + 2 * CH, v.p + c0, CHB, &full[sl], pol);
    bulk_g2s(dst + 3 * CH, v.x + c0, CHB, &full[sl], pol);
    bulk_g2s(dst + 4 * CH, v.r + c0, CHB, &full[sl], pol);
    // w's rows are copied three times (own rows, and the planes above/below of two other
    // chunks): no evict-first hint for them
    bulk_g2s(dst + CTR + (clo - (c0 - nx)), w + clo, (unsigned)(chi - clo) * 8u, &full[sl]);
    if (DIM == 3) {
      if (zlo_hi > zlo_lo)
        bulk_g2s(dst + ZLO + (zlo_lo - (c0 - nxny)), w + zlo_lo, (unsigned)(zlo_hi - zlo_lo) * 8u, &full[sl]);
      if (zhi_hi > zhi_lo) bulk_g2s(dst + ZHI, w + zhi_lo, (unsigned)(zhi_hi - zhi_lo) * 8u, &full[sl]);
    }
  };
  // bounded wait that also gives up once another thread of the block has given up
  auto wait = [&](unsigned long long* bar, unsigned parity) -> bool {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
      if (s_fail || global_ns() - t0 > kTmaWaitNs) {
        s_fail = 1;
        return false;
      }
    }
    return true;
  };
  unsigned issued = 0;   // chunks whose copies thread 0 has issued, in order
  if (threadIdx.x == 0) {
    for (; issued < nk && issued < (unsigned)NST; ++issued) issue(issued);
  }
  const auto stp = op.step(G * kBlock);
  const auto q0 = op.cursor(blockIdx.x * kBlock + threadIdx.x);
  const int tv = threadIdx.x * VEC;
  auto q = q0;
  unsigned k = 0;
  bool failed = false;
  for (; k < nk; ++k, op.advance(q, stp)) {
    const unsigned sl = k % NST;
    // warp-uniform outcome, so that a failing warp leaves the loop as a whole
    if (__any_sync(0xffffffffu, !wait(&full[sl], (k / NST) & 1u))) {
      failed = true;
      break;
    }
    const double* sb = stage + sl * SS;
    double wc[VEC], nv[VEC], z[VEC], s[VEC], p[VEC], x[VEC], r[VEC];
    op.apply_staged(sb + CTR + tv, sb + ZLO + tv, sb + ZHI + tv, q, wc, nv);
    ld_smem<VEC>(sb + 0 * CH + tv, z);
    ld_smem<VEC>(sb + 1 * CH + tv, s);
    ld_smem<VEC>(sb + 2 * CH + tv, p);
    ld_smem<VEC>(sb + 3 * CH + tv, x);
    ld_smem<VEC>(sb + 4 * CH + tv, r);
    // this warp is done with the stage's shared memory
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(&empty[sl]);
    // the producer refills the stage with chunk k + NST once every warp has left it
    if (threadIdx.x == 0 && k + NST < nk) {
      if (wait(&empty[sl], (k / NST) & 1u)) {
        issue(issued++);
      } else {
        failed = true;
      }
    }
    failed = __any_sync(0xffffffffu, failed);
    spcg_unit<VEC, FF>(v, wn, (int)q.c0, S, wc, nv, z, s, p, x, r);
    if (failed) break;
  }
  __syncthreads();
  if (s_fail) {
    // a wait exceeded its time limit: report, wait (bounded) for the copies this block
    // still has in flight, and leave without a partial (the solve stops as timed out)
    if (threadIdx.x == 0) {
      atomicExch(&st->status, ST_TIMEOUT);
      // the last chunk issued into each stage (chunks are issued in order, c into c mod NST)
      for (unsigned c = issued > (unsigned)NST ? issued - NST : 0u; c < issued; ++c)
        mbar_wait_bounded(&full[c % NST], (c / NST) & 1u);
    }
    return;
  }
  // the short last chunk, if this block owns it
  for (; q.c0 < nc; op.advance(q, stp)) spcg_unit_global<Op, FF>(op, v, w, wn, q, S);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NST; ++j) {
      mbar_inval(&full[j]);
      mbar_inval(&empty[j]);
    }
  }
  spcg_sweep_finish<Op, FF>(op, v, wn, q0, stp, nc, S, st, h, partials);
}

// True residual and gap at the current iterate: ||b - A x||, ||(b - A x) - r||
// (Section 3.1, the gap f_i), written at index st->iter.
template <class Op>
__global__ void __launch_bounds__(kBlock) k_true_res(Op op, Vecs v, State* st, Hist h, double* partials) {
  constexpr int VEC = Op::VEC;
  double t2 = 0.0, f2 = 0.0;
  const unsigned nc = (unsigned)op.units() * VEC;
  const auto stp = op.step(gridDim.x * kBlock);
  for (auto q = op.cursor(blockIdx.x * kBlock + threadIdx.x); q.c0 < nc; op.advance(q, stp)) {
    const int c0 = (int)q.c0;
    double xc[VEC], ax[VEC], bv[VEC], rv[VEC];
    op.apply(v.x, q, xc, ax);
    ld_stream<VEC>(v.b + c0, bv);
    ld_stream<VEC>(v.r + c0, rv);
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      const double t = bv[e] - ax[e];
      const double f = t - rv[e];
      t2 = fma(t, t, t2);
      f2 = fma(f, f, f2);
    }
  }
  double vals[2] = {t2, f2}, tot[2];
  if (!reduce_last_block<2>(vals, partials, &st->ticket, tot)) return;
  if (threadIdx.x == 0) {
    const int i = st->iter;
    const double tr = sqrt(tot[0]);
    h.tru[i] = tr;
    h.gap[i] = sqrt(tot[1]);
    // the true-residual stop (checked wherever the true residual is logged)
    if (st->status == ST_RUNNING && st->tol_true > 0.0 && tr <= st->tol_true * st->bnorm) st->status = ST_CONVERGED;
    st->ticket = 0;
  }
}

// u = M^{-1} r for Algorithm 1: D^{-1} r, or r itself for M = I (never stored).
template <int VEC>
__device__ __forceinline__ void cg_precond(const double* dinv, int c0, const double (&r)[VEC], double (&u)[VEC]) {
  if (dinv) {
    double d[VEC];
    ld_stream<VEC>(dinv + c0, d);
#pragma unroll
    for (int e = 0; e < VEC; ++e) u[e] = d[e] * r[e];
  } else {
#pragma unroll
    for (int e = 0; e < VEC; ++e) u[e] = r[e];
  }
}

// Algorithm 1, line 1: u_0 = M^{-1} r_0, p_0 = u_0, gamma_0 = (r_0, u_0), ||r_0||.
template <int VEC>
__global__ void __launch_bounds__(kBlock) k_cg_p0(int n, Vecs v, State* st, Hist h, double* partials) {
  if (st->status != ST_RUNNING) return;
  double g = 0.0, rr = 0.0;
  const int nu = n / VEC;
  for (int u = blockIdx.x * kBlock + threadIdx.x; u < nu; u += gridDim.x * kBlock) {
    const int c0 = u * VEC;
    double r[VEC], uu[VEC];
    ld_stream<VEC>(v.r + c0, r);
    cg_precond<VEC>(v.dinv, c0, r, uu);
    st_plain<VEC>(v.p + c0, uu);
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      g = fma(r[e], uu[e], g);
      rr = fma(r[e], r[e], rr);
    }
  }
  double vals[2] = {g, rr}, tot[2];
  if (!reduce_last_block<2>(vals, partials, &st->ticket, tot)) return;
  if (threadIdx.x == 0) finish_cg_gamma(st, h, tot[0], tot[1], true);
}

// Algorithm 1: s_i = A p_i and (s_i, p_i) -> alpha_i = gamma_i / (s_i, p_i).
template <class Op>
__global__ void __launch_bounds__(kBlock) k_cg_spmv(Op op, Vecs v, State* st, Hist h, double* partials) {
  constexpr int VEC = Op::VEC;
  if (st->status != ST_RUNNING) return;
  double sp = 0.0;
  const unsigned nc = (unsigned)op.units() * VEC;
  const auto stp = op.step(gridDim.x * kBlock);
  for (auto q = op.cursor(blockIdx.x * kBlock + threadIdx.x); q.c0 < nc; op.advance(q, stp)) {
    const int c0 = (int)q.c0;
    double pc[VEC], s[VEC];
    op.apply(v.p, q, pc, s);
    st_plain<VEC>(v.s + c0, s);
#pragma unroll
    for (int e = 0; e < VEC; ++e) sp = fma(s[e], pc[e], sp);
  }
  double vals[1] = {sp}, tot[1];
  if (!reduce_last_block<1>(vals, partials, &st->ticket, tot)) return;
  if (threadIdx.x == 0) {
    const int i = st->iter;
    if (!(tot[0] > 0.0) || !isfinite(tot[0])) {
      st->status = ST_BREAKDOWN;
    } else {
      h.alpha[i] = h.gamma[i] / tot[0];
    }
    st->ticket = 0;
  }
}

// Algorithm 1: x_{i+1} = x_i + alpha_i p_i, r_{i+1} = r_i - alpha_i s_i, gamma_{i+1}.
template <int VEC>
__global__ void __launch_bounds__(kBlock) k_cg_update(int n, Vecs v, State* st, Hist h, double* partials) {
  if (st->status != ST_RUNNING) return;
  const double alpha = h.alpha[st->iter];
  double g = 0.0, rr = 0.0;
  const int nu = n / VEC;
  for (int u = blockIdx.x * kBlock + threadIdx.x; u < nu; u += gridDim.x * kBlock) {
    const int c0 = u * VEC;
    double x[VEC], r[VEC], p[VEC], s[VEC];
    ld_stream<VEC>(v.x + c0, x);
    ld_stream<VEC>(v.r + c0, r);
    ld_stream<VEC>(v.p + c0, p);
    ld_stream<VEC>(v.s + c0, s);
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      x[e] = fma(alpha, p[e], x[e]);
      r[e] = fma(-alpha, s[e], r[e]);
    }
    double uu[VEC];
    cg_precond<VEC>(v.dinv, c0, r, uu);
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      g = fma(r[e], uu[e], g);
      rr = fma(r[e], r[e], rr);
    }
    st_stream<VEC>(v.x + c0, x);
    st_stream<VEC>(v.r + c0, r);
  }
  double vals[2] = {g, rr}, tot[2];
  if (!reduce_last_block<2>(vals, partials, &st->ticket, tot)) return;
  if (threadIdx.x == 0) finish_cg_gamma(st, h, tot[0], tot[1], false);
}

// Algorithm 1: p_{i+1} = u_{i+1} + beta_{i+1} p_i, u_{i+1} = M^{-1} r_{i+1}.
template <int VEC>
__global__ void __launch_bounds__(kBlock) k_cg_p(int n, Vecs v, State* st, Hist h) {
  if (st->status != ST_RUNNING) return;
  const double beta = h.beta[st->iter];
  const int nu = n / VEC;
  for (int u = blockIdx.x * kBlock + threadIdx.x; u < nu; u += gridDim.x * kBlock) {
    const int c0 = u * VEC;
    double r[VEC], uu[VEC], p[VEC];
    ld_stream<VEC>(v.r + c0, r);
    ld_stream<VEC>(v.p + c0, p);
    cg_precond<VEC>(v.dinv, c0, r, uu);
#pragma unroll
    for (int e = 0; e < VEC; ++e) p[e] = fma(beta, p[e], uu[e]);
    st_plain<VEC>(v.p + c0, p);
  }
}

// y = A x (the row evaluation the solver kernels use).
template <class Op>
__global__ void __launch_bounds__(kBlock) k_apply(Op op, const double* __restrict__ x, double* __restrict__ y) {
  constexpr int VEC = Op::VEC;
  const unsigned nc = (unsigned)op.units() * VEC;
  const auto stp = op.step(gridDim.x * kBlock);
  for (auto q = op.cursor(blockIdx.x * kBlock + threadIdx.x); q.c0 < nc; op.advance(q, stp)) {
    double xc[VEC], ax[VEC];
    op.apply(x, q, xc, ax);
    st_plain<VEC>(y + q.c0, ax);
  }
}

// ---------------------------------------------------------------- launchers

template <class Op>
cudaError_t Kernels<Op>::residual(const Op& op, const Launch& L, const double* b, const double* x0, double* x,
                                  double* r, State* st, double* partials) {
  k_residual<Op><<<L.grid, L.block, 0, L.stream>>>(op, b, x0 != nullptr, x, r, st, partials);
  return cudaGetLastError();
}
template <class Op>
cudaError_t Kernels<Op>::spcg_w0(const Op& op, const Launch& L, Vecs v, State* st, Hist h, double* partials) {
  k_spcg_w0<Op><<<L.grid, L.block, 0, L.stream>>>(op, v, st, h, partials);
  return cudaGetLastError();
}
template <class Op>
cudaError_t Kernels<Op>::spcg_iter(const Op& op, const Launch& L, Vecs v, State* st, Hist h, double* partials,
                                   bool ff_dots, int stages) {
  if constexpr (Op::STAGED) {
    if (stages == 2 || stages == 3) {
      const size_t sm = (size_t)stages * spcg_stage_doubles(Op::DIMS, Op::VEC, op.nx) * sizeof(double);
      if (stages == 2) {
        if (ff_dots) {
          k_spcg_iter_tma<Op, true, 2><<<L.grid, L.block, sm, L.stream>>>(op, v, st, h, partials);
        } else {
          k_spcg_iter_tma<Op, false, 2><<<L.grid, L.block, sm, L.stream>>>(op, v, st, h, partials);
        }
      } else {
        if (ff_dots) {
          k_spcg_iter_tma<Op, true, 3><<<L.grid, L.block, sm, L.stream>>>(op, v, st, h, partials);
        } else {
          k_spcg_iter_tma<Op, false, 3><<<L.grid, L.block, sm, L.stream>>>(op, v, st, h, partials);
        }
      }
      return cudaGetLastError();
    }
  }
  if (ff_dots) {
    k_spcg_iter<Op, true><<<L.grid, L.block, 0, L.stream>>>(op, v, st, h, partials);
  } else {
    k_spcg_iter<Op, false><<<L.grid, L.block, 0, L.stream>>>(op, v, st, h, partials);
  }
  return cudaGetLastError();
}

// Resident blocks per SM of the staged sweep (both dot forms; the smaller), after
// allowing the largest opt-in dynamic shared memory for it (the attribute is global to the
// kernel, and contexts with other row lengths launch it with other sizes).
template <class Op, int NST>
cudaError_t spcg_tma_occupancy(const Op& op, int* nb) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  const long long sm = (long long)NST * spcg_stage_doubles(Op::DIMS, Op::VEC, op.nx) * (long long)sizeof(double);
  *nb = 0;
  // the dynamic limit is what the opt-in maximum leaves beside the kernel's static shared memory
  cudaFuncAttributes fa, fb;
  if ((e = cudaFuncGetAttributes(&fa, k_spcg_iter_tma<Op, true, NST>)) != cudaSuccess) return e;
  if ((e = cudaFuncGetAttributes(&fb, k_spcg_iter_tma<Op, false, NST>)) != cudaSuccess) return e;
  const int dyn_a = optin - (int)fa.sharedSizeBytes, dyn_b = optin - (int)fb.sharedSizeBytes;
  if (sm > dyn_a || sm > dyn_b) return cudaSuccess;
  int a = 0, b = 0;
  if ((e = cudaFuncSetAttribute(k_spcg_iter_tma<Op, true, NST>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_a)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_spcg_iter_tma<Op, false, NST>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_b)) !=
      cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_spcg_iter_tma<Op, true, NST>, kBlock, (size_t)sm)) !=
      cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_spcg_iter_tma<Op, false, NST>, kBlock, (size_t)sm)) !=
      cudaSuccess)
    return e;
  *nb = min(a, b);
  return cudaSuccess;
}

// The staging depth the fused iteration will use: `stages` (2 or 3) when this operator
// can be staged and at least two staged blocks fit on an SM, else 0 (register sweep).
template <class Op>
int Kernels<Op>::iter_stages(const Op& op, int stages) {
  if constexpr (Op::STAGED) {
    if (stages != 2 && stages != 3) return 0;
    int nb = 0;
    const cudaError_t e = stages == 2 ? spcg_tma_occupancy<Op, 2>(op, &nb) : spcg_tma_occupancy<Op, 3>(op, &nb);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return nb >= 2 ? stages : 0;
  } else {
    (void)op;
    (void)stages;
    return 0;
  }
}

template <class Op>
cudaError_t Kernels<Op>::true_res(const Op& op, const Launch& L, Vecs v, State* st, Hist h, double* partials) {
  k_true_res<Op><<<L.grid, L.block, 0, L.stream>>>(op, v, st, h, partials);
  return cudaGetLastError();
}
template <class Op>
cudaError_t Kernels<Op>::cg_p0(const Op& op, const Launch& L, Vecs v, State* st, Hist h, double* partials) {
  k_cg_p0<Op::VEC><<<L.grid, L.block, 0, L.stream>>>(op.n, v, st, h, partials);
  return cudaGetLastError();
}
template <class Op>
cudaError_t Kernels<Op>::cg_spmv(const Op& op, const Launch& L, Vecs v, State* st, Hist h, double* partials) {
  k_cg_spmv<Op><<<L.grid, L.block, 0, L.stream>>>(op, v, st, h, partials);
  return cudaGetLastError();
}
template <class Op>
cudaError_t Kernels<Op>::cg_update(const Op& op, const Launch& L, Vecs v, State* st, Hist h, double* partials) {
  k_cg_update<Op::VEC><<<L.grid, L.block, 0, L.stream>>>(op.n, v, st, h, partials);
  return cudaGetLastError();
}
template <class Op>
cudaError_t Kernels<Op>::cg_p(const Op& op, const Launch& L, Vecs v, State* st, Hist h) {
  k_cg_p<Op::VEC><<<L.grid, L.block, 0, L.stream>>>(op.n, v, st, h);
  return cudaGetLastError();
}
template <class Op>
cudaError_t Kernels<Op>::apply(const Op& op, const Launch& L, const double* x, double* y) {
  k_apply<Op><<<L.grid, L.block, 0, L.stream>>>(op, x, y);
  return cudaGetLastError();
}
template <class Op>
int Kernels<Op>::blocks_per_sm(const Op& op, int kind, int stages) {
  int nb = 0;
  cudaError_t e = cudaSuccess;
  if constexpr (Op::STAGED) {
    if (kind == K_SPCG_ITER && (stages == 2 || stages == 3)) {
      e = stages == 2 ? spcg_tma_occupancy<Op, 2>(op, &nb) : spcg_tma_occupancy<Op, 3>(op, &nb);
      return e == cudaSuccess ? nb : 0;
    }
  }
  (void)op;
  switch (kind) {
    case K_RESIDUAL: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_residual<Op>, kBlock, 0); break;
    case K_SPCG_W0: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_spcg_w0<Op>, kBlock, 0); break;
    case K_SPCG_ITER: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_spcg_iter<Op, true>, kBlock, 0); break;
    case K_TRUE_RES: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_true_res<Op>, kBlock, 0); break;
    case K_CG_P0: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cg_p0<Op::VEC>, kBlock, 0); break;
    case K_CG_SPMV: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cg_spmv<Op>, kBlock, 0); break;
    case K_CG_UPDATE: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cg_update<Op::VEC>, kBlock, 0); break;
    case K_CG_P: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cg_p<Op::VEC>, kBlock, 0); break;
    case K_APPLY: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_apply<Op>, kBlock, 0); break;
    default: return 0;
  }
  return e == cudaSuccess ? nb : 0;
}

#endif  // PCG_KERNELS_IMPL

}  // namespace pcgk
