// One rank's share of a single system distributed over several GPUs: a z-slab of the
// 3D 7-point constant-coefficient Laplacian (the paper's setting, Section 1: the SpMV
// needs only neighbour communication, the dot products one global reduction).
//
// The rank holds planes [k0, k1) of the global grid; a neighbour's boundary plane of the
// vector being multiplied arrives in halo_lo (plane k0 - 1) or halo_hi (plane k1).  The
// iteration is split in the phases of pipelined CG so that the global reduction of
// (r, r), (w, r) overlaps the SpMV (Algorithm 3, lines of the reduction and of
// n_i := A m_i):
//   spmv    n = A w on the interior planes, then on the two boundary planes once the
//           halo has arrived;
//   scalars alpha_i, beta_i and the stop tests from the globally reduced dots (one thread);
//   update  the recurrences of z, s, p, x, r, w (w in place: n already holds A w_i) and
//           this rank's partial (r_{i+1}, r_{i+1}), (w_{i+1}, r_{i+1}).
// The communication itself (halo planes, the 2-scalar all-reduce) is the caller's; every
// phase here is one kernel on the slab's stream, with no host round trip.
#include <cuda_runtime.h>
#include <math.h>

#include <new>
#include <string>

#define PCG_KERNELS_IMPL
#include "../../include/pcg.h"
#include "pcg_kernels.cuh"

namespace pcgk {
namespace {

struct SlabGeom {
  int nx, ny, nzl;
  long long nxny;
  int has_lo, has_hi;   // neighbour slab below / above (else the Dirichlet boundary)
};

// dst = A src on planes [kb, ke) of the slab, the z neighbours of the first and last
// plane taken from the halo planes (or 0 at the global boundary).
template <int VEC>
__global__ void __launch_bounds__(kBlock) k_slab_spmv(SlabGeom g, const double* __restrict__ src,
                                                      const double* __restrict__ halo_lo,
                                                      const double* __restrict__ halo_hi, double* __restrict__ dst,
                                                      int kb, int ke) {
  using Op = StencilOp<3, ST_LAP_FIXED, VEC>;
  Op op;
  op.n = (int)(g.nxny * g.nzl);
  op.nx = g.nx;
  op.ny = g.ny;
  op.nz = g.nzl;
  op.nxny = (int)g.nxny;
  op.diag = op.ax = op.ay = op.az = nullptr;
  const unsigned beg = (unsigned)((long long)kb * g.nxny), end = (unsigned)((long long)ke * g.nxny);
  const auto stp = op.step(gridDim.x * kBlock);
  for (auto q = op.cursor((int)(beg / VEC) + blockIdx.x * kBlock + threadIdx.x); q.c0 < end; op.advance(q, stp)) {
    const unsigned c0 = q.c0, i0 = q.i0, j = q.j, k = q.k;
    double c[VEC], ym[VEC], yp[VEC], zm[VEC], zp[VEC];
    Op::template ldg<VEC>(src + c0, c);
    Op::template ldg_if<VEC>(j > 0, src + c0 - g.nx, ym);
    Op::template ldg_if<VEC>(j + 1 < (unsigned)g.ny, src + c0 + g.nx, yp);
    if (k > 0) {
      Op::template ldg<VEC>(src + c0 - g.nxny, zm);
    } else {
      Op::template ldg_if<VEC>(g.has_lo != 0 && pcg_check(c0 + VEC <= (unsigned)g.nxny, CHK_SLAB_HALO), halo_lo + c0,
                               zm);
    }
    if (k + 1 < (unsigned)g.nzl) {
      Op::template ldg<VEC>(src + c0 + g.nxny, zp);
    } else {
      const unsigned hc = c0 - (unsigned)((g.nzl - 1) * g.nxny);
      Op::template ldg_if<VEC>(g.has_hi != 0 && pcg_check(hc + VEC <= (unsigned)g.nxny, CHK_SLAB_HALO),
                               halo_hi + hc, zp);
    }
    const double xl = i0 > 0 ? __ldg(src + c0 - 1) : 0.0;
    const double xr = i0 + VEC < (unsigned)g.nx ? __ldg(src + c0 + VEC) : 0.0;
    double wc[VEC], aw[VEC];
    op.row(q, c, xl, xr, ym, yp, zm, zp, wc, aw);
    st_plain<VEC>(dst + c0, aw);
  }
}

struct SlabVecs {
  Vecs v;          // x, r, z, s, p, b; w0 = w (updated in place); w1 unused
  double* n;       // A w of the current iteration
};

// r = b, x = z = s = p = 0 (x_0 = 0); this rank's (b, b) -> dots[0].
template <int VEC>
__global__ void __launch_bounds__(kBlock) k_slab_start(int n, SlabVecs V, State* st, double* partials,
                                                       double* __restrict__ dots) {
  double bb = 0.0;
  const int nu = n / VEC;
  for (int u = blockIdx.x * kBlock + threadIdx.x; u < nu; u += gridDim.x * kBlock) {
    const int c0 = u * VEC;
    double bv[VEC], zero[VEC];
    ld_stream<VEC>(V.v.b + c0, bv);
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      zero[e] = 0.0;
      bb = fma(bv[e], bv[e], bb);
    }
    st_plain<VEC>(V.v.r + c0, bv);
    st_plain<VEC>(V.v.x + c0, zero);
    st_plain<VEC>(V.v.z + c0, zero);
    st_plain<VEC>(V.v.s + c0, zero);
    st_plain<VEC>(V.v.p + c0, zero);
  }
  double vals[1] = {bb}, tot[1];
  if (!reduce_last_block<1>(vals, partials, &st->ticket, tot)) return;
  if (threadIdx.x == 0) {
    dots[0] = tot[0];
    dots[1] = 0.0;
    st->ticket = 0;
  }
}

// ||b|| and the absolute tolerance from the globally reduced (b, b).
__global__ void k_slab_set_bnorm(State* st, const double* __restrict__ gdots) {
  st->bnorm = sqrt(gdots[0]);
  st->tol_abs = st->tol_abs * st->bnorm;   // tol_abs holds the relative tolerance until here
}

// w_0 = A r_0 - sigma r_0 (w holds A r_0); this rank's (r, r), (w_0, r) -> dots.
template <int VEC>
__global__ void __launch_bounds__(kBlock) k_slab_w0(int n, SlabVecs V, State* st, double* partials,
                                                    double* __restrict__ dots) {
  const double sigma = st->sigma;
  double g = 0.0, o = 0.0;
  const int nu = n / VEC;
  for (int u = blockIdx.x * kBlock + threadIdx.x; u < nu; u += gridDim.x * kBlock) {
    const int c0 = u * VEC;
    double r[VEC], w[VEC];
    ld_stream<VEC>(V.v.r + c0, r);
    ld_stream<VEC>(V.v.w0 + c0, w);
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      w[e] = fma(-sigma, r[e], w[e]);
      g = fma(r[e], r[e], g);
      o = fma(w[e], r[e], o);
    }
    st_plain<VEC>(V.v.w0 + c0, w);
  }
  double vals[2] = {g, o}, tot[2];
  if (!reduce_last_block<2>(vals, partials, &st->ticket, tot)) return;
  if (threadIdx.x == 0) {
    dots[0] = tot[0];
    dots[1] = tot[1];
    st->ticket = 0;
  }
}

// alpha_i, beta_i and the stop tests from the globally reduced gamma_i, omega_i.
__global__ void k_slab_scalars(State* st, Hist h, const double* __restrict__ gdots, int init) {
  if (st->status != ST_RUNNING) return;
  finish_spcg(st, h, gdots[0], gdots[1], init != 0);
}

// The recurrences of iteration i from n = A w_i, w updated in place; this rank's
// (r_{i+1}, r_{i+1}), (w_{i+1}, r_{i+1}) -> dots.
template <int VEC>
__global__ void __launch_bounds__(kBlock) k_slab_update(int n, SlabVecs V, State* st, Hist h, double* partials,
                                                        double* __restrict__ dots) {
  if (st->status != ST_RUNNING) return;
  const int it = st->iter;
  SpcgSweep S;
  S.alpha = h.alpha[it];
  S.beta = h.beta[it];
  S.asg = S.alpha * st->sigma;
  S.sr = S.sw = 0;
  const int nu = n / VEC;
  for (int u = blockIdx.x * kBlock + threadIdx.x; u < nu; u += gridDim.x * kBlock) {
    const int c0 = u * VEC;
    double wc[VEC], nv[VEC], z[VEC], s[VEC], p[VEC], x[VEC], r[VEC];
    ld_stream<VEC>(V.v.w0 + c0, wc);
    ld_stream<VEC>(V.n + c0, nv);
    ld_stream<VEC>(V.v.z + c0, z);
    ld_stream<VEC>(V.v.s + c0, s);
    ld_stream<VEC>(V.v.p + c0, p);
    ld_stream<VEC>(V.v.x + c0, x);
    ld_stream<VEC>(V.v.r + c0, r);
    spcg_unit<VEC, false>(V.v, V.v.w0, c0, S, wc, nv, z, s, p, x, r);
  }
  double vals[2] = {S.g, S.o}, tot[2];
  if (!reduce_last_block<2>(vals, partials, &st->ticket, tot)) return;
  if (threadIdx.x == 0) {
    dots[0] = tot[0];
    dots[1] = tot[1];
    st->ticket = 0;
  }
}

// After n = A x: this rank's ||b - A x||^2 and ||(b - A x) - r||^2 -> dots.
template <int VEC>
__global__ void __launch_bounds__(kBlock) k_slab_tres(int n, SlabVecs V, State* st, double* partials,
                                                      double* __restrict__ dots) {
  double t2 = 0.0, f2 = 0.0;
  const int nu = n / VEC;
  for (int u = blockIdx.x * kBlock + threadIdx.x; u < nu; u += gridDim.x * kBlock) {
    const int c0 = u * VEC;
    double bv[VEC], ax[VEC], rv[VEC];
    ld_stream<VEC>(V.v.b + c0, bv);
    ld_stream<VEC>(V.n + c0, ax);
    ld_stream<VEC>(V.v.r + c0, rv);
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
    dots[0] = tot[0];
    dots[1] = tot[1];
    st->ticket = 0;
  }
}

}  // namespace
}  // namespace pcgk

using namespace pcgk;

struct pcg_slab {
  SlabGeom g{};
  int n = 0, vec = 1, grid = 1, maxit = 0, device = 0;
  SlabVecs V{};
  const double *halo_lo = nullptr, *halo_hi = nullptr;
  State* st = nullptr;
  Hist h{};
  double* hist_mem = nullptr;
  double* partials = nullptr;
  cudaStream_t stream = nullptr;
  std::string err;
};

namespace {

pcg_status slab_cuda(pcg_slab* S, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return PCG_OK;
  cudaGetLastError();
  S->err = std::string(what) + ": " + cudaGetErrorString(e);
  return PCG_ECUDA;
}

const double* slab_vec(const pcg_slab* S, int which) {
  switch (which) {
    case PCG_SLAB_X: return S->V.v.x;
    case PCG_SLAB_R: return S->V.v.r;
    case PCG_SLAB_W: return S->V.v.w0;
    case PCG_SLAB_N: return S->V.n;
    default: return nullptr;
  }
}

}  // namespace

extern "C" {

pcg_status pcg_slab_create(int64_t nx, int64_t ny, int64_t nz_local, int32_t has_below, int32_t has_above,
                           const pcg_slab_vectors* v, int32_t maxit, pcg_slab** out) {
  if (!out) return PCG_EINVAL;
  *out = nullptr;
  if (!v || nx < 1 || ny < 1 || nz_local < 1 || maxit < 0 || nx > INT32_MAX || ny > INT32_MAX ||
      nz_local > INT32_MAX || nx * ny * nz_local > (int64_t)INT32_MAX - 64)
    return PCG_EINVAL;
  if (!v->x || !v->r || !v->w || !v->z || !v->s || !v->p || !v->n || !v->b) return PCG_EINVAL;
  if ((has_below && !v->halo_below) || (has_above && !v->halo_above)) return PCG_EINVAL;
  pcg_slab* S = new (std::nothrow) pcg_slab;
  if (!S) return PCG_ENOMEM;
  S->g.nx = (int)nx;
  S->g.ny = (int)ny;
  S->g.nzl = (int)nz_local;
  S->g.nxny = nx * ny;
  S->g.has_lo = has_below != 0;
  S->g.has_hi = has_above != 0;
  S->n = (int)(nx * ny * nz_local);
  const uintptr_t bits = (uintptr_t)v->x | (uintptr_t)v->r | (uintptr_t)v->w | (uintptr_t)v->z | (uintptr_t)v->s |
                         (uintptr_t)v->p | (uintptr_t)v->n | (uintptr_t)v->b |
                         (uintptr_t)(has_below ? v->halo_below : v->x) | (uintptr_t)(has_above ? v->halo_above : v->x);
  if (bits % 8 != 0) {
    delete S;
    return PCG_EINVAL;
  }
  S->vec = (nx % 2 == 0 && bits % 16 == 0) ? 2 : 1;
  S->maxit = maxit;
  S->V.v.x = v->x;
  S->V.v.r = v->r;
  S->V.v.w0 = S->V.v.w1 = v->w;
  S->V.v.z = v->z;
  S->V.v.s = v->s;
  S->V.v.p = v->p;
  S->V.v.b = v->b;
  S->V.n = v->n;
  S->halo_lo = v->halo_below;
  S->halo_hi = v->halo_above;
  auto fail = [&](pcg_status s) {
    pcg_slab_destroy(S);
    return s;
  };
  if (cudaGetDevice(&S->device) != cudaSuccess) return fail(slab_cuda(S, cudaGetLastError(), "cudaGetDevice"));
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, S->device) != cudaSuccess) return fail(PCG_ECUDA);
  const long long units = S->n / S->vec;
  long long gsz = (long long)sms * 4;
  if ((units + kBlock - 1) / kBlock < gsz) gsz = (units + kBlock - 1) / kBlock;
  S->grid = (int)(gsz < 1 ? 1 : gsz);
  if (cudaMalloc(&S->st, sizeof(State)) != cudaSuccess) return fail(PCG_ENOMEM);
  if (cudaMalloc(&S->partials, sizeof(double) * 2 * kMaxPartialBlocks) != cudaSuccess) return fail(PCG_ENOMEM);
  const size_t k = (size_t)maxit + 1;
  if (cudaMalloc(&S->hist_mem, sizeof(double) * 7 * k) != cudaSuccess) return fail(PCG_ENOMEM);
  S->h.alpha = S->hist_mem;
  S->h.beta = S->hist_mem + k;
  S->h.gamma = S->hist_mem + 2 * k;
  S->h.delta = S->hist_mem + 3 * k;
  S->h.rec = S->hist_mem + 4 * k;
  S->h.tru = S->hist_mem + 5 * k;
  S->h.gap = S->hist_mem + 6 * k;
  *out = S;
  return PCG_OK;
}

pcg_status pcg_slab_set_stream(pcg_slab* S, void* stream) {
  if (!S) return PCG_EINVAL;
  S->stream = (cudaStream_t)stream;
  return PCG_OK;
}

pcg_status pcg_slab_start(pcg_slab* S, double sigma, double tol, double* local_dots) {
  if (!S || !local_dots || !(sigma >= 0.0) || !(tol >= 0.0)) return PCG_EINVAL;
  State st{};
  st.iter = 0;
  st.status = ST_RUNNING;
  st.maxit = S->maxit;
  st.sigma = sigma;
  st.tol_abs = tol;   // relative until pcg_slab_set_bnorm
  pcg_status s = slab_cuda(S, cudaMemcpyAsync(S->st, &st, sizeof st, cudaMemcpyHostToDevice, S->stream), "state");
  if (s != PCG_OK) return s;
  // the copy reads the host State before this call returns
  if ((s = slab_cuda(S, cudaStreamSynchronize(S->stream), "state")) != PCG_OK) return s;
  const size_t k = (size_t)S->maxit + 1;
  if ((s = slab_cuda(S, cudaMemsetAsync(S->hist_mem, 0xFF, sizeof(double) * 7 * k, S->stream), "hist")) != PCG_OK)
    return s;
  if (S->vec == 2) {
    k_slab_start<2><<<S->grid, kBlock, 0, S->stream>>>(S->n, S->V, S->st, S->partials, local_dots);
  } else {
    k_slab_start<1><<<S->grid, kBlock, 0, S->stream>>>(S->n, S->V, S->st, S->partials, local_dots);
  }
  return slab_cuda(S, cudaGetLastError(), "k_slab_start");
}

pcg_status pcg_slab_set_bnorm(pcg_slab* S, const double* global_dots) {
  if (!S || !global_dots) return PCG_EINVAL;
  k_slab_set_bnorm<<<1, 1, 0, S->stream>>>(S->st, global_dots);
  return slab_cuda(S, cudaGetLastError(), "k_slab_set_bnorm");
}

pcg_status pcg_slab_spmv(pcg_slab* S, int32_t src, int32_t dst, int32_t planes) {
  if (!S) return PCG_EINVAL;
  const double* a = slab_vec(S, src);
  double* y = const_cast<double*>(slab_vec(S, dst));
  if (!a || !y || a == y || dst == PCG_SLAB_X || dst == PCG_SLAB_R) return PCG_EINVAL;
  const int nzl = S->g.nzl;
  auto run = [&](int kb, int ke) -> pcg_status {
    if (kb >= ke) return PCG_OK;
    const long long units = (long long)(ke - kb) * S->g.nxny / S->vec;
    long long gsz = (units + kBlock - 1) / kBlock;
    if (gsz > S->grid) gsz = S->grid;
    if (S->vec == 2) {
      k_slab_spmv<2><<<(int)gsz, kBlock, 0, S->stream>>>(S->g, a, S->halo_lo, S->halo_hi, y, kb, ke);
    } else {
      k_slab_spmv<1><<<(int)gsz, kBlock, 0, S->stream>>>(S->g, a, S->halo_lo, S->halo_hi, y, kb, ke);
    }
    return slab_cuda(S, cudaGetLastError(), "k_slab_spmv");
  };
  switch (planes) {
    case PCG_SLAB_ALL_PLANES: return run(0, nzl);
    case PCG_SLAB_INTERIOR_PLANES: return run(1, nzl - 1);
    case PCG_SLAB_BOUNDARY_PLANES: {
      const pcg_status s = run(0, 1);
      if (s != PCG_OK || nzl == 1) return s;
      return run(nzl - 1, nzl);
    }
    default: return PCG_EINVAL;
  }
}

pcg_status pcg_slab_w0(pcg_slab* S, double* local_dots) {
  if (!S || !local_dots) return PCG_EINVAL;
  if (S->vec == 2) {
    k_slab_w0<2><<<S->grid, kBlock, 0, S->stream>>>(S->n, S->V, S->st, S->partials, local_dots);
  } else {
    k_slab_w0<1><<<S->grid, kBlock, 0, S->stream>>>(S->n, S->V, S->st, S->partials, local_dots);
  }
  return slab_cuda(S, cudaGetLastError(), "k_slab_w0");
}

pcg_status pcg_slab_scalars(pcg_slab* S, const double* global_dots, int32_t first) {
  if (!S || !global_dots) return PCG_EINVAL;
  k_slab_scalars<<<1, 1, 0, S->stream>>>(S->st, S->h, global_dots, first != 0);
  return slab_cuda(S, cudaGetLastError(), "k_slab_scalars");
}

pcg_status pcg_slab_update(pcg_slab* S, double* local_dots) {
  if (!S || !local_dots) return PCG_EINVAL;
  if (S->vec == 2) {
    k_slab_update<2><<<S->grid, kBlock, 0, S->stream>>>(S->n, S->V, S->st, S->h, S->partials, local_dots);
  } else {
    k_slab_update<1><<<S->grid, kBlock, 0, S->stream>>>(S->n, S->V, S->st, S->h, S->partials, local_dots);
  }
  return slab_cuda(S, cudaGetLastError(), "k_slab_update");
}

pcg_status pcg_slab_true_residual(pcg_slab* S, double* local_sums) {
  if (!S || !local_sums) return PCG_EINVAL;
  if (S->vec == 2) {
    k_slab_tres<2><<<S->grid, kBlock, 0, S->stream>>>(S->n, S->V, S->st, S->partials, local_sums);
  } else {
    k_slab_tres<1><<<S->grid, kBlock, 0, S->stream>>>(S->n, S->V, S->st, S->partials, local_sums);
  }
  return slab_cuda(S, cudaGetLastError(), "k_slab_tres");
}

pcg_status pcg_slab_state(pcg_slab* S, int32_t* iter, int32_t* status, double* bnorm) {
  if (!S) return PCG_EINVAL;
  State st{};
  pcg_status s = slab_cuda(S, cudaMemcpyAsync(&st, S->st, sizeof st, cudaMemcpyDeviceToHost, S->stream), "state");
  if (s == PCG_OK) s = slab_cuda(S, cudaStreamSynchronize(S->stream), "state");
  if (s != PCG_OK) return s;
  if (iter) *iter = st.iter;
  if (status) {
    *status = st.status == ST_RUNNING ? PCG_PENDING : st.status == ST_CONVERGED ? PCG_OK
              : st.status == ST_BREAKDOWN ? PCG_EBREAKDOWN : PCG_ENOTCONV;
  }
  if (bnorm) *bnorm = st.bnorm;
  return PCG_OK;
}

pcg_status pcg_slab_history(pcg_slab* S, int32_t k, double* alpha, double* beta, double* rec) {
  if (!S || k < 0 || k > S->maxit + 1) return PCG_EINVAL;
  pcg_status s = PCG_OK;
  if (alpha && s == PCG_OK)
    s = slab_cuda(S, cudaMemcpyAsync(alpha, S->h.alpha, sizeof(double) * k, cudaMemcpyDeviceToHost, S->stream), "h");
  if (beta && s == PCG_OK)
    s = slab_cuda(S, cudaMemcpyAsync(beta, S->h.beta, sizeof(double) * k, cudaMemcpyDeviceToHost, S->stream), "h");
  if (rec && s == PCG_OK)
    s = slab_cuda(S, cudaMemcpyAsync(rec, S->h.rec, sizeof(double) * k, cudaMemcpyDeviceToHost, S->stream), "h");
  if (s == PCG_OK) s = slab_cuda(S, cudaStreamSynchronize(S->stream), "history");
  return s;
}

const char* pcg_slab_last_error(const pcg_slab* S) { return S ? S->err.c_str() : "null slab"; }

void pcg_slab_destroy(pcg_slab* S) {
  if (!S) return;
  if (S->stream) cudaStreamSynchronize(S->stream);
  cudaFree(S->st);
  cudaFree(S->partials);
  cudaFree(S->hist_mem);
  delete S;
}

}  // extern "C"
