// Per-cluster solves beyond the binary64, M = I case of pcg_cluster_solve.cuh, shared by
// the batched launch and the serving kernel:
//   cluster_solve_jac<F>      Algorithm 3 with M^{-1} = D^{-1}, binary64
//   cluster_solve_mx<F, JAC>  mixed precision with restarts (iterative refinement),
//                             M = I or M^{-1} = D^{-1}
// The arithmetic per unknown follows the single-system kernels (pcg_general.cuh,
// pcg_mixed.cuh, pcg_mixed_jacobi.cuh); the reductions are the cluster's (cluster_sum).
#pragma once
#include "pcg_cluster_solve.cuh"
#include "pcg_mixed.cuh"

namespace pcgk {

// Default inner tolerance factor eta of the per-cluster mixed-precision solves (batch and
// serving): a restart comes once the recursive residual has fallen by eta.  2^-14 (the
// single-system solver uses 2^-10): on 512 high-contrast 2D systems solved to 1e-8 with
// Jacobi, 2^-10 / 2^-12 / 2^-14 / 2^-16 took 3,215 / 3,022 / 2,978 / 2,982 iterations on
// average, since fewer restarts leave the Krylov space fewer times.
#ifndef PCG_CLUSTER_MIXED_ETA_LOG2
#define PCG_CLUSTER_MIXED_ETA_LOG2 14
#endif
constexpr double kClusterMixedEta = 1.0 / (double)(1ll << PCG_CLUSTER_MIXED_ETA_LOG2);

// The binary32 operator with V unknowns per thread (stencils; CSR rows stay one per thread).
template <int F, int V>
struct FamilyOp32V {
  using T = StencilOp32<(F >= 2 ? 3 : 2), (F == 1 || F == 3), V>;
};
template <int V>
struct FamilyOp32V<4, V> {
  using T = CsrOp32;
};

template <int F, int V = 1>
__device__ __forceinline__ typename FamilyOp32V<F, V>::T make_op32(const BatchSys& d) {
  typename FamilyOp32V<F, V>::T o;
  if constexpr (F == 4) {
    o.n = d.n;
    o.row_ptr = d.row_ptr;
    o.col = d.col;
    o.val = d.val32;
  } else {
    o.n = d.n;
    o.nx = d.nx;
    o.ny = d.ny;
    o.nz = d.nz;
    o.nxny = d.nx * d.ny;
    o.diag = d.diag32;
    o.ax = d.ax32;
    o.ay = d.ay32;
    o.az = d.az32;
  }
  return o;
}

// ||b - A x|| in binary64 over the cluster.
template <int F>
__device__ __forceinline__ double cluster_true_res(cg::cluster_group& cl, double (*part)[4], int& slot,
                                                   const typename FamilyOp<F>::T& op, const double* b,
                                                   const double* x, unsigned nc, int first,
                                                   const typename FamilyOp<F>::T::Step& stp) {
  double tr = 0.0;
  for (auto q = op.cursor(first); q.c0 < nc; op.advance(q, stp)) {
    double xc[1], ax[1];
    op.apply(x, q, xc, ax);
    const double e = b[q.c0] - ax[0];
    tr = fma(e, e, tr);
  }
  double t[1] = {tr}, o[1];
  cluster_sum<1>(cl, t, part, slot, o);
  slot ^= 1;
  return sqrt(o[0]);
}

// Algorithm 3 with M^{-1} = D^{-1} (binary64, x_0 = 0) for one system on the calling cluster.
template <int F>
__device__ __forceinline__ void cluster_solve_jac(cg::cluster_group& cl, double (*part)[4], int& slot,
                                                  const BatchSys& d, const BatchVecs& V, double tol, int maxit,
                                                  BatchOut& res) {
  using Op = typename FamilyOp<F>::T;
  const unsigned rank = cl.block_rank(), C = cl.num_blocks();
  const Op op = make_op<F>(d);
  const double sigma = d.sigma;
  // vector k at b + k * stride (see cluster_solve_mx); addresses formed where used
  double* const vb = const_cast<double*>(V.b) + d.off;
  long long stride = V.stride;
  auto dv = [&](int k) { return vb + (long long)k * stride; };
  const double* b = vb;
  const unsigned nc = (unsigned)d.n;
  const auto stp = op.step(C * kBlock);
  const int first = (int)(rank * kBlock + threadIdx.x);

  scalar_log_clear(d, rank);
  // r_0 = b (x_0 = 0), u_0 = D^{-1} r_0, ||b||
  double bb = 0.0;
  for (unsigned i = first; i < nc; i += C * kBlock) {
    const double bv = b[i];
    dv(2)[i] = bv;
    dv(8)[i] = dv(14)[i] * bv;
    dv(1)[i] = 0.0;
    bb = fma(bv, bv, bb);
  }
  double t1[1] = {bb}, o1[1];
  cluster_sum<1>(cl, t1, part, slot, o1);
  slot ^= 1;
  const double bnorm = sqrt(o1[0]);
  const double tol_abs = tol * bnorm;

  // w_0 = A u_0 - sigma r_0, m_0 = D^{-1} w_0; z = q = s = t = p = 0
  double ru = 0.0, wu = 0.0, rr = 0.0;
  for (auto q = op.cursor(first); q.c0 < nc; op.advance(q, stp)) {
    asm volatile("" : "+l"(stride));
    const unsigned c = q.c0;
    double uc[1], au[1];
    op.apply(dv(8), q, uc, au);
    const double rc = dv(2)[c];
    const double wv = fma(-sigma, rc, au[0]);
    dv(3)[c] = wv;
    dv(11)[c] = dv(14)[c] * wv;
    dv(5)[c] = 0.0;
    dv(9)[c] = 0.0;
    dv(6)[c] = 0.0;
    dv(10)[c] = 0.0;
    dv(7)[c] = 0.0;
    ru = fma(rc, uc[0], ru);
    wu = fma(wv, uc[0], wu);
    rr = fma(rc, rc, rr);
  }
  double t2[3] = {ru, wu, rr}, o2[3];
  cluster_sum<3>(cl, t2, part, slot, o2);
  slot ^= 1;
  double gamma = o2[0], delta = o2[1] + sigma * o2[0];
  int status = ST_RUNNING, it = 0;
  double alpha = 0.0, beta = 0.0;
  if (tol_abs > 0.0 && sqrt(o2[2]) <= tol_abs) {
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
    const int odd = it & 1;
    ru = wu = rr = 0.0;
    for (auto q = op.cursor(first); q.c0 < nc; op.advance(q, stp)) {
      asm volatile("" : "+l"(stride));
      const double* __restrict__ w = dv(odd ? 4 : 3);
      double* __restrict__ wn = dv(odd ? 3 : 4);
      const double* __restrict__ m = dv(odd ? 12 : 11);
      double* __restrict__ mn = dv(odd ? 11 : 12);
      double* __restrict__ x = dv(1);
      double* __restrict__ r = dv(2);
      double* __restrict__ z = dv(5);
      double* __restrict__ s = dv(6);
      double* __restrict__ p = dv(7);
      double* __restrict__ u = dv(8);
      double* __restrict__ qv = dv(9);
      double* __restrict__ t = dv(10);
      const double* __restrict__ dinv = dv(14);
      const unsigned c = q.c0;
      double mc[1], nv[1];
      op.apply(m, q, mc, nv);
      const double wc = w[c], rc = r[c], uc = u[c];
      const double tt = fma(beta, t[c], rc);
      const double ss = fma(beta, s[c], wc);
      const double zz = fma(beta, z[c], nv[0]);
      const double rn = fma(-alpha, ss, fma(-asg, tt, rc));
      const double wv = fma(-alpha, zz, wc);
      const double pp = fma(beta, p[c], uc);
      const double qq = fma(beta, qv[c], mc[0]);
      x[c] = fma(alpha, pp, x[c]);
      const double un = fma(-alpha, qq, fma(-asg, pp, uc));
      t[c] = tt;
      s[c] = ss;
      z[c] = zz;
      p[c] = pp;
      qv[c] = qq;
      r[c] = rn;
      u[c] = un;
      wn[c] = wv;
      mn[c] = dinv[c] * wv;
      ru = fma(rn, un, ru);
      wu = fma(wv, un, wu);
      rr = fma(rn, rn, rr);
    }
    double tv[3] = {ru, wu, rr}, to[3];
    cluster_sum<3>(cl, tv, part, slot, to);
    slot ^= 1;
    ++it;
    const double gn = to[0], dn = to[1] + sigma * to[0];
    if (tol_abs > 0.0 && sqrt(to[2]) <= tol_abs) {
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
  res.iters = it;
  res.status = status;
  res.bnorm = bnorm;
  res.true_res = cluster_true_res<F>(cl, part, slot, op, b, dv(1), nc, first, stp);
}

// Mixed precision with restarts (M = I, or M^{-1} = D^{-1} when JAC), x_0 = 0.
// Storage as in the single-system kernels: x, r binary64; the auxiliary vectors binary32
// (M = I: w, z, s, p; JAC: u, w, m, z, q, s, t, p).  A restart recomputes r = b - A x in
// binary64 and restarts Algorithm 3 from x once the inner residual ||r_i|| reaches
// max(eta * true residual, tol ||b|| / 2); the solve ends when the true residual reaches
// tol ||b||, when a restart does not lower it (reported as maxit), or at maxit.
// VW: unknowns per thread in the binary32 sweeps (1, 2 or 4; a stencil's nx must be a multiple).
template <int F, bool JAC, int VW = 1>
__device__ __forceinline__ void cluster_solve_mx(cg::cluster_group& cl, double (*part)[4], int& slot,
                                                 const BatchSys& d, const BatchVecs& V, double tol, int maxit,
                                                 double eta, int max_restarts, BatchOut& res) {
  using Op = typename FamilyOp<F>::T;
  using Op32 = typename FamilyOp32V<F, VW>::T;
  const unsigned rank = cl.block_rank(), C = cl.num_blocks();
  const Op op = make_op<F>(d);
  const Op32 op32 = make_op32<F, VW>(d);
  const double sigma = d.sigma;
  // Every vector of the layout lies at b + k * stride (k: b 0, x 1, r 2, w0 3, w1 4, z 5, s 6,
  // p 7, u 8, q 9, t 10, m0 11, m1 12, u64 13, dinv 14, dinv32 15).  The addresses are formed
  // from that base and stride where they are used: `stride` is re-declared opaque at the top
  // of every sweep (an empty asm), so no per-vector address stays live across the solve and
  // the registers go to the unknowns in flight instead.
  double* const vb = const_cast<double*>(V.b) + d.off;
  long long stride = V.stride;
  auto dv = [&](int k) { return vb + (long long)k * stride; };
  auto fv = [&](int k) { return reinterpret_cast<float*>(vb + (long long)k * stride); };
  const double* b = vb;
  const unsigned nc = (unsigned)d.n;
  const auto stp = op.step(C * kBlock);
  const auto stp32 = op32.step(C * kBlock);
  const int first = (int)(rank * kBlock + threadIdx.x);

  scalar_log_clear(d, rank);
  double bb = 0.0;
  double* const x0 = dv(1);
  for (unsigned i = first; i < nc; i += C * kBlock) {
    const double bv = b[i];
    x0[i] = 0.0;
    bb = fma(bv, bv, bb);
  }
  double t1[1] = {bb}, o1[1];
  cluster_sum<1>(cl, t1, part, slot, o1);
  slot ^= 1;
  const double bnorm = sqrt(o1[0]);
  const double tol_abs = tol * bnorm;
  int status = ST_RUNNING, it = 0, restarts = 0, par = 0;
  double rprev = INFINITY, true_res = 0.0;
  for (;;) {
    // restart, part 1: r = b - A x (binary64); JAC: u = D^{-1} r rounded to binary32
    double rr = 0.0;
    for (auto q = op.cursor(first); q.c0 < nc; op.advance(q, stp)) {
      asm volatile("" : "+l"(stride));
      const unsigned c = q.c0;
      double xc[1], ax[1];
      op.apply(dv(1), q, xc, ax);
      const double rv = b[c] - ax[0];
      dv(2)[c] = rv;
      rr = fma(rv, rv, rr);
      if constexpr (JAC) {
        const float u32 = f32_of(dv(14)[c] * rv);
        fv(8)[c] = u32;
        dv(13)[c] = f64_of(u32);
      }
    }
    double t2[1] = {rr}, o2[1];
    cluster_sum<1>(cl, t2, part, slot, o2);
    slot ^= 1;
    const double rt = sqrt(o2[0]);
    true_res = rt;
    if (rt <= tol_abs || o2[0] == 0.0) {
      status = ST_CONVERGED;
      break;
    }
    if ((restarts > 0 && !(rt < rprev)) || restarts >= max_restarts || it >= maxit) {
      status = ST_MAXIT;
      break;
    }
    const double inner = fmax(eta * rt, 0.5 * tol_abs);
    rprev = rt;
    ++restarts;
    // restart, part 2: w_0 = A u_0 - sigma r (binary64 operator), auxiliary vectors zero
    double g = 0.0, o = 0.0, rr0 = 0.0;
    for (auto q = op.cursor(first); q.c0 < nc; op.advance(q, stp)) {
      asm volatile("" : "+l"(stride));
      const unsigned c = q.c0;
      double uc[1], au[1];
      op.apply(dv(JAC ? 13 : 2), q, uc, au);
      const double rv = dv(2)[c];
      const float w32 = f32_of(fma(-sigma, rv, au[0]));
      fv(par ? 4 : 3)[c] = w32;
      fv(5)[c] = 0.f;
      fv(6)[c] = 0.f;
      fv(7)[c] = 0.f;
      if constexpr (JAC) {
        fv(par ? 12 : 11)[c] = fv(15)[c] * w32;
        fv(9)[c] = 0.f;
        fv(10)[c] = 0.f;
      }
      g = fma(rv, uc[0], g);
      o = fma(f64_of(w32), uc[0], o);
      rr0 = fma(rv, rv, rr0);
    }
    double t3[3] = {g, o, rr0}, o3[3];
    cluster_sum<3>(cl, t3, part, slot, o3);
    slot ^= 1;
    double gamma = o3[0], delta = o3[1] + sigma * o3[0];
    if (!(delta > 0.0) || !isfinite(delta)) {
      status = ST_BREAKDOWN;
      break;
    }
    double alpha = gamma / delta, beta = 0.0;
    scalar_log(d, rank, it, alpha, beta);
    // inner iterations
    for (;;) {
      const double asg = alpha * sigma;
      const float alpha32 = f32_of(alpha), beta32 = f32_of(beta), asg32 = f32_of(asg);
      double ru = 0.0, wu = 0.0, rn2 = 0.0;
      for (auto q = op32.cursor(first); q.c0 < nc; op32.advance(q, stp32)) {
        asm volatile("" : "+l"(stride));
        const float* __restrict__ w = fv(par ? 4 : 3);
        float* __restrict__ wn = fv(par ? 3 : 4);
        const float* __restrict__ m = fv(par ? 12 : 11);
        float* __restrict__ mn = fv(par ? 11 : 12);
        float* __restrict__ zf = fv(5);
        float* __restrict__ sf = fv(6);
        float* __restrict__ pf = fv(7);
        float* __restrict__ uf = fv(8);
        float* __restrict__ qf = fv(9);
        float* __restrict__ tf = fv(10);
        const float* __restrict__ d32 = fv(15);
        double* __restrict__ r = dv(2);
        double* __restrict__ x = dv(1);
        const unsigned c = q.c0;
        float mc[VW], nv[VW], wc[VW], zz[VW], ss[VW], pp[VW], w1[VW];
        double rc[VW], xv[VW];
        op32.apply(JAC ? m : w, q, mc, nv);
        if constexpr (JAC) {
          ldf<VW>(w + c, wc);
        } else {
#pragma unroll
          for (int e = 0; e < VW; ++e) wc[e] = mc[e];
        }
        ldf<VW>(zf + c, zz);
        ldf<VW>(sf + c, ss);
        ldf<VW>(pf + c, pp);
        ldd<VW>(r + c, rc);
        ldd<VW>(x + c, xv);
        float uu[VW], tt[VW], qq[VW], dd[VW], m1[VW];
        if constexpr (JAC) {
          ldf<VW>(uf + c, uu);
          ldf<VW>(tf + c, tt);
          ldf<VW>(qf + c, qq);
          ldf<VW>(d32 + c, dd);
        }
#pragma unroll
        for (int e = 0; e < VW; ++e) {
          zz[e] = fmaf(beta32, zz[e], nv[e]);
          ss[e] = fmaf(beta32, ss[e], wc[e]);
          w1[e] = fmaf(-alpha32, zz[e], wc[e]);
          if constexpr (JAC) {
            tt[e] = fmaf(beta32, tt[e], f32_of(rc[e]));
            pp[e] = fmaf(beta32, pp[e], uu[e]);
            qq[e] = fmaf(beta32, qq[e], mc[e]);
            xv[e] = fma(alpha, f64_of(pp[e]), xv[e]);
            const double rn = fma(-alpha, f64_of(ss[e]), fma(-asg, f64_of(tt[e]), rc[e]));
            uu[e] = fmaf(-alpha32, qq[e], fmaf(-asg32, pp[e], uu[e]));
            rc[e] = rn;
            m1[e] = dd[e] * w1[e];
            const double ud = f64_of(uu[e]);
            ru = fma(rn, ud, ru);
            wu = fma(f64_of(w1[e]), ud, wu);
            rn2 = fma(rn, rn, rn2);
          } else {
            pp[e] = fmaf(beta32, pp[e], f32_of(rc[e]));
            const double pd = f64_of(pp[e]);
            xv[e] = fma(alpha, pd, xv[e]);
            const double rn = fma(-alpha, f64_of(ss[e]), fma(-asg, pd, rc[e]));
            rc[e] = rn;
            ru = fma(rn, rn, ru);
            wu = fma(f64_of(w1[e]), rn, wu);
          }
        }
        stf<VW>(zf + c, zz);
        stf<VW>(sf + c, ss);
        stf<VW>(pf + c, pp);
        std_<VW>(r + c, rc);
        std_<VW>(x + c, xv);
        stf<VW>(wn + c, w1, false);
        if constexpr (JAC) {
          stf<VW>(uf + c, uu);
          stf<VW>(tf + c, tt);
          stf<VW>(qf + c, qq);
          stf<VW>(mn + c, m1, false);
        }
      }
      if constexpr (!JAC) rn2 = ru;
      double t4[3] = {ru, wu, rn2}, o4[3];
      cluster_sum<3>(cl, t4, part, slot, o4);
      slot ^= 1;
      ++it;
      par ^= 1;
      if (it >= maxit) break;
      const double gn = o4[0], dn = o4[1] + sigma * o4[0];
      if (sqrt(o4[2]) <= inner || gn == 0.0) break;
      const double bt = gn / gamma;
      const double den = dn / gn - bt / alpha;
      if (!(den > 0.0) || !isfinite(den)) break;
      alpha = 1.0 / den;
      beta = bt;
      scalar_log(d, rank, it, alpha, beta);
      gamma = gn;
    }
    if (it >= maxit) {
      true_res = cluster_true_res<F>(cl, part, slot, op, b, dv(1), nc, first, stp);
      status = true_res <= tol_abs ? ST_CONVERGED : ST_MAXIT;
      break;
    }
  }
  res.iters = it;
  res.status = status;
  res.bnorm = bnorm;
  res.true_res = true_res;
}

// Mixed precision with several unknowns per thread in the binary32 sweeps when the system's
// row length allows: four with M = I, two with Jacobi (twice the vectors).  On 512 2D systems
// with Jacobi and 4 resident blocks per SM, two unknowns per thread gave 109.2 solves/s and
// one gave 103.  The batched launch and the serving kernel's large lane use this; its small
// lane keeps one per thread.  The widths can be set at build time (1, 2 or 4).
#ifndef PCG_CLUSTER_MX_JAC_VW
#define PCG_CLUSTER_MX_JAC_VW 2
#endif
#ifndef PCG_CLUSTER_MX_VW
#define PCG_CLUSTER_MX_VW 4
#endif
template <int F, bool JAC>
__device__ __forceinline__ void cluster_solve_mx_auto(cg::cluster_group& cl, double (*part)[4], int& slot,
                                                      const BatchSys& d, const BatchVecs& V, double tol, int maxit,
                                                      double eta, int max_restarts, BatchOut& res) {
  constexpr int W = JAC ? PCG_CLUSTER_MX_JAC_VW : PCG_CLUSTER_MX_VW;
  if constexpr (F != 4 && W > 1) {
    if (d.nx % W == 0) {
      cluster_solve_mx<F, JAC, W>(cl, part, slot, d, V, tol, maxit, eta, max_restarts, res);
      return;
    }
  }
  cluster_solve_mx<F, JAC, 1>(cl, part, slot, d, V, tol, maxit, eta, max_restarts, res);
}

}  // namespace pcgk
