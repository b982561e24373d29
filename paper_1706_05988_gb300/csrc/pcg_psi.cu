// Local rounding-error propagation analysis of shifted pipelined CG
// (arXiv 1706.05988, Section 3.2): psi_i(sigma) = max_{1<=j<=i} ||P_i(sigma) ... P_j(sigma)||_2
// with the 4x4 propagation matrix P_k(sigma) of Eq. (propmat_shifted).
// One thread per shift; the product is extended on the right (Q <- Q P_j for
// j = i, i-1, ..., 1) and its spectral norm taken after every factor.
#include <math.h>

#include "pcg_internal.h"

namespace pcgk {
namespace {

// Largest eigenvalue of a symmetric 4x4 matrix by cyclic Jacobi rotations.
// Each rotation (c, s) in the (p, q) plane zeroes B[p][q]: with
// theta = (B[q][q] - B[p][p]) / (2 B[p][q]), t = sign(theta) / (|theta| + sqrt(theta^2 + 1))
// is the smaller root of t^2 + 2 theta t - 1 = 0, c = 1 / sqrt(1 + t^2), s = t c.
__device__ double sym4_lambda_max(double B[4][4]) {
  for (int sweep = 0; sweep < 32; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int p = 0; p < 4; ++p) {
      dia += B[p][p] * B[p][p];
      for (int q = p + 1; q < 4; ++q) off += B[p][q] * B[p][q];
    }
    if (off <= 1e-34 * dia) break;
    for (int p = 0; p < 3; ++p) {
      for (int q = p + 1; q < 4; ++q) {
        const double bpq = B[p][q];
        if (bpq == 0.0) continue;
        const double theta = (B[q][q] - B[p][p]) / (2.0 * bpq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < 4; ++k) {  // columns p, q
          const double bkp = B[k][p], bkq = B[k][q];
          B[k][p] = c * bkp - s * bkq;
          B[k][q] = s * bkp + c * bkq;
        }
        for (int k = 0; k < 4; ++k) {  // rows p, q
          const double bpk = B[p][k], bqk = B[q][k];
          B[p][k] = c * bpk - s * bqk;
          B[q][k] = s * bpk + c * bqk;
        }
        B[p][q] = B[q][p] = 0.0;
      }
    }
  }
  double m = B[0][0];
  for (int p = 1; p < 4; ++p) m = fmax(m, B[p][p]);
  return m;
}

// ||Q||_2 = m * sqrt(lambda_max((Q/m)^T (Q/m))), m = max |Q_ij| (avoids overflow of Q^T Q).
__device__ double norm2_4x4(const double Q[4][4]) {
  double m = 0.0;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      if (!isfinite(Q[a][b])) return INFINITY;   // the product has overflowed
      m = fmax(m, fabs(Q[a][b]));
    }
  if (m == 0.0) return 0.0;
  double S[4][4], B[4][4];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) S[a][b] = Q[a][b] / m;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      double acc = 0.0;
      for (int k = 0; k < 4; ++k) acc += S[k][a] * S[k][b];
      B[a][b] = acc;
    }
  return m * sqrt(fmax(sym4_lambda_max(B), 0.0));
}

__global__ void k_psi(const double* __restrict__ alpha, const double* __restrict__ beta, int i,
                      const double* __restrict__ sig, int ngrid, double* __restrict__ psi) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ngrid) return;
  const double sg = sig[g];
  double Q[4][4];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) Q[a][b] = a == b ? 1.0 : 0.0;
  double best = 0.0;
  for (int j = i; j >= 1; --j) {
    const double al = alpha[j], be = beta[j];
    // P_j(sigma), Eq. (propmat_shifted)
    const double P[4][4] = {{1.0, -al * be, -al, 0.0},
                            {0.0, be, 1.0, 0.0},
                            {0.0, -al * be * sg, 1.0 - al * sg, -al * be},
                            {0.0, 0.0, 0.0, be}};
    double R[4][4];
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        double acc = 0.0;
        for (int k = 0; k < 4; ++k) acc += Q[a][k] * P[k][b];
        R[a][b] = acc;
      }
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) Q[a][b] = R[a][b];
    best = fmax(best, norm2_4x4(Q));
  }
  psi[g] = best;
}

// Variable shift (Section 4.1): one thread per schedule, P_j(sigma_{j-1}, sigma_j) of
// Eq. (propmat_varshifted); schedule g holds sigma_{-1}, sigma_0, ... at sched[g * stride + 0, 1, ...].
__global__ void k_psi_var(const double* __restrict__ alpha, const double* __restrict__ beta, int i,
                          const double* __restrict__ sched, int stride, int nsched, double* __restrict__ psi) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nsched) return;
  const double* sh = sched + (long long)g * stride;
  double Q[4][4];
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) Q[a][b] = a == b ? 1.0 : 0.0;
  double best = 0.0;
  for (int j = i; j >= 1; --j) {
    const double al = alpha[j], be = beta[j], sp = sh[j], ds = sh[j + 1] - sh[j];
    const double P[4][4] = {{1.0, -al * be, -al, 0.0},
                            {0.0, be, 1.0, 0.0},
                            {0.0, -al * be * sp, 1.0 - al * sp, -al * be},
                            {0.0, -be * ds, -ds, be}};
    double R[4][4];
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        double acc = 0.0;
        for (int k = 0; k < 4; ++k) acc += Q[a][k] * P[k][b];
        R[a][b] = acc;
      }
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) Q[a][b] = R[a][b];
    best = fmax(best, norm2_4x4(Q));
  }
  psi[g] = best;
}

}  // namespace

cudaError_t launch_psi_var(const double* alpha, const double* beta, int i, const double* sched, int stride,
                           int nsched, double* psi, cudaStream_t stream) {
  const int block = 64;
  k_psi_var<<<(nsched + block - 1) / block, block, 0, stream>>>(alpha, beta, i, sched, stride, nsched, psi);
  return cudaGetLastError();
}

cudaError_t launch_psi(const double* alpha, const double* beta, int i, const double* sig, int ngrid, double* psi,
                       cudaStream_t stream) {
  const int block = 64;
  k_psi<<<(ngrid + block - 1) / block, block, 0, stream>>>(alpha, beta, i, sig, ngrid, psi);
  return cudaGetLastError();
}

}  // namespace pcgk
