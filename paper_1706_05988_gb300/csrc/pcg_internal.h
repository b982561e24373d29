// Internal interface between the C-ABI layer (pcg_capi.cu) and the kernels
// (pcg_kernels.cu, pcg_psi.cu).  Plain structs shared by host and device code.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pcgk {

// Run state of one solve (device memory).
// ST_RESTART (mixed precision only): the inner iteration reached its tolerance;
// the restart kernels recompute the true residual in FP64 and restart Algorithm 3.
// ST_STALLED (mixed precision only): a restart did not lower the true residual.
// ST_TIMEOUT (persistent kernel only): a grid-barrier wait exceeded its time limit.
enum : int { ST_RUNNING = 0, ST_CONVERGED = 1, ST_BREAKDOWN = 2, ST_MAXIT = 3, ST_RESTART = 4, ST_STALLED = 5,
             ST_TIMEOUT = 6 };

struct State {
  int iter;              // index i of the next iteration to execute (or of the last iterate once stopped)
  int status;            // ST_*
  int maxit;
  int pad0;
  double sigma;          // shift of Algorithm 3 (0 for Algorithms 1 and 2)
  double tol_abs;        // stop once ||r_i|| <= tol_abs (0: never)
  double bnorm;          // ||b||_2
  unsigned int ticket;   // last-block ticket of the running reduction (reset to 0 by its finisher)
  unsigned int pad1;
  // mixed precision with restarts (iterative refinement)
  double tol_rel;        // outer tolerance on ||b - A x|| / ||b||
  double eta;            // inner tolerance, relative to the true residual at the restart
  double rprev;          // true residual at the previous restart
  int restarts;          // restarts performed
  int max_restarts;
  // grid barrier of the persistent kernel
  unsigned int bar_count;
  unsigned int bar_gen;
  // stop once the logged true residual ||b - A x_i|| <= tol_true ||b|| (0: never)
  double tol_true;
  // power-of-two scales of r and w for the next iteration's FP32-pipe dot products
  // (pcg_ffdot.cuh), set by the finisher of Algorithm 3
  int ff_sr;
  int ff_sw;
};

// Per-iteration histories (device arrays of maxit + 1 entries).
struct Hist {
  double *alpha, *beta, *gamma, *delta, *rec, *tru, *gap;
};

// The operator: a cell-centred stencil (2D 5-point / 3D 7-point, constant or
// variable coefficients) or a CSR matrix.  Device pointers.
struct OpDesc {
  int layout;            // 0 = 2D stencil, 1 = 3D stencil, 2 = CSR
  int fixed_sum;         // constant-coefficient stencil rows in fixed point (pcg_fixedsum.cuh)
  int ff_dots;           // merged dots of the fused iteration on the FP32 pipe (pcg_ffdot.cuh)
  int iter_stages;       // fused iteration: 0 = register sweep, 2 or 3 = TMA-staged ring of that depth
  int n, nx, ny, nz;
  const double *diag, *ax, *ay, *az;   // variable coefficients; diag == nullptr: Laplacian
  const int *row_ptr, *col;
  const double *val;
  // binary32 copies used by the mixed-precision inner iteration
  const float *diag32, *ax32, *ay32, *az32, *val32;
};

// Solver vectors (device, n entries each, 256-byte aligned).
struct Vecs {
  const double* b;
  double *x, *r, *w0, *w1, *z, *s, *p;
  const double* dinv = nullptr;   // Algorithm 1 with M^{-1} = D^{-1} (nullptr: M = I)
};

struct Launch {
  int grid, block;
  cudaStream_t stream;
};

// Number of vector lanes per thread the kernels use for this operator
// (2 = 128-bit loads; needs an even row length for stencils).
int op_vec(const OpDesc& op);

// The staging depth the fused iteration uses for this operator when `stages` (0, 2 or 3)
// is asked for: 0 where the operator cannot be staged or the ring does not fit twice per SM.
int resolve_iter_stages(const OpDesc& op, int stages);

// Resident-grid size of each kernel family for this operator (0 on error).
int grid_for(const OpDesc& op, int kind, int block);
enum { K_RESIDUAL = 0, K_SPCG_W0, K_SPCG_ITER, K_TRUE_RES, K_CG_P0, K_CG_SPMV, K_CG_UPDATE, K_CG_P, K_APPLY, K_NKINDS };

// Kernel launchers (asynchronous; return the launch error).
cudaError_t launch_residual(const OpDesc& op, const Launch& L, const double* b, const double* x0, double* x, double* r,
                            State* st, double* partials);
cudaError_t launch_spcg_w0(const OpDesc& op, const Launch& L, Vecs v, State* st, Hist h, double* partials);
cudaError_t launch_spcg_iter(const OpDesc& op, const Launch& L, Vecs v, State* st, Hist h, double* partials);
cudaError_t launch_true_res(const OpDesc& op, const Launch& L, Vecs v, State* st, Hist h, double* partials);
cudaError_t launch_cg_p0(const OpDesc& op, const Launch& L, Vecs v, State* st, Hist h, double* partials);
cudaError_t launch_cg_spmv(const OpDesc& op, const Launch& L, Vecs v, State* st, Hist h, double* partials);
cudaError_t launch_cg_update(const OpDesc& op, const Launch& L, Vecs v, State* st, Hist h, double* partials);
cudaError_t launch_cg_p(const OpDesc& op, const Launch& L, Vecs v, State* st, Hist h);
cudaError_t launch_apply(const OpDesc& op, const Launch& L, const double* x, double* y);

// General iteration: Jacobi preconditioner and/or variable shift (pcg_general.cuh).
struct GenVecs;
// D^{-1} of a matrix whose arrays are on the device; *bad (device) is set for a non-positive diagonal.
cudaError_t launch_jacobi_dinv(const OpDesc& op, double* dinv, int* bad, cudaStream_t stream);
// jac: D^{-1} recurrences; var: variable-shift correction terms (at least one is set)
int grid_for_general(const OpDesc& op, bool jac, bool var);
cudaError_t launch_gen_w0(const OpDesc& op, const Launch& L, const GenVecs& v, State* st, Hist h, double* partials,
                          bool jac, bool var);
cudaError_t launch_gen_iter(const OpDesc& op, const Launch& L, const GenVecs& v, State* st, Hist h, double* partials,
                            bool jac, bool var);

// Persistent cooperative form of the iteration (pcg_persistent.cuh).
int grid_for_persistent(const OpDesc& op);
cudaError_t launch_spcg_persistent(const OpDesc& op, int grid, cudaStream_t stream, Vecs v, State* st, Hist h,
                                   double* partials, unsigned long long timeout_ns, unsigned phantoms);

// Mixed precision (pcg_mixed.cuh): FP32 w, z, s, p stored in the FP64 buffers of Vecs.
enum { KM_RESTART = 0, KM_W0, KM_ITER, KM_W0_JAC, KM_ITER_JAC, KM_NKINDS };
int mixed_vec(const OpDesc& op);
int grid_for_mixed(const OpDesc& op, int kind, int block);
cudaError_t launch_mx_restart(const OpDesc& op, const Launch& L, Vecs v, State* st, Hist h, double* partials);
cudaError_t launch_mx_w0(const OpDesc& op, const Launch& L, Vecs v, State* st, Hist h, double* partials);
cudaError_t launch_mx_iter(const OpDesc& op, const Launch& L, Vecs v, State* st, Hist h, double* partials);
cudaError_t launch_to_f32(const double* src, float* dst, long long n, cudaStream_t stream);
// Mixed precision with M^{-1} = D^{-1} (pcg_mixed_jacobi.cuh); v holds the binary32 vectors.
cudaError_t launch_mxj_u0(const GenVecs& v, double* u64, int n, const State* st, cudaStream_t stream);
cudaError_t launch_mxj_w0(const OpDesc& op, const Launch& L, const GenVecs& v, double* u64, State* st, Hist h,
                         double* partials);
cudaError_t launch_mxj_iter(const OpDesc& op, const Launch& L, const GenVecs& v, State* st, Hist h,
                           double* partials);

// psi_i(sigma) for every shift of sig[ngrid]; alpha/beta device arrays (>= i+1 entries).
cudaError_t launch_psi_var(const double* alpha, const double* beta, int i, const double* sched, int stride,
                           int nsched, double* psi, cudaStream_t stream);
cudaError_t launch_psi(const double* alpha, const double* beta, int i, const double* sig, int ngrid, double* psi,
                       cudaStream_t stream);

constexpr int kBlockThreads = 256;        // block size of every solver kernel
constexpr int kMaxPartialBlocks = 8192;   // capacity of the per-block partial-sum buffer
constexpr int kPartialsPerBlock = 2;

}  // namespace pcgk
