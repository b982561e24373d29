/*
 * pcg.h -- C ABI of libpcg: shifted pipelined Conjugate Gradients on one GB300.
 *
 * Method: S. Cools, W. Vanroose, "Numerically stable variants of the
 * communication-hiding pipelined Conjugate Gradients algorithm for the
 * parallel solution of large scale symmetric linear systems", arXiv 1706.05988.
 *   PCG_CG    Algorithm 1 (classic CG), Section 1.
 *   PCG_PCG   Algorithm 2 (pipelined CG), Section 2.1 -- run as Algorithm 3
 *             with sigma = 0, which is the same recurrence (end of Section 2.2).
 *   PCG_SPCG  Algorithm 3 (shifted pipelined CG), Section 2.2.
 * The problem is A x = b with A real symmetric positive definite (Section 2.1);
 * M^{-1} = I (the paper's Poisson experiments are unpreconditioned, Table 1).
 *
 * Conventions shared by every entry point
 *   - Every function returns a pcg_status and never aborts the process.
 *   - Vectors are contiguous binary64 arrays of length n.  Stencil unknowns
 *     are ordered x fastest, then y, then z.
 *   - Host pointers unless the entry point says "device"; device pointers
 *     must come from the CUDA device that was current when the context was
 *     created and stay owned by the caller.
 *   - All output buffers are caller-owned.  NULL history pointers are allowed.
 *   - A context is not thread-safe: serialise calls on one context.  Distinct
 *     contexts are independent.
 *   - All GPU work of a context runs on one CUDA stream (its own, or the one
 *     given to pcg_set_stream); solve calls return after that work finished.
 */
#ifndef PCG_H
#define PCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pcg_ctx pcg_ctx;

typedef enum {
  PCG_OK = 0,
  PCG_EINVAL = 1,      /* bad argument; nothing was changed                        */
  PCG_ENOMEM = 2,      /* device or host allocation failed                          */
  PCG_ECUDA = 3,       /* a CUDA call failed; see pcg_last_error                    */
  PCG_EBREAKDOWN = 4,  /* delta <= 0, or a non-finite / non-positive 1/alpha: the
                          iteration stopped; x and histories hold the last iterate */
  PCG_ENOTCONV = 5,    /* maxit reached before tol; x and histories are valid       */
  PCG_ETIMEOUT = 6,    /* a bounded device wait gave up                            */
  PCG_PENDING = 7,
  PCG_ENOTIMPL = 8
} pcg_status;

typedef enum { PCG_STENCIL5_2D = 0, PCG_STENCIL7_3D = 1, PCG_CSR32 = 2 } pcg_layout;
typedef enum { PCG_CG = 0, PCG_PCG = 1, PCG_SPCG = 2 } pcg_method;
typedef enum { PCG_FP64 = 0, PCG_MIXED_IR = 1 } pcg_precision;

/* pcg_create flags */
#define PCG_DEVICE_PTRS 0x1u   /* every array in pcg_matrix is a device pointer          */
#define PCG_PROFILE 0x2u       /* time every launch of the fused iteration kernel with
                                  CUDA events (read back with pcg_kernel_stats)          */
#define PCG_PERSISTENT 0x8u    /* PCG_PCG / PCG_SPCG in FP64 with true_every <= 0: run every
                                  iteration inside one cooperative launch; a grid barrier
                                  replaces the kernel boundary and each block overlaps the
                                  global reduction of (r,r), (w,r) with the SpMV of its next
                                  unit (the paper's communication hiding, Section 1).  Only
                                  the M = I, constant-shift path has this form; solves with
                                  PCG_JACOBI or a variable shift launch per iteration */
#define PCG_JACOBI 0x10u      /* preconditioner M^{-1} = diag(A)^{-1} (the paper's JAC, Table 1):
                                  Algorithm 3 with its separate preconditioned recurrences for
                                  u, q, p (PCG_PCG / PCG_SPCG, in FP64 or PCG_MIXED_IR),
                                  and Algorithm 1 with u = D^{-1} r (PCG_CG, FP64).
                                  D^{-1} is formed at creation: on the host from host
                                  arrays, on the device from PCG_DEVICE_PTRS arrays; a
                                  non-positive diagonal entry gives PCG_EINVAL */
#define PCG_STENCIL_FP64_SUM 0x4u  /* constant-coefficient stencils: sum each row with FP64
                                  additions instead of the default fixed-point row sum.
                                  Default: the row C*w_c - sum(neighbours) is summed exactly
                                  in 64-bit fixed point with 6 guard bits below the largest
                                  term and rounded once to binary64; its error is at most
                                  0.5 ulp of the result plus 6 * 2^-6 ulp of the largest
                                  term, below the worst case of FP64 left-to-right summation */
#define PCG_DOTS_SPLIT32 0x20u /* PCG_PCG / PCG_SPCG, FP64, M = I, constant shift, launch per
                                  iteration: accumulate the merged dots (r,r) and (w,r) on the
                                  FP32 pipe instead of with binary64 fused multiply-adds.  Each
                                  value is split exactly (integer operations) into two binary32
                                  parts after a power-of-two scale taken from the previous
                                  iteration's norms, and the products are summed error-free
                                  (TwoProd/TwoSum); about 2^-47 per term (1e-14 relative to the
                                  sum on Laplacian runs, against 1e-15 for binary64).  Values
                                  outside the scaled binary32 range are summed in binary64.
                                  It frees 2 of the sweep's 9 FP64 operations per unknown but
                                  adds about 50 integer/FP32 instructions; on GB300 the 256^3
                                  sweep is then slower (0.34 against 0.29 ms), so it is opt-in */

/*
 * The operator A.
 *  PCG_STENCIL5_2D / PCG_STENCIL7_3D: matrix-free cell-centred operator on an
 *    nx x ny (x nz) grid with Dirichlet boundary.  With diag == NULL it is the
 *    unscaled Laplacian (4 resp. 6 on the diagonal, -1 to each grid neighbour),
 *    the operator of the paper's lapl200 and Poisson experiments (Section 5).
 *    Otherwise (variable coefficients) row c is
 *        diag[c] x_c - ax[c] x_{c-1} - ax[c+1] x_{c+1} - ay[c] x_{c-nx}
 *                    - ay[c+nx] x_{c+nx} - az[c] x_{c-nx*ny} - az[c+nx*ny] x_{c+nx*ny}
 *    where ax/ay/az[c] is the coefficient of the face between c and its lower
 *    neighbour and must be 0 where that neighbour is outside the grid.  nz = 1
 *    and az unused in 2D.  n is ignored (n = nx*ny*nz).
 *  PCG_CSR32: n x n matrix, nnz entries, row_ptr[n+1] / col[nnz] int32, val[nnz];
 *    columns need not be sorted; every index must lie in [0, n).
 * The caller must pass an SPD matrix; symmetry is not checked.
 */
typedef struct {
  int32_t layout;
  int64_t nx, ny, nz;
  const double *diag, *ax, *ay, *az;
  int64_t n, nnz;
  const int32_t *row_ptr, *col;
  const double *val;
} pcg_matrix;

/*
 * Solve report.  History arrays (caller-owned, host, length maxit+1, may be
 * NULL) follow the index convention of Algorithm 3: alpha_hist[i], beta_hist[i]
 * are the scalars of iteration i (beta_hist[0] = 0), for i < iters;
 * rec_hist[i] = ||r_i||_2, the recursive residual, for i <= iters;
 * true_hist[i] = ||b - A x_i||_2 for i a multiple of true_every and i = iters
 * (other entries NaN; true_every <= 0 logs only i = iters).
 * gap_hist[i] = ||(b - A x_i) - r_i||_2, the residual gap f_i of Section 3.1,
 * logged with true_hist.
 */
typedef struct {
  int32_t iters;                /* out: iterations performed                       */
  int32_t status;               /* out: same value as the return code              */
  double final_true_relres;     /* out: ||b - A x|| / ||b|| at exit                */
  double final_rec_relres;      /* out: ||r_iters|| / ||b||                        */
  double *rec_hist, *true_hist, *gap_hist, *alpha_hist, *beta_hist;
  int32_t true_every;           /* in                                              */
} pcg_result;

/* Create a context for operator A: copies A to the device (or, with
 * PCG_DEVICE_PTRS, references the caller's device arrays, which must outlive
 * the context).  Device work vectors are allocated by the first solve.
 * Errors: PCG_EINVAL for a NULL/inconsistent description (non-positive sizes,
 * nx*ny*nz or nnz beyond int32 indexing, missing arrays); PCG_ENOMEM; PCG_ECUDA. */
pcg_status pcg_create(const pcg_matrix *A, uint32_t flags, pcg_ctx **out);

/* Release every device and host resource of the context.  NULL is a no-op. */
void pcg_destroy(pcg_ctx *ctx);

/* Last error message of the context ("" if none); valid until the next call. */
const char *pcg_last_error(const pcg_ctx *ctx);

/* Run all later GPU work of this context on `stream` (a cudaStream_t of the
 * context's device; NULL = the context's own stream). */
pcg_status pcg_set_stream(pcg_ctx *ctx, void *stream);

/* Solve A x = b.  b, x0 (NULL = zero) and x_out are host arrays of length n.
 * method: pcg_method; sigma: the shift of Algorithm 3 (must be >= 0; ignored
 * by PCG_CG and forced to 0 by PCG_PCG).  maxit >= 0.
 * precision PCG_FP64: every vector and operation in binary64.  tol: stop once the
 *   recursive residual satisfies ||r_i|| <= tol ||b|| (the scaled criterion of
 *   the paper's Section 5.2); tol = 0 runs exactly maxit iterations.
 * precision PCG_MIXED_IR (Algorithm 3 only, not PCG_CG): w, z, s, p stored and
 *   updated in binary32; x, r, the dot products (exact binary64 products, binary64
 *   sums), alpha, beta and sigma in binary64.  When the recursive residual reaches
 *   eta (PCG_PARAM_MIXED_ETA, default 2^-10) times the true residual of the last
 *   restart, the true residual b - A x is recomputed in binary64 and Algorithm 3
 *   restarts from the current x (iterative refinement).  tol applies to the true
 *   residual ||b - A x|| <= tol ||b||; the solve also ends at maxit iterations or
 *   when a restart does not lower the true residual (PCG_ENOTCONV).  true_hist
 *   holds the true residual at every restart and at exit.  On a PCG_JACOBI
 *   context u, q, t, p and m = D^{-1} w are binary32 as well; the restart forms
 *   u_0 = D^{-1} r rounded to binary32 and w_0 = A u_0 - sigma r in binary64.
 *   A variable shift (pcg_set_shifts) with PCG_MIXED_IR gives PCG_ENOTIMPL.
 * Returns PCG_OK on convergence, PCG_ENOTCONV at maxit (always when tol = 0),
 * PCG_EBREAKDOWN; res may be NULL.  x_out is written in every non-error case. */
pcg_status pcg_solve(pcg_ctx *ctx, const double *b, const double *x0, int32_t method, double sigma, double tol,
                     int32_t maxit, int32_t precision, double *x_out, pcg_result *res);

/* pcg_solve with b, x0 (NULL = zero) and x_out given as device pointers. */
pcg_status pcg_solve_device(pcg_ctx *ctx, const double *b, const double *x0, int32_t method, double sigma,
                            double tol, int32_t maxit, int32_t precision, double *x_out, pcg_result *res);

/* y = A x with the context's operator, evaluated exactly as inside the solver
 * (the SpMV of Algorithm 3, line "n_i := A m_i").  x and y are device arrays of
 * n doubles that must not overlap (any alignment).  Errors: PCG_EINVAL for
 * NULL pointers. */
pcg_status pcg_apply(pcg_ctx *ctx, const double *x, double *y);

/* Shift selection (Section 3.2, Eq. (functionpsi); Section 5.1): runs
 * Algorithm 2 (sigma = 0) for `iters` iterations on (A, b) -- b a host array --
 * and evaluates psi_i(sigma) = max_{1<=j<=i} ||P_i(sigma) ... P_j(sigma)||_2 on
 * the device for every shift of grid[ngrid] (host), with i the last iteration
 * whose alpha/beta exist.  sigma_out receives the smallest grid shift whose psi
 * is within a factor 2 of the grid minimum; psi_out (host, ngrid, may be NULL)
 * the psi values.  Errors: PCG_EINVAL (iters < 2, ngrid < 1, a negative shift). */
pcg_status pcg_select_sigma(pcg_ctx *ctx, const double *b, int32_t iters, const double *grid, int32_t ngrid,
                            double *sigma_out, double *psi_out);

/* psi_i(sigma) for given coefficient histories alpha[0..i], beta[0..i] (host)
 * and shifts grid[ngrid] (host), evaluated on the device; psi_out[ngrid] host. */
pcg_status pcg_psi(pcg_ctx *ctx, const double *alpha, const double *beta, int32_t i, const double *grid,
                   int32_t ngrid, double *psi_out);

/* psi_i for variable shifts (Section 4.1): the product of the propagation matrices
 * P_j(sigma_{j-1}, sigma_j) of Eq. (propmat_varshifted), j = i .. 1, with psi_i the
 * largest spectral norm of its partial products.  schedules (host) holds nsched
 * schedules, schedule g at schedules[g * stride ..] with the indexing of
 * pcg_set_shifts (entry 0 = sigma_{-1}, entry k + 1 = sigma_k); stride >= i + 2.
 * alpha[0..i], beta[0..i] host; psi_out[nsched] host.  A constant schedule gives
 * pcg_psi's value.  Errors: PCG_EINVAL for bad sizes or NULL arrays. */
pcg_status pcg_psi_varsh(pcg_ctx *ctx, const double *alpha, const double *beta, int32_t i,
                         const double *schedules, int32_t stride, int32_t nsched, double *psi_out);

/* ---- Batches of independent systems (one persistent launch) ------------------
 * Many systems A_k x_k = b_k, each solved by Algorithm 3 with its own shift (binary64
 * or mixed precision, M = I or Jacobi), advance together: every thread-block cluster
 * takes systems from a device queue (largest first) and runs all iterations of one
 * system, its blocks sharing the unknowns; the dot products reduce through
 * distributed shared memory and one cluster barrier per iteration replaces the
 * paper's global reduction.
 * All systems of a batch share one operator family (2D or 3D stencil, constant or
 * variable coefficients, or CSR) but not their sizes.  Systems are grouped into
 * three size classes (n < 8,192; < 65,536; larger), each with its own queue and
 * cluster size (default 2, 4, 8); the classes run concurrently, one kernel each,
 * launched together as one CUDA graph that is captured once and replayed while
 * the solve parameters stay the same. */
typedef struct pcg_batch pcg_batch;

/* Copy nsys operators (host arrays, pcg_matrix as for pcg_create) to the device,
 * with binary32 copies of their coefficients for mixed precision.  flags: 0 or
 * PCG_JACOBI (M^{-1} = diag(A)^{-1} for every system, as for pcg_create).
 * Errors: PCG_EINVAL (mixed families, invalid description, a non-positive diagonal
 * with PCG_JACOBI), PCG_ENOMEM, PCG_ECUDA. */
pcg_status pcg_batch_create(const pcg_matrix *systems, int32_t nsys, uint32_t flags, pcg_batch **out);

/* Solve every system: b[k] and x_out[k] are host arrays of n_k doubles; method
 * PCG_PCG or PCG_SPCG with sigma[k] >= 0 (sigma may be NULL for PCG_PCG); x_0 = 0;
 * stop at ||r_i|| <= tol ||b_k|| or after maxit iterations.  iters[k], status[k]
 * (a pcg_status per system) and true_relres[k] = ||b_k - A_k x_k|| / ||b_k|| may be
 * NULL.  Returns PCG_OK when every system converged, else PCG_ENOTCONV.
 * With precision PCG_MIXED_IR (pcg_batch_set_precision) each system runs the
 * mixed-precision iteration with restarts of pcg_solve's PCG_MIXED_IR and tol
 * applies to the true residual ||b_k - A_k x_k||; a restart that does not lower
 * the true residual ends that system's solve as not converged. */
pcg_status pcg_batch_solve(pcg_batch *batch, const double *const *b, double *const *x_out, int32_t method,
                           const double *sigma, double tol, int32_t maxit, int32_t *iters, int32_t *status,
                           double *true_relres);

/* Autotuner: times probe_iters iterations of the whole batch with one cluster size in
 * {1, 2, 4, 8, 16} for every class (ms_out[5], may be NULL: the time of each candidate,
 * NaN where a size cannot be launched; cluster_out, may be NULL: the fastest), then
 * times each size class alone for every candidate size and both register variants of
 * its kernel (see pcg_batch_classes) and keeps the fastest pair per class for later
 * solves.  pcg_batch_set_cluster sets one size for every class. */
pcg_status pcg_batch_autotune(pcg_batch *batch, const double *const *b, const double *sigma, int32_t probe_iters,
                              int32_t *cluster_out, double *ms_out);
pcg_status pcg_batch_set_cluster(pcg_batch *batch, int32_t cluster_size);

/* The three size classes: systems per class, current cluster size and the resident
 * blocks per SM of the class's kernel variant (arrays of 3, any may be NULL; blocks per SM
 * is 0 for a class not launched yet).  Each class's kernel exists compiled for 2 resident
 * blocks per SM (128 registers) and for 4 (64 registers, with spills): by default a class
 * takes 4 when it has more systems than a 2-block grid holds clusters, else 2; the
 * autotuner times both.  pcg_batch_set_class_cluster sets one class's cluster size (1, 2,
 * 4, 8 or 16), pcg_batch_set_class_occupancy its variant (2, 4, or 0 for the default
 * rule).  Errors: PCG_EINVAL. */
pcg_status pcg_batch_classes(const pcg_batch *batch, int32_t *nsys, int32_t *cluster, int32_t *blocks_per_sm);
pcg_status pcg_batch_set_class_cluster(pcg_batch *batch, int32_t size_class, int32_t cluster_size);
pcg_status pcg_batch_set_class_occupancy(pcg_batch *batch, int32_t size_class, int32_t blocks_per_sm);

/* Precision of later pcg_batch_solve calls: PCG_FP64 (default) or PCG_MIXED_IR.
 * pcg_batch_set_param takes PCG_PARAM_MIXED_ETA and PCG_PARAM_MAX_RESTARTS with the
 * meaning they have for pcg_set_param; the batch's default eta is 2^-14 (the per-cluster
 * solves restart less often than the single-system solver, default 2^-10), and
 * max_restarts defaults to 200 as there.  Errors: PCG_EINVAL. */
pcg_status pcg_batch_set_precision(pcg_batch *batch, int32_t precision);
pcg_status pcg_batch_set_param(pcg_batch *batch, int32_t param, double value);

/* CUDA-event time (ms) of the last batch kernel. */
pcg_status pcg_batch_last_kernel_ms(const pcg_batch *batch, double *ms);

/* alpha_i and beta_i (Algorithm 3, lines of the scalar step) of the first k iterations of
 * every system in the last pcg_batch_solve: alpha[s * k + i], beta[s * k + i] (host arrays
 * of nsys * k doubles, either may be NULL), 1 <= k <= PCG_SCALAR_LOG.  Entries past the
 * iterations a system ran are NaN; beta_0 = 0.  With PCG_MIXED_IR, i counts the inner
 * iterations across restarts, and a restart starts again from beta = 0.  The per-cluster
 * solvers record these values as they run (one store per iteration, i < PCG_SCALAR_LOG),
 * so they can be compared with a reference implementation iteration by iteration.
 * Waits for the batch's stream.  Errors: PCG_EINVAL, PCG_ECUDA. */
#define PCG_SCALAR_LOG 32
pcg_status pcg_batch_scalars(const pcg_batch *batch, int32_t k, double *alpha, double *beta);

void pcg_batch_destroy(pcg_batch *batch);

/* ---- Serving: continuous batching of solve requests ----------------------------
 * A server owns a device arena of hbm_budget_bytes.  pcg_submit admits a request when
 * its operator and vectors fit in the arena and a slot is free (first come, first
 * served); otherwise the request waits on the host until earlier requests are polled.
 * Admitted requests go to a persistent kernel whose thread-block clusters take them as
 * they come free, so requests that arrive while others run overlap on the device;
 * each request is solved by one cluster exactly as in pcg_batch (x_0 = 0).  There are
 * two such kernels side by side on a fixed split of the GPU: requests with
 * n < 32,768 go to one with many clusters of 2 blocks, larger requests to one with
 * 8 clusters of 16 blocks (a large request on a small cluster would set the tail
 * latency).  Requests with n >= 524,288 are solved on the whole GPU by
 * pcg_create/pcg_solve from host threads of the server (two such solves may run at the
 * same time), while both kernels pause (they finish what they hold, exit, and are
 * relaunched afterwards); their device memory is allocated outside the arena.  Another
 * host thread creates their solver contexts (device memory, the operator's upload) in
 * submission order, at most three at a time, so that these uploads overlap other work.
 * Smaller requests go first: a whole-GPU solve starts once the clusters have taken every
 * smaller request already published, or after 100 ms, whichever comes first.  Host data
 * of an admitted request is packed
 * into a pinned staging ring and copied without blocking; a request is published to
 * its kernel when its copies are done.  A request's arithmetic is fixed by its own
 * cluster (or by the single-system solver), so its result does not depend on what
 * else runs.  With no work for 20 ms a kernel exits and is relaunched by the next
 * submit or poll.  The server is internally synchronised (calls may come from several
 * host threads). */
typedef struct pcg_server pcg_server;

/* max_slots >= 1 requests in flight at once; hbm_budget_bytes >= 1 MiB.
 * Errors: PCG_EINVAL, PCG_ENOMEM (the arena cannot be allocated), PCG_ECUDA. */
pcg_status pcg_server_create(size_t hbm_budget_bytes, int32_t max_slots, pcg_server **out);

/* Queue a solve of A x = b (host arrays, copied): method PCG_PCG or PCG_SPCG, stop at
 * ||r_i|| <= tol ||b|| or maxit.  sigma < 0 selects the mean diagonal entry of A (for
 * the unscaled Laplacians half the top of the spectrum, as Table 1's lapl200 shift).
 * *ticket identifies the request.  Errors: PCG_EINVAL; PCG_ENOMEM when the request can
 * never fit in the arena. */
pcg_status pcg_submit(pcg_server *server, const pcg_matrix *A, const double *b, double tol, int32_t method,
                      double sigma, int32_t maxit, uint64_t *ticket);

/* pcg_submit with a preconditioner and a precision for this request: flags 0 or
 * PCG_JACOBI (M^{-1} = diag(A)^{-1}, as for pcg_create); precision PCG_FP64 or
 * PCG_MIXED_IR (binary32 auxiliary vectors with binary64 restarts as in pcg_solve,
 * at most 200 restarts, eta = 2^-14 in the cluster lanes and pcg_solve's default 2^-10
 * for requests of n >= 2^19, which the single-system solver takes on the whole GPU;
 * tol then applies to the true residual).  The
 * request's arena block also holds its Jacobi vectors and binary32 coefficients.
 * With PCG_JACOBI, sigma < 0 selects 1, the mean diagonal entry of M^{-1} A.
 * pcg_submit(...) is pcg_submit_ex(..., 0, PCG_FP64, ticket).  Errors as pcg_submit,
 * and PCG_EINVAL for unknown flags or precision or a non-positive diagonal. */
pcg_status pcg_submit_ex(pcg_server *server, const pcg_matrix *A, const double *b, double tol, int32_t method,
                         double sigma, int32_t maxit, uint32_t flags, int32_t precision, uint64_t *ticket);

/* PCG_PENDING until the request is done; then x_out (host, n doubles, may be NULL) and
 * res (iters, status, final_true_relres; may be NULL) are filled, the request's memory
 * is released and its status is returned (PCG_OK, PCG_ENOTCONV, PCG_EBREAKDOWN); the
 * ticket is then no longer valid (PCG_EINVAL).  When res->alpha_hist / res->beta_hist
 * are set, their first min(iters, PCG_SCALAR_LOG) entries receive alpha_i and beta_i of
 * the request's solve (as pcg_batch_scalars reports them); the other histories are not
 * kept for served requests. */
pcg_status pcg_poll(pcg_server *server, uint64_t ticket, double *x_out, pcg_result *res);

/* Requests waiting for admission, requests admitted and not yet polled, free arena bytes. */
pcg_status pcg_server_stats(pcg_server *server, int64_t *waiting, int64_t *inflight, size_t *free_bytes);

/* Stops the kernel and releases everything (pending requests are dropped). */
void pcg_server_destroy(pcg_server *server);

/* Self-check of the binary32 <-> binary64 conversions that the mixed-precision
 * kernels perform with integer operations (the paper has no counterpart):
 * f_out[i] = (float)d_in[i] (round to nearest even) and d_out[i] = (double)f_in[i],
 * for i < n, on device arrays; synchronises the device.  NaN inputs give a quiet NaN.
 * Errors: PCG_EINVAL (n < 0 or a NULL array with n > 0), PCG_ECUDA. */
pcg_status pcg_convert_check(const double *d_in, float *f_out, const float *f_in, double *d_out, int64_t n);

/* Largest n accepted by pcg_true_residual_noalloc. */
#define PCG_NOALLOC_MAX_N 16777216

/* ||b - A x||_2 and ||(b - A x) - r||_2 without allocating anything.
 * The paper has no counterpart: this entry point exists for callers that must not
 * allocate device memory -- an application whose device memory is owned by another
 * allocator (a framework's caching pool that holds the whole GPU), a latency-bound
 * loop that cannot afford cudaMalloc's implicit device synchronisation, or a
 * program that fixes its memory footprint at start-up.  It needs no context: A
 * describes the operator as for pcg_create with PCG_DEVICE_PTRS (every array a
 * device pointer); b, x and r (r may be NULL) are device arrays of n doubles,
 * 16-byte aligned; norms is a device array of 2 doubles that receives
 * ||b - A x||_2 and ||(b - A x) - r||_2 (NaN when r is NULL).  A is evaluated as
 * inside the solver (fixed-point rows for constant-coefficient stencils).
 * The work is queued on `stream` (NULL = the default stream) and the call returns
 * without waiting; norms is valid once the stream reaches that point.
 * Scratch: one file-scope device array of 64 KiB (per-block partial sums and a
 * ticket), held by every GPU that loads this library until the process exits.  Every
 * call made outside stream capture looks up that array's address in the current
 * context (no device work) and keeps it for the device; a call on a capturing stream
 * uses the address kept by the last call outside capture on that device.  So make
 * one call outside capture before capturing, and again after anything that destroys
 * and recreates the device's context (cudaDeviceReset).  Every call shares the array: calls whose
 * work overlaps on a GPU (other streams, other host threads) race and give wrong
 * norms; serialise them.  No cudaMalloc, cudaFree or other allocating call is made.
 * Errors: PCG_EINVAL for NULL pointers, an invalid description, a vector or norms
 * not 8-byte aligned, b, x or r not 16-byte aligned where the operator reads two
 * unknowns per thread (stencils with an even row length), or n > PCG_NOALLOC_MAX_N (16,777,216 unknowns); PCG_ECUDA if a CUDA call fails. */
pcg_status pcg_true_residual_noalloc(const pcg_matrix *A, const double *b, const double *x, const double *r,
                                     double *norms, void *stream);

/* ---- one rank's share of a single system on several GPUs (Section 1; Section 5.2's MPI
 * setting).  The global grid is the 3D 7-point constant-coefficient Laplacian of
 * pcg_matrix (PCG_STENCIL7_3D, no coefficients), cut into slabs of whole z planes, one per
 * rank.  The SpMV of a rank needs its neighbours' boundary planes (one plane below, one
 * above); the dot products need one global reduction of two scalars per iteration.
 * A slab runs the phases of Algorithm 3 as kernels on its stream; the caller moves the
 * halo planes and reduces the dots (torch.distributed / NCCL, or copies between slabs in
 * one process) between the phases, so that the reduction overlaps the SpMV:
 *
 *   pcg_slab_start(local)           r = b, x = z = s = p = 0; local (b, b)
 *   reduce(local -> global); pcg_slab_set_bnorm(global)
 *   halo <- neighbours' boundary planes of r; pcg_slab_spmv(R, W, all planes)
 *   pcg_slab_w0(local)              w_0 = A r_0 - sigma r_0; local (r, r), (w_0, r)
 *   for i = 0, 1, ...:
 *     start reduce(local -> global); start halo <- neighbours' boundary planes of w
 *     pcg_slab_spmv(W, N, interior planes); wait halo; pcg_slab_spmv(W, N, boundary planes)
 *     wait reduce; pcg_slab_scalars(global, i == 0)      alpha_i, beta_i, stop tests
 *     pcg_slab_update(local)       z, s, p, x, r, w (in place); local (r, r), (w, r)
 *
 * All vectors are caller-owned device arrays of nx*ny*nz_local doubles (8-byte aligned;
 * 16-byte aligned with an even nx for two unknowns per thread), the halos nx*ny doubles;
 * the dots are device arrays of 2 doubles.  Plane k of a vector starts at k*nx*ny. */
typedef struct pcg_slab pcg_slab;
typedef struct {
  double *x, *r, *w, *z, *s, *p, *n;    /* n receives A w (or A x for the true residual) */
  const double *b;
  const double *halo_below, *halo_above;   /* the neighbour's plane next to this slab */
} pcg_slab_vectors;
#define PCG_SLAB_X 0
#define PCG_SLAB_R 1
#define PCG_SLAB_W 2
#define PCG_SLAB_N 3
#define PCG_SLAB_ALL_PLANES 0
#define PCG_SLAB_INTERIOR_PLANES 1   /* planes 1 .. nz_local - 2: no halo needed */
#define PCG_SLAB_BOUNDARY_PLANES 2   /* planes 0 and nz_local - 1 */

/* A slab of nz_local planes of an nx x ny grid; has_below / has_above: a neighbour slab
 * exists on that side (else the Dirichlet boundary of the global grid); maxit: the most
 * iterations (histories of maxit + 1 entries are kept on the device).
 * Errors: PCG_EINVAL (sizes, NULL or misaligned vectors), PCG_ENOMEM, PCG_ECUDA. */
pcg_status pcg_slab_create(int64_t nx, int64_t ny, int64_t nz_local, int32_t has_below, int32_t has_above,
                           const pcg_slab_vectors *v, int32_t maxit, pcg_slab **out);
pcg_status pcg_slab_set_stream(pcg_slab *slab, void *stream);
/* sigma >= 0: the shift; tol: stop once ||r_i|| <= tol ||b|| (0: run maxit iterations). */
pcg_status pcg_slab_start(pcg_slab *slab, double sigma, double tol, double *local_dots);
pcg_status pcg_slab_set_bnorm(pcg_slab *slab, const double *global_dots);
/* dst = A src on the given planes (src, dst: PCG_SLAB_*; dst is W or N and differs from src). */
pcg_status pcg_slab_spmv(pcg_slab *slab, int32_t src, int32_t dst, int32_t planes);
pcg_status pcg_slab_w0(pcg_slab *slab, double *local_dots);
pcg_status pcg_slab_scalars(pcg_slab *slab, const double *global_dots, int32_t first);
pcg_status pcg_slab_update(pcg_slab *slab, double *local_dots);
/* After pcg_slab_spmv(X, N, ...): local ||b - A x||^2 and ||(b - A x) - r||^2. */
pcg_status pcg_slab_true_residual(pcg_slab *slab, double *local_sums);
/* Waits for the slab's stream; status: PCG_PENDING while running, then PCG_OK /
 * PCG_ENOTCONV (maxit) / PCG_EBREAKDOWN; iter: the last iteration's index; bnorm: ||b||. */
pcg_status pcg_slab_state(pcg_slab *slab, int32_t *iter, int32_t *status, double *bnorm);
/* The first k entries of alpha_i, beta_i and ||r_i|| (host arrays, any may be NULL). */
pcg_status pcg_slab_history(pcg_slab *slab, int32_t k, double *alpha, double *beta, double *rec);
const char *pcg_slab_last_error(const pcg_slab *slab);
void pcg_slab_destroy(pcg_slab *slab);

/* Variable shift, Algorithm 4 (Section 4.1): later PCG_SPCG solves on this context use
 * shifts[0] = sigma_{-1} (the shift of w_0) and shifts[k + 1] = sigma_k for iteration k,
 * with the correction terms of Algorithm 4 in s, q, z and w; the sigma argument of the
 * solve is then ignored.  count must be at least maxit + 1 at solve time (else the solve
 * fails with PCG_EINVAL).  shifts = NULL or count <= 0 returns to a constant shift.
 * Errors: PCG_EINVAL for a negative or non-finite shift. */
pcg_status pcg_set_shifts(pcg_ctx *ctx, const double *shifts, int32_t count);

/* Solver parameters (not part of the paper's method statement).
 *   PCG_PARAM_MIXED_ETA      inner tolerance of PCG_MIXED_IR, in (0, 1); default 2^-10
 *   PCG_PARAM_MAX_RESTARTS   most restarts of one PCG_MIXED_IR solve, >= 1; default 200
 *   PCG_PARAM_TRUE_TOL       PCG_FP64 solves with res->true_every > 0: also stop once a
 *                            logged true residual satisfies ||b - A x_i|| <= value ||b||
 *                            (the true residual is checked every true_every iterations);
 *                            0 (the default) turns it off
 *   PCG_PARAM_BARRIER_TIMEOUT_MS, PCG_PARAM_TEST_BARRIER_PHANTOMS, PCG_PARAM_ITER_STAGES: see below
 * Errors: PCG_EINVAL for an unknown parameter or a value out of range. */
#define PCG_PARAM_MIXED_ETA 1
#define PCG_PARAM_MAX_RESTARTS 2
#define PCG_PARAM_BARRIER_TIMEOUT_MS 3   /* PCG_PERSISTENT: longest grid-barrier wait before
                                            the solve ends with PCG_ETIMEOUT; default 2000 */
#define PCG_PARAM_TEST_BARRIER_PHANTOMS 4 /* PCG_PERSISTENT, for tests of the time limit: the
                                            barrier waits for this many arrivals that never
                                            come (0 = off, the default) */
#define PCG_PARAM_TRUE_TOL 5
#define PCG_PARAM_ITER_STAGES 6   /* the fused iteration of PCG_PCG / PCG_SPCG (FP64, M = I,
                                     constant shift, launch per iteration) on a constant-
                                     coefficient stencil with an even row length: 2 or 3 =
                                     every operand of a block's chunk (z, s, p, x, r, and w's
                                     rows with their neighbour rows and planes) is staged in
                                     shared memory by TMA bulk copies, a ring of that many
                                     chunks; 0 (default) = every thread loads its own
                                     unknowns.  The staged ring takes 72 KB per block at
                                     256^3, so 3 blocks fit on an SM instead of 4, and the
                                     256^3 sweep is slower (0.33 against 0.29 ms) */
pcg_status pcg_set_param(pcg_ctx *ctx, int32_t param, double value);

/* The current value of a parameter of pcg_set_param.  For PCG_PARAM_ITER_STAGES this is the
 * depth in use: 0 where the operator cannot be staged (CSR, variable coefficients, odd row
 * length) or where two blocks' rings do not fit in one SM's shared memory.
 * Errors: PCG_EINVAL for a NULL argument or an unknown parameter. */
pcg_status pcg_get_param(const pcg_ctx *ctx, int32_t param, double *value);

/* Kernel accounting of the context since creation (or the last reset):
 * total launches of every kernel of this library, and -- with PCG_PROFILE --
 * the launches and summed CUDA-event time (ms) of the fused iteration kernel. */
pcg_status pcg_kernel_stats(pcg_ctx *ctx, int64_t *launches_total, int64_t *iter_launches, double *iter_ms);
pcg_status pcg_kernel_stats_reset(pcg_ctx *ctx);

/* Index checks of the checked build (libpcg_checked.so, compiled with -DPCG_CHECKED; the
 * paper has no counterpart: a stand-in for a memory checker).  The kernels of that build
 * check every index they turn into an address (stencil neighbours and coefficients, CSR
 * rows and columns, bulk copies, halo planes); a failed check records its code and skips
 * the access.  This call waits for the device, reports the first recorded code since the
 * last call in *code (0: none; the codes are listed in csrc/pcg_check.cuh) and clears it;
 * *checked (may be NULL) is 1 in the checked build, 0 in others (where *code is always 0).
 * Errors: PCG_EINVAL (code NULL), PCG_ECUDA. */
pcg_status pcg_check_status(uint32_t *code, int32_t *checked);

/* Version string of the library build. */
const char *pcg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PCG_H */
