/*
 * Oracle for the pipelined-CG hot path: plain, slow, single-threaded FP64 C.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header or helper with the CUDA path.
 *
 * The vector loops carry OpenMP pragmas.  The library the tests and the parity checks
 * use is built without -fopenmp, so the pragmas are ignored and every loop runs in the
 * order written.  bench.py also times a second build with -fopenmp (a baseline on all
 * host cores); its reductions sum in another order, so it is never used as a reference.
 *
 * Source: S. Cools, W. Vanroose, "Numerically stable variants of the
 * communication-hiding pipelined Conjugate Gradients algorithm for the parallel
 * solution of large scale symmetric linear systems" (arXiv 1706.05988).
 *
 *   oracle_cg      Algorithm 1 (classic preconditioned CG), Section 1.
 *   oracle_pcg     Algorithm 2 (pipelined CG), Section 2.1.
 *   oracle_pcg_sh  Algorithm 3 (shifted pipelined CG), Section 2.2, with the
 *                  auxiliary definitions of Eq. (pipe_cg_shift_aux).
 *   oracle_pcg_varsh  Algorithm 4 (variable shift), Section 4.1.
 *   oracle_apply   the operator A (CSR or a matrix-free 5/7-point stencil).
 *
 * Readings of the paper taken here:
 *   - M^{-1} is either the identity (minv == NULL) or a diagonal matrix given
 *     by its entries; the nine-vector general form is kept in every case.
 *   - In the three-term recurrences for r and u the second and third terms
 *     are summed first (Section 3.1, remark after Eq. (errorterms)):
 *     r - (alpha*s + (alpha*sigma)*t).  Build with -ffp-contract=off so that
 *     no multiply-add is fused.
 *   - delta is the dot product (w + sigma*r, u) formed element by element.
 *   - Breakdown: gamma == 0 means the residual vanished exactly (converged);
 *     a non-finite or non-positive delta, or denominator of alpha, is a breakdown.
 *   - Dots and norms are plain left-to-right sums.
 *
 * Pins: every routine is checked by tests/test_oracle.py.  Parity unpinned: the
 * level at which oracle_pcg (unshifted) stalls on lapl200, printed as 3.1e-7 in
 * Table 1; it depends on rounding after the iteration has lost its way, and only
 * its order relative to CG is tested.
 *
 * All history arrays are optional (NULL) and, when given, hold maxit+1 entries.
 * Index conventions (both methods): alpha[i], beta[i] are the scalars used in
 * iteration i (beta[0] = 0); rec[i] = ||r_i||_2 (recursive residual);
 * tru[i] = ||b - A x_i||_2 and gap[i] = ||(b - A x_i) - r_i||_2 when i is a
 * multiple of log_every and at the final iterate (NaN otherwise; log_every <= 0
 * disables them).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

enum { OP_CSR = 0, OP_STENCIL2D = 1, OP_STENCIL3D = 2 };

/* Threads of the OpenMP build (returns the count in use; 1 in the serial build). */
int oracle_threads(int32_t nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
  return omp_get_max_threads();
#else
  (void)nthreads;
  return 1;
#endif
}

typedef struct {
  int32_t kind;
  int64_t n, nx, ny, nz;
  const int32_t *row_ptr, *col;
  const double *val;
  /* variable-coefficient stencil (NULL = constant Laplacian, diagonal 4 or 6,
     off-diagonals -1): diag[c]; ax/ay/az[c] = coefficient of the face between
     cell c and its lower x / y / z neighbour (0 on the boundary) */
  const double *diag, *ax, *ay, *az;
} oracle_op;

typedef struct {
  int32_t iters;     /* iterations performed */
  int32_t status;    /* 0 maxit reached, 1 converged (tolerance or exact), 2 breakdown */
} oracle_info;

/* Optional final-state export of Algorithm 3 (any pointer may be NULL). */
typedef struct {
  double *x, *r, *u, *w, *z, *q, *s, *t, *p;
} oracle_state;

/* ---- operator ------------------------------------------------------------ */

/* y = A x.  CSR: row sums in storage order.  Stencil: centre term, then the
   neighbours -x, +x, -y, +y, -z, +z that lie inside the Dirichlet domain. */
void oracle_apply(const oracle_op *A, const double *x, double *y) {
  if (A->kind == OP_CSR) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < A->n; ++i) {
      double acc = 0.0;
      for (int32_t k = A->row_ptr[i]; k < A->row_ptr[i + 1]; ++k) acc += A->val[k] * x[A->col[k]];
      y[i] = acc;
    }
    return;
  }
  const int64_t nx = A->nx, ny = A->ny, nz = (A->kind == OP_STENCIL3D) ? A->nz : 1;
  const int is3d = (A->kind == OP_STENCIL3D);
  const double centre = is3d ? 6.0 : 4.0;
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        const int64_t c = (k * ny + j) * nx + i;
        double acc;
        if (A->diag == NULL) {
          acc = centre * x[c];
          if (i > 0) acc -= x[c - 1];
          if (i < nx - 1) acc -= x[c + 1];
          if (j > 0) acc -= x[c - nx];
          if (j < ny - 1) acc -= x[c + nx];
          if (is3d && k > 0) acc -= x[c - nx * ny];
          if (is3d && k < nz - 1) acc -= x[c + nx * ny];
        } else {
          acc = A->diag[c] * x[c];
          if (i > 0) acc -= A->ax[c] * x[c - 1];
          if (i < nx - 1) acc -= A->ax[c + 1] * x[c + 1];
          if (j > 0) acc -= A->ay[c] * x[c - nx];
          if (j < ny - 1) acc -= A->ay[c + nx] * x[c + nx];
          if (is3d && k > 0) acc -= A->az[c] * x[c - nx * ny];
          if (is3d && k < nz - 1) acc -= A->az[c + nx * ny] * x[c + nx * ny];
        }
        y[c] = acc;
      }
}

double oracle_dot(int64_t n, const double *a, const double *b) {
  double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

double oracle_nrm2(int64_t n, const double *a) { return sqrt(oracle_dot(n, a, a)); }

/* M^{-1} v (identity when minv == NULL). */
static void apply_minv(int64_t n, const double *minv, const double *v, double *out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) out[i] = minv ? minv[i] * v[i] : v[i];
}

/* tru/gap logging: ||b - A x|| and ||(b - A x) - r|| */
static void log_true(const oracle_op *A, const double *b, const double *x, const double *r, double *work,
                     double *tru_out, double *gap_out) {
  const int64_t n = A->n;
  oracle_apply(A, x, work);
  double s1 = 0.0, s2 = 0.0;
#pragma omp parallel for reduction(+ : s1, s2) schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    const double e = b[i] - work[i];
    const double g = e - r[i];
    s1 += e * e;
    s2 += g * g;
  }
  if (tru_out) *tru_out = sqrt(s1);
  if (gap_out) *gap_out = sqrt(s2);
}

static int want_log(int64_t i, int32_t log_every) { return log_every > 0 && (i % log_every) == 0; }

static void fill_nan(double *a, int32_t m) {
  if (!a) return;
  for (int32_t i = 0; i < m; ++i) a[i] = NAN;
}

static double *zeros(int64_t n) { return (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double)); }

/* ---- Algorithm 1: classic preconditioned CG ------------------------------ */

/* Stops after maxit iterations, or before iteration i once ||r_i|| <= rtol*||b||
   (rtol > 0), or once the logged true residual satisfies ||b-Ax_i|| <= ttol*||b||
   (ttol > 0).  x holds x0 on entry (NULL x0 means zero) and x_i on exit. */
int oracle_cg(const oracle_op *A, const double *minv, const double *b, double *x, int32_t maxit, double rtol,
              double ttol, int32_t log_every, double *alpha, double *beta, double *rec, double *tru, double *gap,
              oracle_info *info) {
  const int64_t n = A->n;
  double *r = zeros(n), *u = zeros(n), *p = zeros(n), *s = zeros(n), *work = zeros(n);
  if (!r || !u || !p || !s || !work) return -1;
  fill_nan(alpha, maxit + 1); fill_nan(beta, maxit + 1); fill_nan(rec, maxit + 1);
  fill_nan(tru, maxit + 1); fill_nan(gap, maxit + 1);
  const double bnorm = oracle_nrm2(n, b);

  oracle_apply(A, x, work);                         /* r_0 := b - A x_0 */
  #pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j) r[j] = b[j] - work[j];
  apply_minv(n, minv, r, u);                        /* u_0 := M^{-1} r_0 */
  memcpy(p, u, (size_t)n * sizeof(double));         /* p_0 := u_0 */
  double gamma = oracle_dot(n, r, u);
  if (beta) beta[0] = 0.0;

  int32_t i = 0, status = 0;
  for (;; ++i) {
    if (rec) rec[i] = oracle_nrm2(n, r);
    if (want_log(i, log_every)) log_true(A, b, x, r, work, tru ? &tru[i] : NULL, gap ? &gap[i] : NULL);
    if (rtol > 0 && oracle_nrm2(n, r) <= rtol * bnorm) { status = 1; break; }
    if (ttol > 0 && want_log(i, log_every) && tru && tru[i] <= ttol * bnorm) { status = 1; break; }
    if (i >= maxit) break;
    if (gamma == 0.0) { status = 1; break; }
    oracle_apply(A, p, s);                          /* s_i := A p_i */
    const double sp = oracle_dot(n, s, p);
    if (!(sp > 0.0) || !isfinite(sp)) { status = 2; break; }
    const double a = gamma / sp;                    /* alpha_i := (r_i,u_i)/(s_i,p_i) */
    if (alpha) alpha[i] = a;
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) x[j] = x[j] + a * p[j];
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) r[j] = r[j] - a * s[j];
    apply_minv(n, minv, r, u);
    const double gamma_new = oracle_dot(n, r, u);
    const double bt = gamma_new / gamma;            /* beta_{i+1} */
    if (beta) beta[i + 1] = bt;
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) p[j] = u[j] + bt * p[j];
    gamma = gamma_new;
  }
  if (log_every > 0 && !want_log(i, log_every))   /* the final iterate is always logged */
    log_true(A, b, x, r, work, tru ? &tru[i] : NULL, gap ? &gap[i] : NULL);
  if (info) { info->iters = i; info->status = status; }
  free(r); free(u); free(p); free(s); free(work);
  return 0;
}

/* ---- Algorithm 3: shifted pipelined CG (Algorithm 2 when sigma == 0) ------ */

/* ||A a - sigma c - d||_2 (c may be NULL: no shift term); work holds A a afterwards. */
static double gap_norm(const oracle_op *A, const double *a, double sigma, const double *c, const double *d,
                       double *work) {
  const int64_t n = A->n;
  oracle_apply(A, a, work);
  double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (int64_t j = 0; j < n; ++j) {
    const double e = (c ? work[j] - sigma * c[j] : work[j]) - d[j];
    s += e * e;
  }
  return sqrt(s);
}

/* Algorithm 3.  gg, hh, jj (optional, maxit+1 entries): the norms of the gaps of Section
   3.1 at the logged iterations (NaN elsewhere):
     hh[i] = ||(A u_i - sigma r_i) - w_i||   (at the start of iteration i),
     gg[i] = ||(A p_i - sigma t_i) - s_i||   (after p_i, t_i, s_i are formed),
     jj[i] = ||A q_i - z_i||                 (after q_i, z_i are formed);
   the final iterate logs hh only. */
int oracle_pcg_sh(const oracle_op *A, const double *minv, const double *b, double *x, double sigma, int32_t maxit,
                  double rtol, double ttol, int32_t log_every, double *alpha, double *beta, double *rec, double *tru,
                  double *gap, double *gamma_h, double *delta_h, oracle_info *info, oracle_state *state,
                  double *gg, double *hh, double *jj) {
  const int64_t n = A->n;
  double *r = zeros(n), *u = zeros(n), *w = zeros(n), *m = zeros(n), *nn = zeros(n), *z = zeros(n), *q = zeros(n),
         *s = zeros(n), *t = zeros(n), *p = zeros(n), *work = zeros(n);
  if (!r || !u || !w || !m || !nn || !z || !q || !s || !t || !p || !work) return -1;
  fill_nan(alpha, maxit + 1); fill_nan(beta, maxit + 1); fill_nan(rec, maxit + 1);
  fill_nan(tru, maxit + 1); fill_nan(gap, maxit + 1); fill_nan(gamma_h, maxit + 1); fill_nan(delta_h, maxit + 1);
  fill_nan(gg, maxit + 1); fill_nan(hh, maxit + 1); fill_nan(jj, maxit + 1);
  const double bnorm = oracle_nrm2(n, b);

  /* r_0 := b - A x_0; u_0 := M^{-1} r_0; w_0 := A u_0 - sigma r_0 */
  oracle_apply(A, x, work);
  #pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j) r[j] = b[j] - work[j];
  apply_minv(n, minv, r, u);
  oracle_apply(A, u, work);
  #pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j) w[j] = work[j] - sigma * r[j];

  double gamma_prev = 0.0, alpha_prev = 0.0;
  int32_t i = 0, status = 0;
  for (;; ++i) {
    if (rec) rec[i] = oracle_nrm2(n, r);
    if (want_log(i, log_every)) log_true(A, b, x, r, work, tru ? &tru[i] : NULL, gap ? &gap[i] : NULL);
    if (hh && want_log(i, log_every)) hh[i] = gap_norm(A, u, sigma, r, w, work);
    if (rtol > 0 && oracle_nrm2(n, r) <= rtol * bnorm) { status = 1; break; }
    if (ttol > 0 && want_log(i, log_every) && tru && tru[i] <= ttol * bnorm) { status = 1; break; }
    if (i >= maxit) break;

    const double gamma = oracle_dot(n, r, u);       /* gamma_i := (r_i, u_i) */
    double delta = 0.0;                             /* delta := (w_i + sigma r_i, u_i) */
#pragma omp parallel for reduction(+ : delta) schedule(static)
    for (int64_t j = 0; j < n; ++j) delta += (w[j] + sigma * r[j]) * u[j];
    if (gamma_h) gamma_h[i] = gamma;
    if (delta_h) delta_h[i] = delta;
    if (gamma == 0.0) { status = 1; break; }
    apply_minv(n, minv, w, m);                      /* m_i := M^{-1} w_i */
    oracle_apply(A, m, nn);                         /* n_i := A m_i */
    double a, bt;
    if (i > 0) {
      bt = gamma / gamma_prev;                      /* beta_i := gamma_i / gamma_{i-1} */
      const double den = delta / gamma - bt / alpha_prev;
      if (!(den > 0.0) || !isfinite(den)) { status = 2; break; }
      a = 1.0 / den;                                /* alpha_i := (delta/gamma_i - beta_i/alpha_{i-1})^{-1} */
    } else {
      if (!(delta > 0.0) || !isfinite(delta)) { status = 2; break; }
      bt = 0.0;
      a = gamma / delta;                            /* alpha_0 := gamma_0 / delta */
    }
    if (alpha) alpha[i] = a;
    if (beta) beta[i] = bt;
    const double as = a * sigma;
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) z[j] = nn[j] + bt * z[j];   /* z_i */
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) q[j] = m[j] + bt * q[j];    /* q_i */
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) s[j] = w[j] + bt * s[j];    /* s_i */
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) t[j] = r[j] + bt * t[j];    /* t_i */
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) p[j] = u[j] + bt * p[j];    /* p_i */
    if (gg && want_log(i, log_every)) gg[i] = gap_norm(A, p, sigma, t, s, work);
    if (jj && want_log(i, log_every)) jj[i] = gap_norm(A, q, 0.0, NULL, z, work);
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) x[j] = x[j] + a * p[j];     /* x_{i+1} */
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) r[j] = r[j] - (a * s[j] + as * t[j]);   /* r_{i+1} */
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) u[j] = u[j] - (a * q[j] + as * p[j]);   /* u_{i+1} */
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) w[j] = w[j] - a * z[j];     /* w_{i+1} */
    gamma_prev = gamma;
    alpha_prev = a;
  }
  if (log_every > 0 && !want_log(i, log_every)) {   /* the final iterate is always logged */
    log_true(A, b, x, r, work, tru ? &tru[i] : NULL, gap ? &gap[i] : NULL);
    if (hh) hh[i] = gap_norm(A, u, sigma, r, w, work);
  }
  if (info) { info->iters = i; info->status = status; }
  if (state) {
    const size_t bytes = (size_t)n * sizeof(double);
    if (state->x) memcpy(state->x, x, bytes);
    if (state->r) memcpy(state->r, r, bytes);
    if (state->u) memcpy(state->u, u, bytes);
    if (state->w) memcpy(state->w, w, bytes);
    if (state->z) memcpy(state->z, z, bytes);
    if (state->q) memcpy(state->q, q, bytes);
    if (state->s) memcpy(state->s, s, bytes);
    if (state->t) memcpy(state->t, t, bytes);
    if (state->p) memcpy(state->p, p, bytes);
  }
  free(r); free(u); free(w); free(m); free(nn); free(z); free(q); free(s); free(t); free(p); free(work);
  return 0;
}

/* ---- Algorithm 2 written out on its own (no shift terms at all) ---------- */

int oracle_pcg(const oracle_op *A, const double *minv, const double *b, double *x, int32_t maxit, int32_t log_every,
               double *alpha, double *beta, double *rec, double *tru, double *gap, oracle_info *info) {
  const int64_t n = A->n;
  double *r = zeros(n), *u = zeros(n), *w = zeros(n), *m = zeros(n), *nn = zeros(n), *z = zeros(n), *q = zeros(n),
         *s = zeros(n), *t = zeros(n), *p = zeros(n), *work = zeros(n);
  if (!r || !u || !w || !m || !nn || !z || !q || !s || !t || !p || !work) return -1;
  fill_nan(alpha, maxit + 1); fill_nan(beta, maxit + 1); fill_nan(rec, maxit + 1);
  fill_nan(tru, maxit + 1); fill_nan(gap, maxit + 1);

  oracle_apply(A, x, work);                         /* r_0 := b - A x_0 */
  #pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j) r[j] = b[j] - work[j];
  apply_minv(n, minv, r, u);                        /* u_0 := M^{-1} r_0 */
  oracle_apply(A, u, w);                            /* w_0 := A u_0 */
  double gamma_prev = 0.0, alpha_prev = 0.0;
  int32_t i = 0, status = 0;
  for (;; ++i) {
    if (rec) rec[i] = oracle_nrm2(n, r);
    if (want_log(i, log_every)) log_true(A, b, x, r, work, tru ? &tru[i] : NULL, gap ? &gap[i] : NULL);
    if (i >= maxit) break;
    const double gamma = oracle_dot(n, r, u);       /* gamma_i := (r_i, u_i) */
    const double delta = oracle_dot(n, w, u);       /* delta := (w_i, u_i) */
    if (gamma == 0.0) { status = 1; break; }
    apply_minv(n, minv, w, m);                      /* m_i := M^{-1} w_i */
    oracle_apply(A, m, nn);                         /* n_i := A m_i */
    double a, bt;
    if (i > 0) {
      bt = gamma / gamma_prev;
      const double den = delta / gamma - bt / alpha_prev;
      if (!(den > 0.0) || !isfinite(den)) { status = 2; break; }
      a = 1.0 / den;
    } else {
      if (!(delta > 0.0) || !isfinite(delta)) { status = 2; break; }
      bt = 0.0;
      a = gamma / delta;
    }
    if (alpha) alpha[i] = a;
    if (beta) beta[i] = bt;
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) z[j] = nn[j] + bt * z[j];
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) q[j] = m[j] + bt * q[j];
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) s[j] = w[j] + bt * s[j];
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) t[j] = r[j] + bt * t[j];
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) p[j] = u[j] + bt * p[j];
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) x[j] = x[j] + a * p[j];
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) r[j] = r[j] - a * s[j];
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) u[j] = u[j] - a * q[j];
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) w[j] = w[j] - a * z[j];
    gamma_prev = gamma;
    alpha_prev = a;
  }
  if (log_every > 0 && !want_log(i, log_every))   /* the final iterate is always logged */
    log_true(A, b, x, r, work, tru ? &tru[i] : NULL, gap ? &gap[i] : NULL);
  if (info) { info->iters = i; info->status = status; }
  free(r); free(u); free(w); free(m); free(nn); free(z); free(q); free(s); free(t); free(p); free(work);
  return 0;
}

/* ---- Algorithm 4: pipelined CG with a variable shift -------------------- */

/* shifts[0] = sigma_{-1}, shifts[k + 1] = sigma_k (maxit + 1 entries).  The
   correction terms follow the algorithm statement of Section 4.1 (z_i uses
   s_i + sigma_i t_i; the garbled sign in the error analysis of Section 4.2 does
   not concern the algorithm).  Same logging and stop rules as oracle_pcg_sh. */
int oracle_pcg_varsh(const oracle_op *A, const double *minv, const double *b, double *x, const double *shifts,
                     int32_t maxit, double rtol, int32_t log_every, double *alpha, double *beta, double *rec,
                     double *tru, double *gap, oracle_info *info) {
  const int64_t n = A->n;
  double *r = zeros(n), *u = zeros(n), *w = zeros(n), *m = zeros(n), *nn = zeros(n), *z = zeros(n), *q = zeros(n),
         *s = zeros(n), *t = zeros(n), *p = zeros(n), *work = zeros(n);
  if (!r || !u || !w || !m || !nn || !z || !q || !s || !t || !p || !work) return -1;
  fill_nan(alpha, maxit + 1); fill_nan(beta, maxit + 1); fill_nan(rec, maxit + 1);
  fill_nan(tru, maxit + 1); fill_nan(gap, maxit + 1);
  const double bnorm = oracle_nrm2(n, b);

  /* r_0 := b - A x_0; u_0 := M^{-1} r_0; w_0 := A u_0 - sigma_{-1} r_0 */
  oracle_apply(A, x, work);
  #pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j) r[j] = b[j] - work[j];
  apply_minv(n, minv, r, u);
  oracle_apply(A, u, work);
  #pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; ++j) w[j] = work[j] - shifts[0] * r[j];

  double gamma_prev = 0.0, alpha_prev = 0.0;
  int32_t i = 0, status = 0;
  for (;; ++i) {
    if (rec) rec[i] = oracle_nrm2(n, r);
    if (want_log(i, log_every)) log_true(A, b, x, r, work, tru ? &tru[i] : NULL, gap ? &gap[i] : NULL);
    if (rtol > 0 && oracle_nrm2(n, r) <= rtol * bnorm) { status = 1; break; }
    if (i >= maxit) break;
    const double sprev = shifts[i], scur = shifts[i + 1];   /* sigma_{i-1}, sigma_i */
    const double ds = scur - sprev;
    const double gamma = oracle_dot(n, r, u);        /* gamma_i := (r_i, u_i) */
    double delta = 0.0;                              /* delta := (w_i + sigma_{i-1} r_i, u_i) */
#pragma omp parallel for reduction(+ : delta) schedule(static)
    for (int64_t j = 0; j < n; ++j) delta += (w[j] + sprev * r[j]) * u[j];
    if (gamma == 0.0) { status = 1; break; }
    apply_minv(n, minv, w, m);                       /* m_i := M^{-1} w_i */
    oracle_apply(A, m, nn);                          /* n_i := A m_i */
    double a, bt;
    if (i > 0) {
      bt = gamma / gamma_prev;
      const double den = delta / gamma - bt / alpha_prev;
      if (!(den > 0.0) || !isfinite(den)) { status = 2; break; }
      a = 1.0 / den;
    } else {
      if (!(delta > 0.0) || !isfinite(delta)) { status = 2; break; }
      bt = 0.0;
      a = gamma / delta;
    }
    if (alpha) alpha[i] = a;
    if (beta) beta[i] = bt;
    const double as = a * scur;
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) t[j] = r[j] + bt * t[j];                    /* t_i */
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) p[j] = u[j] + bt * p[j];                    /* p_i */
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) s[j] = (w[j] + bt * s[j]) - ds * t[j];      /* s_i */
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) q[j] = (m[j] + bt * q[j]) - ds * p[j];      /* q_i */
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) z[j] = (nn[j] + bt * z[j]) - ds * (s[j] + scur * t[j]);   /* z_i */
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) x[j] = x[j] + a * p[j];                     /* x_{i+1} */
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) w[j] = (w[j] - a * z[j]) - ds * r[j];       /* w_{i+1} (before r) */
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) r[j] = r[j] - (a * s[j] + as * t[j]);       /* r_{i+1} */
    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) u[j] = u[j] - (a * q[j] + as * p[j]);       /* u_{i+1} */
    gamma_prev = gamma;
    alpha_prev = a;
  }
  if (log_every > 0 && !want_log(i, log_every))
    log_true(A, b, x, r, work, tru ? &tru[i] : NULL, gap ? &gap[i] : NULL);
  if (info) { info->iters = i; info->status = status; }
  free(r); free(u); free(w); free(m); free(nn); free(z); free(q); free(s); free(t); free(p); free(work);
  return 0;
}
