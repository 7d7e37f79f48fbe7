/*
 * pa_oracle.c -- plain, serial, FP64 reference of the Projected Adam estimator
 * of the L2 condition number (the paper's section "Computing the condition
 * number of a matrix": Eq. nabla_loss, Algorithm 1 "Projected Adam Optimizer").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this code:
 * only the test suite, the package smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no source, header or helper with the CUDA
 * library; it is compiled with -O2 -ffp-contract=off so every operation is
 * rounded as written (no fused multiply-add), and every sum runs sequentially
 * from the first index to the last.
 *
 * Contents
 *   po_splitmix64_at      SplitMix64 output i of a seed (Steele, Lea & Flood,
 *                         "Fast splittable pseudorandom number generators",
 *                         OOPSLA 2014), used for the start vector x_init.
 *   po_start_vector       x_init: x_i = 2 u_i - 1 from SplitMix64, then x/||x||.
 *   po_spmv               y = A x, row by row in CSR order.
 *   po_spmv_t             z = A^T y by scattering each row of A (never forms A^T).
 *   po_spmv_dd/_t_dd      the same products with compensated (double-double)
 *                         accumulation: TwoProduct (Dekker 1971, via Veltkamp
 *                         splitting, no FMA) and TwoSum (Knuth), the "Dot2"
 *                         scheme of Ogita, Rump & Oishi (SISC 2005).
 *   po_projected_adam     Algorithm 1 with the gradient of Eq. nabla_loss.
 *   po_equilibrate_pow2   row then column 2-norm scaling (the paper's "Row and
 *                         Column Scaling" subsection), each factor rounded to the
 *                         nearest power of two.
 *   po_error_bounds       the residual of an approximate solution (Dot2) and
 *                         the error bounds of the paper's Theorems 1-4.
 *   po_projected_adam_lu  Algorithm 1 on A^{-1} with the gradient of Algorithm 2
 *                         (triangular solves with given L, U factors):
 *                         sigma_min(A) = 1 / ||A^{-1}||_2.
 *
 * Timing build: compiled with -fopenmp (oracle.build(openmp=True)), the
 * "#pragma omp" lines below run the row loops and the element loops on all
 * host cores and reduce the sums (dot products, the transposed scatter) per
 * thread.  That changes the summation order, so the OpenMP build only times
 * the oracle on many cores; the checker is always the serial build, where
 * the pragmas are ignored.
 *
 * Readings where the paper is silent (all stated again in the design notes):
 *   - sigma_min: minimise L(x) = log||Ax|| - log||x|| on the sphere with the
 *     same Algorithm 1 (the negated loss of Eq. nabla_loss), not the LU route
 *     of Algorithm 2.
 *   - loss = quadratic: L = -||Ax||^2 (sigma_max) or +||Ax||^2 (sigma_min),
 *     gradient -2 A^T A x or +2 A^T A x.
 *   - Algorithm 1 scores L(x) right after normalising x in iteration t; that x
 *     is the one the next iteration differentiates, so the oracle computes
 *     y = A x once and uses it for both (the same numbers Algorithm 1 would
 *     compute twice).  After the last iteration one more product scores x_T.
 *     x_init itself is never scored, L_min starts at +inf, and "<" is strict.
 *   - ||Ax|| == 0 stops the run with status PO_SINGULAR; a NaN or Inf in a
 *     reduction stops it with status PO_NONFINITE.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PO_OK 0
#define PO_SINGULAR 1
#define PO_NONFINITE (-4)
#define PO_BADARG (-1)

#define PO_SIGMA_MAX 1
#define PO_SIGMA_MIN 2
#define PO_LOSS_LOGRATIO 0
#define PO_LOSS_QUADRATIC 1

#define PO_FLAG_DD 1          /* compensated products for y and z */
#define PO_FLAG_NO_TANGENT 2  /* ablation: drop the tangent projection   */
#define PO_FLAG_NO_NORMALISE 4 /* ablation: drop the re-normalisation    */

/* ---------------------------------------------------------------- RNG --- */

static uint64_t po_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Output number i (0-based) of the SplitMix64 generator started at `seed`:
 * the state advances by the golden gamma before each output. */
uint64_t po_splitmix64_at(uint64_t seed, uint64_t i) {
  return po_mix64(seed + (i + 1) * 0x9E3779B97F4A7C15ull);
}

/* Start vector: x_i = 2*u_i - 1 with u_i = (out_i >> 11) * 2^-53, then x/||x||. */
void po_start_vector(int64_t n, uint64_t seed, double* x) {
  for (int64_t i = 0; i < n; ++i) {
    double u = (double)(po_splitmix64_at(seed, (uint64_t)i) >> 11) * 0x1.0p-53;
    x[i] = 2.0 * u - 1.0;
  }
  double q = 0.0;
  for (int64_t i = 0; i < n; ++i) q = q + x[i] * x[i];
  double nrm = sqrt(q);
  for (int64_t i = 0; i < n; ++i) x[i] = x[i] / nrm;
}

/* ------------------------------------------------------------ products --- */

void po_spmv(int32_t n_rows, const int32_t* row_ptr, const int32_t* col, const double* val,
             const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int32_t i = 0; i < n_rows; ++i) {
    double acc = 0.0;
    for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) acc = acc + val[k] * x[col[k]];
    y[i] = acc;
  }
}

/* z = A^T y as a scatter over the rows of A: contributions to z_j arrive in
 * increasing row order i. */
void po_spmv_t(int32_t n_rows, int32_t n_cols, const int32_t* row_ptr, const int32_t* col,
               const double* val, const double* y, double* z) {
  for (int32_t j = 0; j < n_cols; ++j) z[j] = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : z[:n_cols])
  for (int32_t i = 0; i < n_rows; ++i)
    for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) z[col[k]] = z[col[k]] + val[k] * y[i];
}

/* Error-free transformations (no FMA: products split a la Veltkamp/Dekker). */
static void two_sum(double a, double b, double* s, double* e) {
  double x = a + b;
  double z = x - a;
  *e = (a - (x - z)) + (b - z);
  *s = x;
}
static void split(double a, double* hi, double* lo) {
  double c = 134217729.0 * a; /* 2^27 + 1 */
  double h = c - (c - a);
  *hi = h;
  *lo = a - h;
}
static void two_prod(double a, double b, double* p, double* e) {
  double x = a * b, ah, al, bh, bl;
  split(a, &ah, &al);
  split(b, &bh, &bl);
  *e = al * bl - (((x - ah * bh) - al * bh) - ah * bl);
  *p = x;
}

/* y = A x in Dot2 accumulation; returns the unevaluated sum y_hi + y_lo with
 * y_hi = fl(y_hi + y_lo) (normalised by one final TwoSum). */
void po_spmv_dd(int32_t n_rows, const int32_t* row_ptr, const int32_t* col, const double* val,
                const double* x, double* y_hi, double* y_lo) {
  for (int32_t i = 0; i < n_rows; ++i) {
    double s = 0.0, c = 0.0;
    for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
      double p, pe, t, te;
      two_prod(val[k], x[col[k]], &p, &pe);
      two_sum(s, p, &t, &te);
      s = t;
      c = c + (te + pe);
    }
    double h, l;
    two_sum(s, c, &h, &l);
    y_hi[i] = h;
    y_lo[i] = l;
  }
}

/* z = A^T (y_hi + y_lo) with Dot2 accumulation per column, rounded to double.
 * Scatter order: rows of A in increasing order, hi term before lo term. */
void po_spmv_t_dd(int32_t n_rows, int32_t n_cols, const int32_t* row_ptr, const int32_t* col,
                  const double* val, const double* y_hi, const double* y_lo, double* z) {
  double* s = (double*)calloc((size_t)n_cols, sizeof(double));
  double* c = (double*)calloc((size_t)n_cols, sizeof(double));
  for (int32_t i = 0; i < n_rows; ++i) {
    for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
      int32_t j = col[k];
      double p, pe, t, te;
      two_prod(val[k], y_hi[i], &p, &pe);
      two_sum(s[j], p, &t, &te);
      s[j] = t;
      c[j] = c[j] + (te + pe);
      two_prod(val[k], y_lo[i], &p, &pe);
      two_sum(s[j], p, &t, &te);
      s[j] = t;
      c[j] = c[j] + (te + pe);
    }
  }
  for (int32_t j = 0; j < n_cols; ++j) z[j] = s[j] + c[j];
  free(s);
  free(c);
}

static double po_dot(int64_t n, const double* a, const double* b) {
  double acc = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : acc)
  for (int64_t i = 0; i < n; ++i) acc = acc + a[i] * b[i];
  return acc;
}

/* Loss of Algorithm 1 from s = ||Ax||^2 and q = ||x||^2. */
static double po_loss(int mode, int loss, double s, double q) {
  if (loss == PO_LOSS_QUADRATIC) return mode == PO_SIGMA_MAX ? -s : s;
  double lx = log(sqrt(q)), lax = log(sqrt(s));
  return mode == PO_SIGMA_MAX ? lx - lax : lax - lx;
}

/* Gradient of the loss (Eq. nabla_loss) from x, z = A^T A x, s = ||Ax||^2 and
 * q = ||x||^2; negated for sigma_min.  Quadratic reading: -2z / +2z. */
static void po_grad_from(int mode, int loss, int64_t n, const double* x, const double* z,
                         double s, double q, double* g) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double gi;
    if (loss == PO_LOSS_LOGRATIO)
      gi = x[i] / q - z[i] / s;
    else
      gi = -2.0 * z[i];
    g[i] = (mode == PO_SIGMA_MAX) ? gi : -gi;
  }
}

/* L(x) and grad L(x) from scratch (one product each way); returns L. */
double po_loss_grad(int32_t n_rows, int32_t n_cols, const int32_t* row_ptr, const int32_t* col,
                    const double* val, int mode, int loss, const double* x, double* g) {
  double* y = (double*)malloc(sizeof(double) * (n_rows > 0 ? n_rows : 1));
  double* z = (double*)malloc(sizeof(double) * n_cols);
  po_spmv(n_rows, row_ptr, col, val, x, y);
  double s = po_dot(n_rows, y, y);
  double q = po_dot(n_cols, x, x);
  po_spmv_t(n_rows, n_cols, row_ptr, col, val, y, z);
  if (g) po_grad_from(mode, loss, n_cols, x, z, s, q, g);
  free(y);
  free(z);
  return po_loss(mode, loss, s, q);
}

/* ------------------------------------------------------- Algorithm 1 ----- */
/*
 * Runs `iters` iterations of Projected Adam from x_init (n_cols entries).
 * Outputs (any may be NULL):
 *   x_min[n_cols]    the tracked minimiser (Algorithm 1's return value)
 *   x_last[n_cols]   x after the last iteration
 *   out[4]           {L_min, t_min (iteration whose x is x_min, 0 = x_init),
 *                     L(x_T), iterations actually run}
 *   L_trace[iters]   L(x_t) for t = 1..iters (NaN after an early stop)
 *   x_trace[n_trace][n_cols]  x_t for t = 1..n_trace
 * Returns PO_OK, PO_SINGULAR or PO_NONFINITE.
 */
int po_projected_adam(int32_t n_rows, int32_t n_cols, const int32_t* row_ptr, const int32_t* col,
                      const double* val, int mode, int loss, int64_t iters, double lr,
                      double beta1, double beta2, double eps, const double* x_init, int flags,
                      double* x_min, double* x_last, double* out, double* L_trace,
                      double* x_trace, int64_t n_trace) {
  if ((mode != PO_SIGMA_MAX && mode != PO_SIGMA_MIN) ||
      (loss != PO_LOSS_LOGRATIO && loss != PO_LOSS_QUADRATIC) || iters < 0 || n_cols <= 0)
    return PO_BADARG;
  const int64_t n = n_cols;
  double* x = (double*)malloc(sizeof(double) * n);
  double* xm = (double*)malloc(sizeof(double) * n);
  double* m = (double*)calloc(n, sizeof(double));
  double* v = (double*)calloc(n, sizeof(double));
  double* g = (double*)malloc(sizeof(double) * n);
  double* dx = (double*)malloc(sizeof(double) * n);
  double* z = (double*)malloc(sizeof(double) * n);
  double* y = (double*)malloc(sizeof(double) * (n_rows > 0 ? n_rows : 1));
  double* ylo = (double*)malloc(sizeof(double) * (n_rows > 0 ? n_rows : 1));
  memcpy(x, x_init, sizeof(double) * n);
  memcpy(xm, x_init, sizeof(double) * n); /* x_min <- x_init            */
  double L_min = INFINITY;                /* L_min <- infinity          */
  int64_t t_min = 0, t_done = 0;
  double L_last = NAN;
  int status = PO_OK;
  if (L_trace)
    for (int64_t t = 0; t < iters; ++t) L_trace[t] = NAN;

  for (int64_t t = 1; t <= iters + 1; ++t) {
    /* y = A x for the current x; it scores x (if t > 1) and feeds the gradient. */
    if (flags & PO_FLAG_DD)
      po_spmv_dd(n_rows, row_ptr, col, val, x, y, ylo);
    else
      po_spmv(n_rows, row_ptr, col, val, x, y);
    double s = po_dot(n_rows, y, y);
    double q = po_dot(n, x, x);
    if (!isfinite(s) || !isfinite(q)) { status = PO_NONFINITE; break; }
    if (t > 1) {
      double L = po_loss(mode, loss, s, q);
      L_last = L;
      if (L_trace) L_trace[t - 2] = L;
      if (L < L_min) { /* if L(x) < L_min: L_min <- L(x); x_min <- x */
        L_min = L;
        t_min = t - 1;
        memcpy(xm, x, sizeof(double) * n);
      }
    }
    if (s == 0.0) {
      /* A x = 0: x is a null vector and the gradient is undefined.  For
       * sigma_min it is the minimiser (scored above when t > 1; x_init when
       * t == 1); for sigma_max the best iterate so far stands. */
      if (mode == PO_SIGMA_MIN && t == 1) {
        L_min = po_loss(mode, loss, s, q);
        t_min = 0;
        memcpy(xm, x, sizeof(double) * n);
      }
      status = PO_SINGULAR;
      break;
    }
    if (t == iters + 1) break;

    /* g <- grad L(x)  (Eq. nabla_loss, negated for sigma_min) */
    if (flags & PO_FLAG_DD)
      po_spmv_t_dd(n_rows, n_cols, row_ptr, col, val, y, ylo, z);
    else
      po_spmv_t(n_rows, n_cols, row_ptr, col, val, y, z);
    po_grad_from(mode, loss, n, x, z, s, q, g);
    /* biased moments, bias correction, update */
    double bc1 = 1.0 - pow(beta1, (double)t);
    double bc2 = 1.0 - pow(beta2, (double)t);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
      v[i] = beta2 * v[i] + (1.0 - beta2) * (g[i] * g[i]);
      double mh = m[i] / bc1;
      double vh = v[i] / bc2;
      dx[i] = lr * mh / (sqrt(vh) + eps);
    }
    /* project the update onto the tangent space of the sphere at x */
    if (!(flags & PO_FLAG_NO_TANGENT)) {
      double c = po_dot(n, x, dx);
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; ++i) dx[i] = dx[i] - c * x[i];
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) x[i] = x[i] - dx[i];
    /* back onto the unit sphere */
    if (!(flags & PO_FLAG_NO_NORMALISE)) {
      double nrm = sqrt(po_dot(n, x, x));
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; ++i) x[i] = x[i] / nrm;
    }
    t_done = t;
    if (x_trace && t <= n_trace) memcpy(x_trace + (t - 1) * n, x, sizeof(double) * n);
  }

  if (x_min) memcpy(x_min, xm, sizeof(double) * n);
  if (x_last) memcpy(x_last, x, sizeof(double) * n);
  if (out) {
    out[0] = L_min;
    out[1] = (double)t_min;
    out[2] = L_last;
    out[3] = (double)t_done;
  }
  free(x); free(xm); free(m); free(v); free(g); free(dx); free(z); free(y); free(ylo);
  return status;
}

/* sigma = ||A x|| / ||x||, the operator-norm quotient of Eq. max_sup_equivalence,
 * with plain (flags = 0) or compensated (PO_FLAG_DD) products. */
double po_sigma(int32_t n_rows, int32_t n_cols, const int32_t* row_ptr, const int32_t* col,
                const double* val, const double* x, int flags) {
  double* y = (double*)malloc(sizeof(double) * (n_rows > 0 ? n_rows : 1));
  double* ylo = (double*)malloc(sizeof(double) * (n_rows > 0 ? n_rows : 1));
  if (flags & PO_FLAG_DD)
    po_spmv_dd(n_rows, row_ptr, col, val, x, y, ylo);
  else
    po_spmv(n_rows, row_ptr, col, val, x, y);
  double s = po_dot(n_rows, y, y);
  double q = po_dot(n_cols, x, x);
  free(y);
  free(ylo);
  return sqrt(s) / sqrt(q);
}

/* ---------------------------------------------------- equilibration ----- */

/* Nearest power of two to a positive finite r: r = f * 2^e with f in [0.5, 1);
 * 2^e when f >= sqrt(1/2), else 2^(e-1).  Zero rows/columns get 1. */
static double po_nearest_pow2(double r) {
  if (!(r > 0.0) || !isfinite(r)) return 1.0;
  int e;
  double f = frexp(r, &e);
  return f >= 0.70710678118654752440 ? ldexp(1.0, e) : ldexp(1.0, e - 1);
}

/* D_row = nearest-pow2 of the row 2-norms of A; D_col = nearest-pow2 of the
 * column 2-norms of D_row^-1 A; val_hat = entries of D_row^-1 A D_col^-1.
 * Powers of two make every scaling exact. */
void po_equilibrate_pow2(int32_t n_rows, int32_t n_cols, const int32_t* row_ptr,
                         const int32_t* col, const double* val, double* d_row, double* d_col,
                         double* val_hat) {
  for (int32_t i = 0; i < n_rows; ++i) {
    double s = 0.0;
    for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) s = s + val[k] * val[k];
    d_row[i] = po_nearest_pow2(sqrt(s));
  }
  double* cs = (double*)calloc((size_t)n_cols, sizeof(double));
  for (int32_t i = 0; i < n_rows; ++i)
    for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
      double a = val[k] / d_row[i];
      cs[col[k]] = cs[col[k]] + a * a;
    }
  for (int32_t j = 0; j < n_cols; ++j) d_col[j] = po_nearest_pow2(sqrt(cs[j]));
  for (int32_t i = 0; i < n_rows; ++i)
    for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
      val_hat[k] = val[k] / d_row[i] / d_col[col[k]];
  free(cs);
}

/* The paper's error analysis ("Error estimates and conditioning"): the
 * residual of an approximate solution x_hat of A x = b and the bounds of its
 * Theorems 1-4, given kappa = kappa_2(A) and norm_a = ||A||_2.
 *
 * r_i = sum_k a_ik x_hat_k - b_i, accumulated in Dot2 (the row's products in
 * CSR order, then -b_i as one more term, then s + c), so a residual near the
 * rounding level of A x_hat is not lost to cancellation.
 *
 * out[0] ||r||          out[1] ||b||          out[2] ||x_hat||
 * out[3] Theorem 1 lower bound of ||x_hat - x|| / ||x||:  (||r|| / ||b||) / kappa
 * out[4] Theorem 1 upper bound:                            kappa ||r|| / ||b||
 * out[5] Theorem 2 lower bound of ||x_hat - x|| / ||x_hat||: ||r|| / (||A|| ||x_hat||)
 * out[6] Theorem 2 upper bound eps:               kappa ||r|| / (||A|| ||x_hat||)
 * out[7] Theorem 3 bound of ||x_hat - x|| / ||x||: eps / (1 - eps), +inf if eps >= 1
 * out[8] Theorem 4 rounding bound 2 u kappa / (1 - kappa u), +inf if kappa u >= 1
 * out[9] 1 when kappa u >= 1 (numerically singular at precision u), else 0 */
void po_error_bounds(int32_t n_rows, int32_t n_cols, const int32_t* row_ptr, const int32_t* col,
                     const double* val, const double* x_hat, const double* b, double kappa,
                     double norm_a, double u, double* out) {
  double rr = 0.0, bb = 0.0, xx = 0.0;
  for (int32_t i = 0; i < n_rows; ++i) {
    double s = 0.0, c = 0.0, t, te;
    for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
      double p, pe;
      two_prod(val[k], x_hat[col[k]], &p, &pe);
      two_sum(s, p, &t, &te);
      s = t;
      c = c + (te + pe);
    }
    two_sum(s, -b[i], &t, &te);
    s = t;
    c = c + te;
    double r = s + c;
    rr = rr + r * r;
    bb = bb + b[i] * b[i];
  }
  for (int32_t j = 0; j < n_cols; ++j) xx = xx + x_hat[j] * x_hat[j];
  double nr = sqrt(rr), nb = sqrt(bb), nx = sqrt(xx);
  out[0] = nr;
  out[1] = nb;
  out[2] = nx;
  out[3] = (nr / nb) / kappa;
  out[4] = kappa * (nr / nb);
  out[5] = nr / (norm_a * nx);
  double eps = kappa * (nr / (norm_a * nx));
  out[6] = eps;
  out[7] = eps < 1.0 ? eps / (1.0 - eps) : INFINITY;
  double ku = kappa * u;
  out[8] = ku < 1.0 ? 2.0 * u * kappa / (1.0 - ku) : INFINITY;
  out[9] = ku >= 1.0 ? 1.0 : 0.0;
}

/* ------------------------------------------------ Algorithm 2 (LU route) --- */
/*
 * sigma_min(A) = 1 / ||A^{-1}||_2, with ||A^{-1}||_2 found by Algorithm 1 on
 * the operator B = A^{-1}, whose gradient Algorithm 2 computes from one LU
 * factorisation: r = A^{-1} x by L U r = x, s = A^{-T} r by U^T L^T s = r,
 * grad L(x) = x / ||x||^2 - s / ||r||^2.
 *
 * Factors: P A Q = L U with L lower and U upper triangular (n x n CSR, each
 * row holding its diagonal entry; L need not be unit), p[i] = the row of A
 * that is row i of P A, q[j] = the column of A that is column j of A Q
 * (NULL = identity).  Then A^{-1} = Q U^{-1} L^{-1} P and
 * A^{-T} = P^T L^{-T} U^{-T} Q^T.
 */

/* L x = b by forward substitution: x_i = (b_i - sum_{j<i} l_ij x_j) / l_ii,
 * the sum in CSR order. */
void po_lower_solve(int32_t n, const int32_t* rp, const int32_t* ci, const double* va,
                    const double* b, double* x) {
  for (int32_t i = 0; i < n; ++i) {
    double acc = 0.0, d = 0.0;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
      if (ci[k] < i) acc = acc + va[k] * x[ci[k]];
      else if (ci[k] == i) d = va[k];
    }
    x[i] = (b[i] - acc) / d;
  }
}

/* U x = b by back substitution: x_i = (b_i - sum_{j>i} u_ij x_j) / u_ii. */
void po_upper_solve(int32_t n, const int32_t* rp, const int32_t* ci, const double* va,
                    const double* b, double* x) {
  for (int32_t i = n - 1; i >= 0; --i) {
    double acc = 0.0, d = 0.0;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
      if (ci[k] > i) acc = acc + va[k] * x[ci[k]];
      else if (ci[k] == i) d = va[k];
    }
    x[i] = (b[i] - acc) / d;
  }
}

/* U^T x = b from the rows of U (column-oriented forward substitution: once
 * x_i is known, row i of U scatters u_ij x_i into the pending sums of the
 * later unknowns j). */
void po_upper_t_solve(int32_t n, const int32_t* rp, const int32_t* ci, const double* va,
                      const double* b, double* x) {
  double* acc = (double*)calloc((size_t)n, sizeof(double));
  for (int32_t i = 0; i < n; ++i) {
    double d = 0.0;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
      if (ci[k] == i) d = va[k];
    x[i] = (b[i] - acc[i]) / d;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
      if (ci[k] > i) acc[ci[k]] = acc[ci[k]] + va[k] * x[i];
  }
  free(acc);
}

/* L^T x = b from the rows of L (column-oriented back substitution). */
void po_lower_t_solve(int32_t n, const int32_t* rp, const int32_t* ci, const double* va,
                      const double* b, double* x) {
  double* acc = (double*)calloc((size_t)n, sizeof(double));
  for (int32_t i = n - 1; i >= 0; --i) {
    double d = 0.0;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
      if (ci[k] == i) d = va[k];
    x[i] = (b[i] - acc[i]) / d;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
      if (ci[k] < i) acc[ci[k]] = acc[ci[k]] + va[k] * x[i];
  }
  free(acc);
}

typedef struct {
  int32_t n;
  const int32_t *l_rp, *l_ci, *u_rp, *u_ci, *p, *q;
  const double *l_va, *u_va;
} po_lu;

/* r = A^{-1} x = Q U^{-1} L^{-1} P x.  Returns u = Q^T r (||u|| = ||r||); r
 * itself goes to r_out when it is not NULL. */
static void po_lu_apply(const po_lu* f, const double* x, double* w, double* t, double* u,
                        double* r_out) {
  const int32_t n = f->n;
  for (int32_t i = 0; i < n; ++i) w[i] = x[f->p ? f->p[i] : i];
  po_lower_solve(n, f->l_rp, f->l_ci, f->l_va, w, t);
  po_upper_solve(n, f->u_rp, f->u_ci, f->u_va, t, u);
  if (r_out)
    for (int32_t j = 0; j < n; ++j) r_out[f->q ? f->q[j] : j] = u[j];
}

/* s = A^{-T} r = P^T L^{-T} U^{-T} (Q^T r), from u = Q^T r. */
static void po_lu_apply_t(const po_lu* f, const double* u, double* a, double* c, double* s) {
  const int32_t n = f->n;
  po_upper_t_solve(n, f->u_rp, f->u_ci, f->u_va, u, a);
  po_lower_t_solve(n, f->l_rp, f->l_ci, f->l_va, a, c);
  for (int32_t i = 0; i < n; ++i) s[f->p ? f->p[i] : i] = c[i];
}

/* r = A^{-1} x and s = A^{-T} A^{-1} x through the factors (test access). */
void po_lu_products(int32_t n, const int32_t* l_rp, const int32_t* l_ci, const double* l_va,
                    const int32_t* u_rp, const int32_t* u_ci, const double* u_va,
                    const int32_t* p, const int32_t* q, const double* x, double* r, double* s) {
  po_lu f = {n, l_rp, l_ci, u_rp, u_ci, p, q, l_va, u_va};
  double* w = (double*)malloc(sizeof(double) * n);
  double* t = (double*)malloc(sizeof(double) * n);
  double* u = (double*)malloc(sizeof(double) * n);
  po_lu_apply(&f, x, w, t, u, r);
  if (s) po_lu_apply_t(&f, u, w, t, s);
  free(w); free(t); free(u);
}

/* Algorithm 1 on B = A^{-1} with the gradient of Algorithm 2.  Arguments and
 * outputs as po_projected_adam (mode sigma_max of B, log-ratio loss,
 * L(x) = log||x|| - log||A^{-1} x||); out[4] = sigma_max(B) = ||B x_min|| /
 * ||x_min||, so sigma_min(A) = 1 / out[4]. */
int po_projected_adam_lu(int32_t n, const int32_t* l_rp, const int32_t* l_ci, const double* l_va,
                         const int32_t* u_rp, const int32_t* u_ci, const double* u_va,
                         const int32_t* p, const int32_t* q, int64_t iters, double lr,
                         double beta1, double beta2, double eps, const double* x_init,
                         double* x_min, double* x_last, double* out, double* L_trace,
                         double* x_trace, int64_t n_trace) {
  if (iters < 0 || n <= 0) return PO_BADARG;
  po_lu f = {n, l_rp, l_ci, u_rp, u_ci, p, q, l_va, u_va};
  double* x = (double*)malloc(sizeof(double) * n);
  double* xm = (double*)malloc(sizeof(double) * n);
  double* m = (double*)calloc(n, sizeof(double));
  double* v = (double*)calloc(n, sizeof(double));
  double* g = (double*)malloc(sizeof(double) * n);
  double* dx = (double*)malloc(sizeof(double) * n);
  double* u = (double*)malloc(sizeof(double) * n);
  double* sv = (double*)malloc(sizeof(double) * n);
  double* w1 = (double*)malloc(sizeof(double) * n);
  double* w2 = (double*)malloc(sizeof(double) * n);
  memcpy(x, x_init, sizeof(double) * n);
  memcpy(xm, x_init, sizeof(double) * n);
  double L_min = INFINITY, L_last = NAN;
  int64_t t_min = 0, t_done = 0;
  int status = PO_OK;
  if (L_trace)
    for (int64_t t = 0; t < iters; ++t) L_trace[t] = NAN;

  for (int64_t t = 1; t <= iters + 1; ++t) {
    /* r = A^{-1} x (Algorithm 2: solve L U r = x) and norm_r */
    po_lu_apply(&f, x, w1, w2, u, NULL);
    double rr = po_dot(n, u, u);
    double q2 = po_dot(n, x, x);
    if (!isfinite(rr) || !isfinite(q2) || rr == 0.0) { status = PO_NONFINITE; break; }
    if (t > 1) {
      double L = log(sqrt(q2)) - log(sqrt(rr));
      L_last = L;
      if (L_trace) L_trace[t - 2] = L;
      if (L < L_min) {
        L_min = L;
        t_min = t - 1;
        memcpy(xm, x, sizeof(double) * n);
      }
    }
    if (t == iters + 1) break;
    /* s = A^{-T} r (solve U^T L^T s = r); grad L = x / ||x||^2 - s / ||r||^2 */
    po_lu_apply_t(&f, u, w1, w2, sv);
    for (int32_t i = 0; i < n; ++i) g[i] = x[i] / q2 - sv[i] / rr;
    double bc1 = 1.0 - pow(beta1, (double)t);
    double bc2 = 1.0 - pow(beta2, (double)t);
    for (int32_t i = 0; i < n; ++i) {
      m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
      v[i] = beta2 * v[i] + (1.0 - beta2) * (g[i] * g[i]);
      double mh = m[i] / bc1;
      double vh = v[i] / bc2;
      dx[i] = lr * mh / (sqrt(vh) + eps);
    }
    double c = po_dot(n, x, dx);
    for (int32_t i = 0; i < n; ++i) dx[i] = dx[i] - c * x[i];
    for (int32_t i = 0; i < n; ++i) x[i] = x[i] - dx[i];
    double nrm = sqrt(po_dot(n, x, x));
    for (int32_t i = 0; i < n; ++i) x[i] = x[i] / nrm;
    t_done = t;
    if (x_trace && t <= n_trace) memcpy(x_trace + (t - 1) * n, x, sizeof(double) * n);
  }

  /* sigma_max(A^{-1}) at the tracked maximiser */
  po_lu_apply(&f, xm, w1, w2, u, NULL);
  double sig = sqrt(po_dot(n, u, u)) / sqrt(po_dot(n, xm, xm));
  if (x_min) memcpy(x_min, xm, sizeof(double) * n);
  if (x_last) memcpy(x_last, x, sizeof(double) * n);
  if (out) {
    out[0] = L_min;
    out[1] = (double)t_min;
    out[2] = L_last;
    out[3] = (double)t_done;
    out[4] = sig;
  }
  free(x); free(xm); free(m); free(v); free(g); free(dx); free(u); free(sv); free(w1); free(w2);
  return status;
}
