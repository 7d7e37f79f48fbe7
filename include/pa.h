/*
 * pa.h -- C ABI of the GB300-native Projected Adam estimator of the L2
 * condition number, kappa_2(A) = ||A||_2 ||A^-1||_2 = sigma_max / sigma_min
 * (paper: section "Computing the condition number of a matrix", the identity
 * kappa_2 = max sigma / min sigma, Theorem "Equivalent definitions of the L2
 * matrix norm" and Eq. max_sup_equivalence, the loss and its gradient
 * Eq. nabla_loss, and Algorithm 1 "Projected Adam Optimizer").
 *
 * One library, one GPU.  Every entry point that computes runs CUDA kernels of
 * this library; there is no CPU fallback.  All work of a handle is enqueued on
 * the CUDA stream given to pa_create (NULL = the legacy default stream); the
 * calls that return numbers to host memory synchronise that stream first.
 *
 * Conventions (all entry points):
 *   - CSR is 0-based: row_ptr[0] = 0, row_ptr non-decreasing,
 *     row_ptr[n_rows] = nnz, 0 <= col_idx[k] < n_cols.  Column indices may be
 *     unsorted and may repeat (repeats add up).  Violations give
 *     PA_ERR_INVALID_CSR.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     device memory of the current device.  Which one a call takes is stated
 *     beside it.  Output pointers documented as "may be NULL" are skipped.
 *   - Statuses < 0 are errors: outputs are left untouched and
 *     pa_last_error() holds a message.  PA_WARN_SINGULAR (> 0) is a result.
 *   - The library copies every input; callers keep ownership of their arrays.
 *   - Handles are not thread-safe: one thread at a time per handle.
 */
#ifndef PA_H
#define PA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pa_ctx* pa_handle; /* opaque; owned by the library */

typedef enum {
  PA_SIGMA_MAX = 1,    /* maximise L: sigma_max = ||A||_2                  */
  PA_SIGMA_MIN = 2,    /* minimise ||Ax||/||x|| on the sphere: sigma_min  */
  PA_BOTH = 3,
  PA_SIGMA_MIN_LU = 4, /* sigma_min = 1 / ||A^{-1}||_2 by Algorithm 1 on
                          A^{-1} with the gradient of Algorithm 2 (needs the
                          factors of pa_attach_lu)                         */
  PA_BOTH_LU = 5       /* PA_SIGMA_MAX + PA_SIGMA_MIN_LU                    */
} pa_mode;

typedef enum {
  PA_OK = 0,
  PA_WARN_SINGULAR = 1,      /* ||A x|| == 0 met: sigma_min = 0, kappa = +inf */
  PA_ERR_INVALID_ARG = -1,
  PA_ERR_INVALID_CSR = -2,
  PA_ERR_NOT_SQUARE = -3,    /* sigma_min needs n_rows >= n_cols            */
  PA_ERR_NONFINITE = -4,     /* a NaN or Inf reached a reduction            */
  PA_ERR_TIMEOUT = -5,       /* a device-side wait ran out of time          */
  PA_ERR_CUDA = -6,
  PA_ERR_OOM = -7,
  PA_ERR_LAUNCH = -8,        /* the persistent grid does not fit the GPU    */
  PA_ERR_UNSUPPORTED = -9
} pa_status;

enum { PA_HOST = 0, PA_DEVICE = 1 };                   /* pointer kinds        */
enum { PA_LOSS_LOGRATIO = 0, PA_LOSS_QUADRATIC = 1 };  /* loss forms           */
enum { PA_FP64 = 0, PA_MIXED = 1, PA_DF64 = 2 };       /* precision modes      */
enum { PA_EQ_NONE = 0, PA_EQ_STORAGE = 1, PA_EQ_TARGET = 2 }; /* equilibration */
enum { PA_ENGINE_AUTO = 0, PA_ENGINE_GRID = 1, PA_ENGINE_CLUSTER = 2, PA_ENGINE_MERGED = 3,
       PA_ENGINE_SINGLE = 4 };
enum { PA_ABLATE_NO_TANGENT = 1, PA_ABLATE_NO_NORMALISE = 2 };

typedef struct {
  /* Loss of Algorithm 1.  LOGRATIO (default) is the paper's
   * L(v) = log||v|| - log||Av|| with gradient Eq. nabla_loss (negated for
   * sigma_min).  QUADRATIC is L = -||Av||^2 (sigma_max) / +||Av||^2
   * (sigma_min) with gradient -/+ 2 A^T A v. */
  int loss;
  /* FP64 (default): every product, the Adam state and every reduction in
   * FP64.  MIXED (log-ratio loss only): sigma_max iterates with FP32
   * products and FP32 Adam state on the power-of-two-equilibrated matrix
   * D_r^-1 A D_c^-1 (norms reduced in FP64), then runs its last fp64_tail
   * iterations in FP64 from that state; x_min is whichever tracked iterate
   * of the two stages scores the larger ||A x|| / ||x|| in FP64.  sigma_min
   * uses compensated (double-double, Dot2) products for A x and A^T y and
   * for its final sigma.  DF64 (log-ratio loss only): the input stays FP64
   * and sigma is recomputed from it in FP64, but the iteration stores its
   * matrix values (as 2^-k A, k from the largest |a_ij|, exact) and vectors
   * as double-float pairs (hi + lo, two floats, about 48 significant bits,
   * the same 8 bytes per value) and runs its products and its per-row Adam
   * arithmetic in double-float on the FP32 pipe, with the reductions in
   * FP64.  A matrix whose non-zeros span more than 2^99, or a run whose
   * ||2^-k A x||^2 leaves [2^-100, 2^100], runs the FP64 kernel instead. */
  int precision;
  /* Equilibration with the paper's row and column 2-norm scaling (rows
   * first, then the columns of D_r^-1 A), each factor rounded to the nearest
   * power of two so the scaling is exact.  STORAGE (implied by MIXED): the
   * handle keeps D_r^-1 A D_c^-1 for its FP32 copies but every result still
   * refers to A.  TARGET: the handle's matrix IS A_hat = D_r^-1 A D_c^-1;
   * sigmas, kappa, products and the transpose all refer to A_hat (the
   * paper's kappa of the scaled system). */
  int equilibrate;
  int engine;       /* GRID: cooperative grid with timed software barriers
                       and three phases per iteration (product, transposed
                       product with Adam, update of x; two full barriers);
                       MERGED: the same grid with the update of x folded
                       into the next product (one full grid barrier per
                       iteration) -- what PA_DF64 always runs, opt-in for
                       FP64;
                       CLUSTER: one thread-block cluster (<= 16 CTAs) with
                       the hardware cluster barrier (plain FP64 only);
                       SINGLE: the grid reading A once per iteration with
                       no transposed copy: each CTA owns a block of rows
                       and the same x positions, sums A^T y over its rows'
                       column window and the owners add the overlapping
                       windows in CTA order (FP64, square matrices, rows of
                       at most 255 entries; PA_ERR_UNSUPPORTED otherwise);
                       AUTO: CLUSTER when the grid would use <= 16 CTAs    */
  int ablation;     /* PA_ABLATE_* bits: drop the tangent projection and/or
                       the normalisation of Algorithm 1 (the paper's vanilla
                       Adam comparison); 0 = Algorithm 1 as printed        */
  int64_t barrier_timeout_ns; /* device wait limit per barrier; <= 0 -> 2 s */
  int grid_blocks;  /* CTAs of the persistent grid: 0 = chosen from the size
                       (about four rows per thread, at most the GPU), > 0 =
                       that many (at most the GPU and the slice count)     */
  int debug_skip_arrival; /* test hook: > 0 makes CTA 0 skip the barrier of
                             that iteration, so the others time out (0 = off) */
  int fp64_tail;    /* MIXED sigma_max: the last iterations, run in FP64 from
                       the FP32 state (x, m, v) near convergence; < 0 (default)
                       = iters / 10, 0 = none */
  int autotune;     /* > 0: after each of the first `autotune` - 1 runs of
                       the grid engine, re-split the slices among the CTAs at
                       equal measured busy time (per-CTA timers of that run),
                       and after run `autotune` keep the fastest of the
                       partitions those runs used (cost-model start included);
                       before the first FP64 run of at least 20 iterations
                       on the AUTO engine with more than 16 CTAs and no
                       explicit grid_blocks, time 40-iteration trials of the
                       three-phase kernel with two and with one CTA per SM,
                       the merged-phase kernel and the single-pass kernel,
                       and keep the fastest (cached per matrix signature for
                       later handles; see pa_launch_choice);
                       and when this handle is the first of a
                       pa_estimate_batched call, time short trials of the
                       batch with restart blocks of 8, 4 and 2 vectors and
                       keep the fastest width (cached per k_restarts).
                       Both choices set the order of reductions, so tuned
                       runs are reproducible only for the same choice; 0
                       (default) keeps the fixed cost model and width 8. */
} pa_options;

/* Fill *opt with the defaults above (LOGRATIO, FP64, no equilibration, AUTO
 * engine, no ablation, 2 s barrier limit, full grid, no debug hook, FP64 tail
 * of iters / 10 in MIXED mode). */
void pa_options_default(pa_options* opt);

/* Build a handle for the n_rows x n_cols matrix A given in CSR.
 * row_ptr (n_rows+1 int32), col_idx (nnz int32) and vals (nnz float64) are
 * host pointers (ptr_kind = PA_HOST) or device pointers (PA_DEVICE); both are
 * copied.  On the device the library validates the CSR, builds the explicit
 * CSR of A^T with a stable (row-ordered) transpose, and, when opt asks for
 * it, the power-of-two equilibration of the paper's "Row and Column Scaling"
 * subsection.  opt may be NULL (defaults).  cuda_stream is a cudaStream_t or
 * NULL.  Errors: PA_ERR_INVALID_ARG (sizes < 0, NULL pointers with nnz > 0),
 * PA_ERR_INVALID_CSR, PA_ERR_OOM, PA_ERR_CUDA. */
pa_status pa_create(pa_handle* out, int32_t n_rows, int32_t n_cols, int64_t nnz,
                    const int32_t* row_ptr, const int32_t* col_idx, const double* vals,
                    int ptr_kind, const pa_options* opt, void* cuda_stream);

/* Estimate sigma_max and/or sigma_min of A with Algorithm 1: `iters`
 * iterations of Projected Adam (step size lr, moment decays beta1, beta2,
 * epsilon eps) from the start vector x_i = 2u_i - 1, u_i the i-th SplitMix64
 * output of `seed` scaled to [0, 1), normalised to unit length.  Each sigma
 * is ||A x_min|| / ||x_min|| for the tracked minimiser x_min.  The handle keeps
 * the latest sigma_max and sigma_min, so kappa = sigma_max / sigma_min once
 * both modes have run (NaN before).  Host outputs; each may be NULL.
 * PA_SIGMA_MIN_LU / PA_BOTH_LU take sigma_min through the attached LU
 * factors (Algorithm 2); the same start vector serves both modes.
 * Returns PA_OK, PA_WARN_SINGULAR or an error (PA_ERR_NONFINITE,
 * PA_ERR_TIMEOUT, PA_ERR_NOT_SQUARE for sigma_min with n_rows < n_cols,
 * PA_ERR_INVALID_ARG for an LU mode without factors). */
pa_status pa_estimate(pa_handle h, pa_mode mode, int iters, double lr, double beta1,
                      double beta2, double eps, uint64_t seed, double* sigma_max,
                      double* sigma_min, double* kappa);

/* Attach an LU factorisation P A Q = L U of the handle's (square) matrix for
 * the paper's sigma_min route (Algorithm 2: r = A^{-1} x from L U r = x,
 * s = A^{-T} r from U^T L^T s = r, gradient x/||x||^2 - s/||r||^2, inside
 * Algorithm 1 on A^{-1}).  The library does not factorise: the factors come
 * from the caller's direct solver.
 *   L: lower triangular, U: upper triangular, n x n CSR (int32 row_ptr[n+1],
 *   col[nnz], float64 val[nnz]; each row stores its non-zero diagonal; L
 *   need not be unit).  p[i] = the row of A that is row i of P A, q[j] = the
 *   column of A that is column j of A Q (int32[n]; NULL = identity).
 *   Host pointers (ptr_kind = PA_HOST) or device pointers (PA_DEVICE); all
 *   are copied, a second call replaces the factors.
 * The host orders each triangular system by dependency level once here.  With
 * engine AUTO the iteration runs as one CTA that walks the levels while the
 * factors have fewer than 8,192 rows and the solve vector fits its shared
 * memory; past that as one thread-block cluster of 16 CTAs that walks the
 * same levels, each CTA applying the entries of the rows it holds (the solve
 * vector spread over their shared memories, up to about 430k rows on GB300);
 * past that on the whole grid, each row solved as soon as the values it
 * depends on are written.  Engine GRID forces the grid, CLUSTER the cluster
 * (when the vector fits).  The cost per iteration grows with the number of
 * dependency levels, so fill-reducing orderings with short elimination trees
 * run fastest.
 * Errors: PA_ERR_NOT_SQUARE, PA_ERR_INVALID_ARG (NULL pointers, a factor that
 * is not triangular, has an entry out of range or a zero or missing
 * diagonal, p or q not a permutation), PA_ERR_OOM, PA_ERR_CUDA. */
pa_status pa_attach_lu(pa_handle h, const int32_t* l_row_ptr, const int32_t* l_col,
                       const double* l_val, const int32_t* u_row_ptr, const int32_t* u_col,
                       const double* u_val, const int32_t* p, const int32_t* q, int ptr_kind);

/* Algorithm 1 for one mode (PA_SIGMA_MAX, PA_SIGMA_MIN or PA_SIGMA_MIN_LU) from a given
 * start vector x_init (n_cols float64, host or device per x_kind, used as
 * is: Algorithm 1 does not normalise x_init).  Host outputs, each may be NULL:
 *   x_min[n_cols]   Algorithm 1's return value
 *   x_last[n_cols]  the iterate after the last iteration
 *   info[4]         {L_min, t_min (0 = x_init), L(x_T), iterations run}
 *   L_trace[iters]  L(x_t) for t = 1..iters
 *   x_trace[n_trace * n_cols]  x_t for t = 1..n_trace (n_trace <= iters)
 *   sigma           ||A x_min|| / ||x_min||; for PA_SIGMA_MIN_LU the
 *                   iterates live on A^{-1}: L(x) = log||x|| - log||A^{-1} x||
 *                   and sigma = ||x_min|| / ||A^{-1} x_min|| = sigma_min(A)
 */
pa_status pa_run(pa_handle h, pa_mode mode, int iters, double lr, double beta1, double beta2,
                 double eps, const double* x_init, int x_kind, double* x_min, double* x_last,
                 double* info, double* L_trace, double* x_trace, int n_trace, double* sigma);

/* Many independent estimates in one persistent launch (captured in a CUDA
 * graph): item (i, r), i < n_mat, r < k_restarts, runs Algorithm 1 on the
 * matrix of handles[i] from the start vector of seed s_ir = SplitMix64 output
 * number (i * k_restarts + r) of `seed`; the k restarts of a matrix advance
 * together as a block of k vectors (SpMM).  iters[0] iterations for sigma_max
 * and iters[1] for sigma_min.  All handles must share one stream and one
 * precision mode.  With MIXED handles sigma_max runs, like pa_estimate, an
 * FP32 stage (FP32 products and Adam state on D_r^-1 A D_c^-1, norms in
 * FP64) for iters[0] - fp64_tail iterations and then the FP64 tail from that
 * state (fp64_tail of the first handle); each item's sigma_max is the larger
 * of the two stages' tracked minimisers scored in FP64; sigma_min runs with
 * Dot2 (compensated) products, as in pa_estimate.  With PA_DF64 handles the
 * products and Adam run in double-float per vector (FP64 reductions), as in
 * pa_estimate, in blocks of 4 restarts by default; a batch with a matrix
 * outside the double-float range, or a block whose ||A x|| leaves it, runs
 * in FP64.  Host outputs:
 *   out[(i * k_restarts + r) * 3 + {0,1,2}] = {sigma_max, sigma_min, kappa}
 *   item_status[i * k_restarts + r]  (may be NULL)
 * mode selects which sigmas run (the others are written as NaN). */
pa_status pa_estimate_batched(int n_mat, const pa_handle* handles, pa_mode mode, int k_restarts,
                              const int* iters, double lr, double beta1, double beta2, double eps,
                              uint64_t seed, double* out, pa_status* item_status);

/* 1 when the calling thread's latest pa_estimate_batched ran as one CUDA
 * graph (start vectors, resets, the persistent launches and the sigma
 * kernels captured and replayed), 0 when the driver refused the capture and
 * the same sequence ran as ordinary launches. */
int pa_last_batch_graph(void);

/* x_min of the latest run of `which` (PA_SIGMA_MAX, PA_SIGMA_MIN or
 * PA_SIGMA_MIN_LU) into the host array x_min_host[n_cols] (Algorithm 1's
 * output; for PA_SIGMA_MIN_LU the maximiser of ||A^{-1} x|| / ||x||). */
pa_status pa_get_vector(pa_handle h, pa_mode which, double* x_min_host);

/* y = A x (n_rows outputs) or z = A^T y over the explicit transpose (n_cols
 * outputs) with the library's CSR product kernels; ptr_kind says whether x/y
 * are host or device pointers.  Used to check the product kernels. */
pa_status pa_spmv(pa_handle h, const double* x, double* y, int ptr_kind);
pa_status pa_spmv_t(pa_handle h, const double* y, double* z, int ptr_kind);

/* The CSR of A^T as built on the device (host outputs: row_ptr_t[n_cols+1],
 * col_t[nnz], val_t[nnz]; each may be NULL). */
pa_status pa_get_transpose(pa_handle h, int32_t* row_ptr_t, int32_t* col_t, double* val_t);

/* The paper's error analysis (section "Error estimates and conditioning",
 * Theorems 1-4) for an approximate solution x_hat of A x = b, A being the
 * handle's matrix (A_hat under PA_EQ_TARGET).
 *   x_hat: n_cols float64; b: n_rows float64; host (ptr_kind = PA_HOST) or
 *   device (PA_DEVICE) pointers, read only.
 *   kappa, norm_a: kappa_2(A) and ||A||_2; a value <= 0 takes the handle's
 *   latest estimates (sigma_max / sigma_min and sigma_max).
 *   u: unit roundoff for Theorem 4 (<= 0: 2^-53, FP64).
 *   out: host array of 10 float64:
 *     [0] ||r||, r = A x_hat - b accumulated in Dot2 (compensated: each row's
 *         products in CSR order, then -b_i); [1] ||b||; [2] ||x_hat||;
 *     [3], [4] Theorem 1: ||x_hat - x|| / ||x|| lies in
 *         [(||r||/||b||) / kappa, kappa ||r||/||b||];
 *     [5], [6] Theorem 2: ||x_hat - x|| / ||x_hat|| lies in
 *         [||r|| / (||A|| ||x_hat||), eps = kappa ||r|| / (||A|| ||x_hat||)];
 *     [7] Theorem 3: ||x_hat - x|| / ||x|| <= eps / (1 - eps) (+inf if eps >= 1);
 *     [8] Theorem 4: the rounding error bound 2 u kappa / (1 - kappa u)
 *         (+inf if kappa u >= 1); [9] 1 if kappa u >= 1 (numerically singular
 *         at precision u), else 0.
 *   Divisions follow IEEE rules (b = 0 gives inf/NaN in [3], [4]).
 * Bit-reproducible for a given matrix and inputs.  Synchronises the handle's
 * stream.  Errors: PA_ERR_INVALID_ARG (NULL pointers, no estimates to default
 * to), PA_ERR_OOM, PA_ERR_CUDA. */
pa_status pa_error_bounds(pa_handle h, const double* x_hat, const double* b, int ptr_kind,
                          double kappa, double norm_a, double u, double* out);

/* The power-of-two equilibration factors D_r (n_rows) and D_c (n_cols) of the
 * handle (host outputs): those of A_hat = D_r^-1 A D_c^-1 under PA_EQ_TARGET,
 * else those of the STORAGE copies; PA_ERR_INVALID_ARG when the handle has
 * none. */
pa_status pa_get_equilibration(pa_handle h, double* d_row, double* d_col);

/* Diagnostics of the latest persistent run of the handle: *grid = number of
 * CTAs, and (when busy_ns is not NULL and holds 2 * *grid entries) the time
 * each CTA spent working in phase A (y = A x) and in phases B and C (the
 * transposed product, Adam, the update of x), barrier waits excluded, in
 * nanoseconds of the GPU's global timer.  Host outputs. */
pa_status pa_last_run_profile(pa_handle h, int* grid, double* busy_ns);

/* Checkpoint/resume: continue the handle's latest single-vector run for
 * `iters` more iterations of Algorithm 1, from the state that run left on the
 * device (its last iterate x_T, Adam's moments m and v, the iteration count
 * for the bias corrections, and the tracked minimum L_min with x_min).  The
 * run being continued must be a successful PA_FP64 pa_estimate / pa_run of
 * PA_SIGMA_MAX or PA_SIGMA_MIN on the three-phase grid or the cluster kernel,
 * or an earlier pa_continue, with the same hyperparameters (else
 * PA_ERR_INVALID_ARG).  A run of T1 iterations continued for T2 gives the
 * same bits as one run of T1 + T2 (same partition: autotune 0 or finished):
 * x_min, the returned sigma, x_last and L_min.  Host outputs, each may be
 * NULL: sigma (||A x_min|| / ||x_min|| for the continued mode), x_last
 * (n_cols float64, source order), info[4] = {L_min, t_min, L_last,
 * iterations run in total}.  Also updates the sigma pa_estimate reports for
 * that mode. */
pa_status pa_continue(pa_handle h, int iters, double lr, double beta1, double beta2, double eps,
                      double* sigma, double* x_last, double* info);

/* z = A^T (A x) (Eq. nabla_loss's A^T A v term) through the single-pass
 * engine's per-CTA window plans, without the transposed copy: y = A x over
 * each CTA's row block, each CTA's window sums of A^T y in row order, and the
 * owners of the positions add the overlapping windows in CTA order (so the
 * result is reproducible bit for bit).  x and z have n_cols float64 entries
 * (source order), host or device memory per ptr_kind; the caller owns both.
 * Builds the plans on first use (square matrices with rows of at most 255
 * entries; PA_ERR_UNSUPPORTED otherwise). */
pa_status pa_spmv_ata(pa_handle h, const double* x, double* z, int ptr_kind);

/* The launch-shape tuner's choice (see the autotune option), into out[4]
 * (host): kernel (-1 none yet; 0 three-phase, 1 merged-phase, 6 single-pass,
 * as in pa_last_run_info), CTAs, source (0 none, 1 this handle's trials,
 * 2 an earlier handle of a matrix with the same signature) and the number of
 * trial candidates (at most 4).  cand (8 entries, kernel and CTAs per
 * candidate) and ms (4 entries, each trial's time) may be NULL. */
pa_status pa_launch_choice(pa_handle h, int64_t* out, int64_t* cand, double* ms);

/* The single-pass engine's plan sizes, into out[6] (host): CTAs it was built
 * for (0 before first use), window columns over all CTAs (halo slots), plan
 * entries (one per non-zero), plan slots (entries plus the padding of the
 * 32-column groups), groups, and padded entries of the sliced copy of A. */
pa_status pa_single_pass_info(pa_handle h, int64_t* out);

/* The route the LU route's next run takes for the attached factors (Algorithm
 * 2; see pa_attach_lu), into out[4] (host): route (0 one CTA, 1 the grid,
 * 2 a thread-block cluster), the cluster's CTAs, its staging-slot records,
 * and 1 when its CTAs also keep the rows' final values (steps then end
 * without memory ordering) or 0 when its steps end with a release barrier;
 * the last three are 0 for the other routes.
 * Errors: PA_ERR_INVALID_ARG (NULL argument, no factors attached). */
pa_status pa_lu_route_info(pa_handle h, int64_t* out);

/* Facts about the handle's latest single-vector run (pa_estimate, pa_run),
 * into out[4] (host):
 *   out[0] kernel: 0 the three-phase grid kernel, 1 the merged-phase grid
 *          kernel in FP64, 2 the merged-phase grid kernel in double-float
 *          (PA_DF64), 3 the cluster kernel, 4 the LU route on one CTA, 5 the
 *          LU route on the grid, 6 the single-pass kernel, 7 the LU route on
 *          one thread-block cluster; -1 before any run;
 *   out[1] iterations of the merged-phase kernel that multiplied x itself
 *          instead of folding the update of x into the product (see the
 *          engine option);
 *   out[2] PA_DF64 runs that left the double-float range and were redone in
 *          FP64, since the handle was created;
 *   out[3] CTAs of the run's grid. */
pa_status pa_last_run_info(pa_handle h, int64_t* out);

/* Launches of this library's kernels since the handle was created (a
 * counter kept by the host code at every launch). */
int64_t pa_kernel_launches(pa_handle h);

/* sigma = ||A x||_2 / ||x||_2 for a CSR matrix and a vector already in
 * device memory, with no device memory allocated by the call.  (The paper has
 * no counterpart: this exists for callers that cannot allocate at this point,
 * e.g. because their device memory is fully held by another allocator or
 * because cudaMalloc's implicit device-wide synchronisation is not
 * acceptable there.)
 *   row_ptr (n_rows+1 int32), col_idx and vals (nnz int32 / float64), x
 *   (n_cols float64): device pointers, read only, none of them NULL (for a
 *   matrix without entries pass any valid device address as col_idx and
 *   vals); the CSR is not validated.
 *   sigma: device pointer to one float64, written by the call's kernels.
 *   cuda_stream: cudaStream_t (NULL = legacy default stream); the call only
 *   enqueues work and returns without synchronising.
 * Scratch: a fixed 128 KiB array of device memory inside the library (held
 * on every GPU that loads it until the process exits) limits
 * max(n_rows, n_cols) to 2,097,152; larger sizes give PA_ERR_INVALID_ARG.
 * The first call on a device looks up that array's address (once per
 * device) and keeps it for the process: calls must run in the device's
 * primary context (the CUDA runtime's), and a cudaDeviceReset between calls
 * is not supported.  Make that first call before any stream capture.  All calls share
 * the array: calls whose kernels may overlap on the GPU race and must be
 * ordered by the caller (same stream or events).  Errors: PA_ERR_INVALID_ARG,
 * PA_ERR_CUDA, PA_ERR_UNSUPPORTED (device index 64 or above). */
pa_status pa_sigma_noalloc(int32_t n_rows, int32_t n_cols, const int32_t* row_ptr,
                           const int32_t* col_idx, const double* vals, const double* x,
                           double* sigma, void* cuda_stream);

/* Release the handle and its device memory (NULL-safe). */
void pa_destroy(pa_handle h);

/* Message of the latest error on this thread ("" if none). */
const char* pa_last_error(void);

/* Device allocator hooks (for example the PyTorch caching allocator).  With
 * none installed the library uses cudaMallocAsync/cudaFreeAsync on the
 * handle's stream.  alloc returns NULL on failure.  Affects handles created
 * after the call. */
typedef void* (*pa_alloc_fn)(size_t bytes, void* cuda_stream, void* ctx);
typedef void (*pa_free_fn)(void* ptr, size_t bytes, void* cuda_stream, void* ctx);
void pa_set_allocator(pa_alloc_fn alloc, pa_free_fn free_fn, void* ctx);

#ifdef __cplusplus
}
#endif
#endif /* PA_H */
