// pa_internal.h -- types shared by the host runtime (pa_api.cu) and the
// kernel translation units of the Projected Adam library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pa.h"

namespace pa {

constexpr int kBlock = 512;       // threads per CTA of the persistent kernels
constexpr int kMinBlocksPerSM = 2;
constexpr int kPartSlots = 4;     // per-CTA partial sums: s, q, p1, p2

// State of one persistent run; lives in device memory, read back at the end.
struct RunState {
  int status;          // pa_status
  int minb;            // buffer index holding x_min
  int cur;             // buffer index holding the last iterate
  int t_min;           // iteration whose iterate is x_min (0 = x_init)
  double L_min;
  double L_last;
  int iters_run;
  int timeout_site;    // barrier number where a wait gave up (-1 = none)
  unsigned int barrier;  // monotonically increasing arrival counter
  unsigned int abort;    // set by the first CTA that gives up
  double sigma;        // ||A x_min|| / ||x_min||, written by the sigma kernel
  double pad;
};

// Everything one Projected Adam run needs; passed by value to the kernels.
struct IterParams {
  int32_t n_rows, n_cols;
  const int32_t* rp;  const int32_t* ci;  const double* va;   // A (CSR)
  const int32_t* rpt; const int32_t* cit; const double* vat;  // A^T (CSR)
  const int32_t* part_a;   // [G+1] row ranges of A per CTA
  const int32_t* part_t;   // [G+1] row ranges of A^T per CTA
  double* X0; double* X1; double* X2;  // three iterate buffers
  double* m; double* v;                // Adam moments
  double* y; double* ylo;              // y = A x (ylo: low part, compensated mode)
  double* dx;                          // Adam step of the current iteration
  double* partials;                    // [G][kPartSlots]
  const double2* bias;                 // [iters]: {lr/(1-b1^t), 1/(1-b2^t)}
  double* L_trace;                     // [iters] or null
  double* x_trace;                     // [n_trace][n_cols] or null
  int n_trace;
  RunState* st;
  int iters;
  int mode;       // PA_SIGMA_MAX / PA_SIGMA_MIN
  int ablation;   // PA_ABLATE_* bits
  double beta1, beta2, eps;
  long long timeout_ns;
  int skip_arrival;
};

// ---- launch wrappers implemented in the kernel translation units --------
// Each returns the CUDA error of its launch(es) and adds its launch count to
// *launches.

cudaError_t launch_validate_csr(int32_t n_rows, int32_t n_cols, int64_t nnz, const int32_t* rp,
                                const int32_t* ci, int* flag, cudaStream_t s, int64_t* launches);

// Stable transpose of CSR(A) into CSR(A^T).  Scratch: cursor[n_cols],
// src[nnz], rowid[nnz], blocksums[scan_blocks(n_cols+1)].  *long_flag is set
// when a column holds more entries than the segment sort supports.
int scan_blocks(int64_t n);
cudaError_t launch_transpose(int32_t n_rows, int32_t n_cols, int64_t nnz, const int32_t* rp,
                             const int32_t* ci, const double* va, int32_t* rpt, int32_t* cit,
                             double* vat, int32_t* cursor, int32_t* src, int32_t* rowid,
                             int32_t* blocksums, int* long_flag, cudaStream_t s,
                             int64_t* launches);

cudaError_t launch_partition(const int32_t* rp, int32_t n, int G, int row_weight, int32_t* part,
                             cudaStream_t s, int64_t* launches);

cudaError_t launch_start_vector(int32_t n, uint64_t seed, double* x, double* blockpart,
                                cudaStream_t s, int64_t* launches);
int start_vector_blocks(int32_t n);

cudaError_t launch_spmv(int32_t n_rows, const int32_t* rp, const int32_t* ci, const double* va,
                        const double* x, double* y, cudaStream_t s, int64_t* launches);

// sigma = ||A x_sel|| / ||x_sel|| where x_sel is the buffer st->minb of
// {X0, X1, X2} (or X0 when use_minb == 0); result into st->sigma.
int sigma_blocks(int32_t n_rows, int32_t n_cols);
cudaError_t launch_sigma(int32_t n_rows, int32_t n_cols, const int32_t* rp, const int32_t* ci,
                         const double* va, const double* X0, const double* X1, const double* X2,
                         int use_minb, RunState* st, double* blockpart, cudaStream_t s,
                         int64_t* launches);

// Persistent cooperative Projected Adam run (Algorithm 1) over a grid of G CTAs.
int persistent_max_blocks(int loss, int* blocks_per_sm);
cudaError_t launch_persistent(const IterParams& p, int loss, int G, cudaStream_t s,
                              int64_t* launches);

}  // namespace pa
