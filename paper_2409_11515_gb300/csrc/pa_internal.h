// pa_internal.h -- types shared by the host runtime (pa_api.cu) and the
// kernel translation units of the Projected Adam library.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>
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
  int refreshes;       // merged-phase kernel: iterations that multiplied x itself
  int have_best;       // three-phase kernel: the tracked minimum at the end of
  double best_s, best_q;  // the run (for a continued run): ||y||^2, ||x||^2
};

// A row- and column-permuted copy P A Q^T of a matrix in sliced ELL form:
// rows are stable-sorted by length (descending) inside windows of kWindow
// rows, cut into slices of 32 rows, and each slice is stored column-major
// (entry k of lane l at 32 * (wp[s] + k) + l) padded to its longest row with
// zero values.  Entry order inside a row is the order of the source CSR.
constexpr int kWindow = 1024;
struct Sell {
  int32_t n_rows = 0;      // rows of the permuted matrix
  int32_t n_slices = 0;    // ceil(n_rows / 32)
  int32_t* wp = nullptr;   // [n_slices + 1] exclusive scan of slice widths
  int32_t* col = nullptr;  // [32 * wp[n_slices]] permuted column positions
  double* val = nullptr;   // [32 * wp[n_slices]]
  int32_t* perm = nullptr; // [n_rows] position -> source row
  int32_t* pos = nullptr;  // [n_rows] source row -> position
};

// Everything one Projected Adam run needs; passed by value to the kernels.
struct IterParams {
  int32_t n_rows, n_cols;
  const int32_t* a_wp; const int32_t* a_col; const double* a_val;  // P A Q^T (sliced ELL)
  const int32_t* t_wp; const int32_t* t_col; const double* t_val;  // Q A^T P^T
  const int32_t* part_a;   // [G+1] slice ranges of P A Q^T per CTA
  const int32_t* part_t;   // [G+1] slice ranges of Q A^T P^T per CTA (own x rows)
  // each CTA's slices dealt to its kBlock/32 warps: warp w of CTA b takes
  // a_list[a_woff[b (NW+1) + w] .. a_woff[b (NW+1) + w + 1]) (t_*: A^T)
  const int32_t* a_list; const int32_t* a_woff;
  const int32_t* t_list; const int32_t* t_woff;
  double* X0; double* X1; double* X2;  // three iterate buffers
  double* m; double* v;                // Adam moments
  double* y; double* ylo;              // y = A x (ylo: low part, compensated mode)
  double* dx;                          // Adam step of the current iteration
  double* partials;                    // [G][kPartSlots]
  unsigned* ready;                     // [G] last iteration whose x_t each CTA has written
  unsigned long long* cta_ns;          // [2G] per-CTA time in phases A and B+C (ns), or null
  unsigned long long* cta_lat;         // [G] per-CTA sum over iterations of (end of phase A -
                                       // start of the previous phase C), or null
  const int32_t* dep;                  // [2G] CTAs whose x rows CTA b's phase A reads: [lo, hi]
  const double2* bias;                 // [iters]: {lr sqrt(1-b2^t)/(1-b1^t), eps sqrt(1-b2^t)}
  double* L_trace;                     // [iters] or null
  double* x_trace;                     // [n_trace][n_cols] or null
  int n_trace;
  RunState* st;
  int iters;
  int t0;         // iterations already done (bias corrections continue at t0 + 1)
  int mode;       // PA_SIGMA_MAX / PA_SIGMA_MIN
  int ablation;   // PA_ABLATE_* bits
  double beta1, beta2, eps;
  double omb1;    // 1 - beta1
  double w2;      // (1 - beta2) / (1 - beta1)^2
  long long timeout_ns;
  int skip_arrival;
  // ---- continued runs of k_persistent (pa_continue): the tracked state of
  // the run being continued; all zero for a fresh run ----
  int init_have_best, init_t_min, init_minb;
  double init_best_s, init_best_q;
  int t_min_base;                      // iteration numbers of this run start after it
  // ---- the merged-phase kernel (k_merged) ----
  double* u;                           // u_t = x_{t-1} - dx_t (FP64 variant)
  // double-float variant (PA_DF64): values of 2^-k P A Q^T and of its
  // transpose as (hi, lo) float pairs, and the vectors in the same form
  const float2* a_val2; const float2* t_val2;
  float2 *XD0, *XD1, *XD2;             // iterate buffers
  float2 *ud, *md, *vd, *yd;           // u, Adam moments, y = 2^-k A x
  const float4* bias2;                 // [iters]: K1 and K2 of `bias` as (hi, lo) pairs
  double s_scale;                      // 4^k: ||A x||^2 = s_scale ||2^-k A x||^2
  int win_slices;                      // slices per CTA whose products wait in shared memory
  // ---- the single-pass engine (k_single): part_a is its row/position
  // partition, dep its window's owners, a_list/a_woff its warp lists ----
  // CTA b's window columns (those its rows touch, sorted by entry count) come
  // in groups of 32, one per lane: groups [sp_goff[b], sp_goff[b+1]); group
  // g's entries sit column-major at sp_ent[32 (sp_gp[g] + k) + lane], k <
  // sp_gp[g+1] - sp_gp[g], each (row - 32 part_a[b]) << 8 | slot in the row,
  // or kPlanPad; lane l's column is window slot sp_gcol[32 g + l] (-1: none)
  const int32_t* sp_cmin;   // [G] first x position of CTA b's column window
  const int32_t* sp_woff;   // [G+1] CTA b's window columns are slots [sp_woff[b], sp_woff[b+1])
  const int32_t* sp_goff;   // [G+1]
  const int32_t* sp_gp;     // [groups + 1]
  const int32_t* sp_gcol;   // [32 groups]
  const uint32_t* sp_ent;   // [32 sp_gp[groups]]
  double* sp_halo;          // [sp_woff[G]] CTA b's partial sums of A^T y over its window
  const int32_t* sp_rdep;   // [2G] CTAs whose windows meet CTA b's own positions: [lo, hi]
};

constexpr uint32_t kPlanPad = 0xffffffffu;  // a padding slot of a plan group
// The single-pass engine: Algorithm 1 reading P A Q^T once per iteration
// (no transposed copy); needs a square matrix, slices at most 255 wide.
int single_max_blocks(int loss);
cudaError_t launch_single(const IterParams& p, int loss, int G, cudaStream_t s, int64_t* launches);
// z = A^T (A x) at positions through the same plan (y is left in p.y).
cudaError_t launch_single_product(const IterParams& p, int G, const double* x, double* z,
                                  cudaStream_t s, int64_t* launches);

// The mixed-precision sigma_max iteration (FP32 products and Adam state on
// the power-of-two-equilibrated matrix, FP64 norms).
struct IterParams32 {
  int32_t n_rows, n_cols;
  const int32_t* a_wp; const int32_t* a_col; const float* a_val;  // P A_hat Q^T (sliced)
  const int32_t* t_wp; const int32_t* t_col; const float* t_val;  // Q A_hat^T P^T
  const float* dr;   // [n_rows] D_r at the row positions of P A Q^T
  const float* dc;   // [n_cols] D_c at the x positions
  const int32_t* part_a; const int32_t* part_t; const int32_t* dep;
  float* X0; float* X1; float* X2;  // iterate buffers
  float* W;                          // D_c x of the latest iterate
  float* m; float* v; float* y; float* dx;
  double* partials;
  unsigned* ready;
  unsigned long long* cta_ns;
  const double2* bias;
  double* L_trace;
  RunState* st;
  int iters;
  int ablation;
  double beta1, beta2;
  double omb1;    // 1 - beta1
  double w2;      // (1 - beta2) / (1 - beta1)^2
  long long timeout_ns;
  int skip_arrival;
};

// One matrix of a batched launch: its sliced copies, its group of CTAs and
// its n x K (row-major) blocks of vectors.
struct BatchItem {
  int32_t n_rows, n_cols;
  const int32_t* a_wp; const int32_t* a_col; const double* a_val;
  const int32_t* t_wp; const int32_t* t_col; const double* t_val;
  int cta0, ncta;                       // CTAs [cta0, cta0 + ncta) of the grid
  const int32_t* part_a; const int32_t* part_t;  // [ncta + 1] slice ranges
  double* partials;                     // [ncta][4][K]
  unsigned* barrier;                    // the group's arrival counter
  double *X0, *X1, *XMIN, *M, *V, *DX, *Y;
  double* YLO;                          // low parts of Y (Dot2 products only)
  double* result;                       // [K][4]: L_min, t_min, L_last, iterations
  int* status;                          // [1]
  const int32_t* pos_c;                 // source column -> x position (Q)
  int32_t n_slices_a;                   // slices of P A Q^T
  // MIXED sigma_max stage (k_batched32): FP32 values of the sliced
  // A_hat = D_r^-1 A D_c^-1 and its transpose, the power-of-two D_r, D_c in
  // FP32 (positions of the sliced copies), and the FP32 block vectors
  const float* a_val32; const float* t_val32; const float* dr32; const float* dc32;
  float *X0f, *X1f, *XMINf, *Mf, *Vf, *DXf, *Yf, *Wf;
  // PA_DF64 (k_batched_df): the sliced values of 2^-k A and of its
  // transpose as (hi, lo) float pairs, and 4^k (||A x||^2 = 4^k ||2^-k A x||^2);
  // the block vectors above are then read as float pairs
  const float2* a_val2; const float2* t_val2;
  double s_scale;
};

struct BatchParams {
  const BatchItem* items;
  const int32_t* cta_item;   // [G] item of each CTA
  const double2* bias;       // [iters] as in IterParams
  RunState* st;              // shared abort flag
  int iters, mode, loss, ablation;
  int t0;     // iteration t uses bias[t0 + t - 1] (a continued run)
  double beta1, beta2;
  double w2;  // (1 - beta2) / (1 - beta1)^2
  long long timeout_ns;
  const float4* bias2;       // [iters] the bias constants as (hi, lo) pairs (k_batched_df)
};

int batched_threads();
// dd: Dot2 products in both phases (YLO holds the low parts of Y).
int batched_max_blocks(int k, bool dd = false);
cudaError_t launch_batched(const BatchParams& p, int k, int G, bool dd, cudaStream_t s,
                           int64_t* launches);
// The MIXED sigma_max stage of a batch (log-ratio loss): FP32 products and
// FP32 Adam state on A_hat, per-column norms reduced in FP64, the same CTA
// groups, partitions and result layout as k_batched.  Reads X0f (x_init);
// leaves x_{iters} in X0f (iters even) or X1f, the tracked minimisers in XMINf.
// The PA_DF64 form of k_batched (log-ratio loss): double-float products and
// Adam state per column, FP64 reductions; the same groups, partitions and
// result layout.  Reads X0 and XMIN as float pairs (x_init), M and V zero.
int batched_df_max_blocks(int k);
cudaError_t launch_batched_df(const BatchParams& p, int k, int G, cudaStream_t s, int64_t* launches);
int batched32_max_blocks(int k);
cudaError_t launch_batched32(const BatchParams& p, int k, int G, cudaStream_t s, int64_t* launches);

// Start vectors of a batch: column c of item i is the SplitMix64 stream of
// seed splitmix64_at(seed, (i0 + i) * k_stride + r0 + c), normalised per
// column (columns >= k_used repeat column 0).  blk_item/blk_row0 describe
// the blocks ([nb] each, rows [row0, row0 + rows)).
cudaError_t launch_batch_start(const BatchItem* items_dev, int n_items, int K, int k_used,
                               int k_stride, int i0, int r0, uint64_t seed, const int32_t* blk_item,
                               const int32_t* blk_row0, int nb, int rows_per_block,
                               double* blockpart, const int32_t* item_blk0, cudaStream_t s,
                               int64_t* launches);
// sigma per (item, column) of XMIN: out[(i * K + c)] for c < K.
cudaError_t launch_batch_sigma(const BatchItem* items_dev, int n_items, int K,
                               const int32_t* blk_item, const int32_t* blk_row0, int nb,
                               int rows_per_block, double* blockpart, const int32_t* item_blk0,
                               double* out, bool dd, cudaStream_t s, int64_t* launches);

// Record a message for pa_last_error() (printf-style) and return st.
pa_status set_error(pa_status st, const char* fmt, ...);

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

// Slice partition of the persistent grid: part[b] = first slice whose
// cumulative cost 32 * wp[s] + row_weight * 32 * s reaches b / G of the total.
cudaError_t launch_partition(const int32_t* wp, int32_t n_slices, int G, int row_weight,
                             int32_t* part, cudaStream_t s, int64_t* launches);

// Sliced ELL of P M Q^T from CSR(M): perm/pos of the rows (window sort by
// length), then slice widths, their scan and the column-major fill; col
// indices go through col_pos (the column permutation).  `lens` and `widths`
// are scratch of n_rows and n_slices + 1 entries, `blocksums` of
// scan_blocks(n_slices + 1).
int32_t sell_slices(int32_t n_rows);
// Non-zero values per row (explicit zeros are not stored in the sliced copies).
cudaError_t launch_row_lengths(int32_t n_rows, const int32_t* rp, const double* va,
                               int32_t* lens, cudaStream_t s, int64_t* launches);
cudaError_t launch_window_sort(int32_t n, const int32_t* lens, int32_t* perm, int32_t* pos,
                               cudaStream_t s, int64_t* launches);
cudaError_t launch_sell_build(int32_t n_rows, const int32_t* rp, const int32_t* ci,
                              const double* va, const int32_t* lens, const int32_t* col_pos,
                              Sell* out, int32_t* widths, int32_t* blocksums, int64_t* total,
                              cudaStream_t s, int64_t* launches);
cudaError_t launch_sell_fill(int32_t n_rows, const int32_t* rp, const int32_t* ci,
                             const double* va, const int32_t* lens, const int32_t* col_pos,
                             const Sell& out, cudaStream_t s, int64_t* launches);

// out[pos[i]] = in[i] (to permuted order) and out[i] = in[pos[i]] (back).
cudaError_t launch_permute(int32_t n, const int32_t* pos, const double* in, double* out,
                           cudaStream_t s, int64_t* launches);
cudaError_t launch_unpermute(int32_t n, int32_t count, const int32_t* pos, const double* in,
                             double* out, cudaStream_t s, int64_t* launches);

// Start vector in source coordinates i, written at position pos[i], normalised.
cudaError_t launch_start_vector(int32_t n, uint64_t seed, const int32_t* pos, double* x,
                                double* blockpart, cudaStream_t s, int64_t* launches);
int start_vector_blocks(int32_t n);

// y = M x for a sliced-ELL matrix (permuted coordinates on both sides).
cudaError_t launch_sell_spmv(const Sell& m, const double* x, double* y, cudaStream_t s,
                             int64_t* launches);

// sigma = ||M x_sel|| / ||x_sel|| where x_sel is the buffer st->minb of
// {X0, X1, X2} (or X0 when use_minb == 0); result into st->sigma.
int sigma_blocks(int32_t n_slices, int32_t n_cols);
cudaError_t launch_sigma(const Sell& m, int32_t n_cols, const double* X0, const double* X1,
                         const double* X2, int use_minb, RunState* st, double* blockpart,
                         bool dd, cudaStream_t s, int64_t* launches);

// dep[2b], dep[2b+1] = first and last CTA owning an x position that a
// non-zero of CTA b's slices of the (permuted) matrix reads.
cudaError_t launch_dependencies(const int32_t* wp, const int32_t* col, const double* val,
                                const int32_t* part_a, const int32_t* part_t, int G,
                                int32_t* dep, cudaStream_t s, int64_t* launches);

int persistent32_max_blocks(int* blocks_per_sm);
cudaError_t launch_persistent32(const IterParams32& p, int G, cudaStream_t s, int64_t* launches);

// Power-of-two equilibration (the paper's row then column 2-norm scaling,
// each factor rounded to the nearest power of two), computed with the same
// operation order as the CPU oracle: d_row from CSR(A), d_col from the
// transpose (entries in row order) of D_row^-1 A.
cudaError_t launch_equilibrate(int32_t n_rows, int32_t n_cols, const int32_t* rp,
                               const double* va, const int32_t* rpt, const int32_t* cit,
                               const double* vat, double* d_row, double* d_col, cudaStream_t s,
                               int64_t* launches);
// ---- Algorithm 2 (sigma_min through ||A^{-1}|| with given LU factors) ----
// One triangular system T x = b in level-scheduled, column-level form.  A
// row's level is one more than the highest level of the rows it depends on.
// Each row's off-diagonal entries are split into segments by the level of
// their column; the segment whose columns are at level l is applied in step l
// (l = 0 .. nproc-1, nproc = levels - 1), when those x_j are final:
//   x_i <- x_i + sum_{j in segment} va_ij x_j,  va_ij = -T_ij / T_ii,
// starting from x_i = b_i / T_ii (dinv), so a row is final after its last
// segment and no step needs a division or a subtraction.  Step l's items
// (one per segment) are items[linfo[l].x .. linfo[l].y & kItemMask); a
// one-entry segment is the item {row, column, value as two words}, a longer
// one {~row, first entry, end entry, 0} with its entries in ci/va, and step
// l's entries are ci/va[linfo[l].z .. linfo[l].w).  Bits 27.. of linfo[l].y
// hold log2 of the lanes per item.  ci/va are padded so that 16-byte windows
// around any step's entries stay inside.
constexpr int kItemMask = (1 << 27) - 1;
struct TriSys {
  int32_t nproc;
  int32_t max_items;   // most items in one step
  int32_t max_ent;     // largest 16-byte window of one step's entries
  const double* dinv;  // [n] 1 / T_ii
  const int4* linfo;   // [nproc]
  const int4* items;
  const int32_t* ci;
  const double* va;
};
// Algorithm 1 on B = A^{-1} = Q U^{-1} L^{-1} P, everything in source order.
struct LuParams {
  int32_t n;
  TriSys L, U, Ut, Lt;       // L t = P x, U u = t, U^T a = u, L^T c = a
  const int32_t* p;          // [n] row i of P A is row p[i] of A (null = identity)
  double* x; double* xmin;   // iterate, tracked maximiser of ||B x|| / ||x||
  double* m; double* v; double* dx;
  double* w;                 // s = P^T c
  double* y;                 // the solve vector when it is not in shared memory
  const double2* bias;       // as IterParams
  double* L_trace; double* x_trace; int n_trace;
  RunState* st;
  int iters, t0;
  double beta1, beta2;
  int smem_mode;             // 1: the solve vector in shared memory; 0: in global
  int slot_items, slot_ent;  // items and entries one staging slot holds
};
constexpr int kLuThreads = 512;
constexpr size_t kLuSmemBudget = 218 * 1024;  // dynamic shared memory the LU kernel may use
// Chooses p->smem_mode and the slot sizes from n and the factors' largest steps;
// returns the item's dynamic shared memory.
size_t lu_layout(LuParams* p);
// Items (device array of n_items LuParams, each with its own vectors and run
// state), one CTA each; smem = the dynamic shared memory of the launch, which
// must cover lu_layout() of every item; all_smem: every item has smem_mode 1
// (else all items run with their solve vector in global memory).
cudaError_t launch_lu_iter(const LuParams* items_dev, int n_items, size_t smem, bool all_smem,
                           cudaStream_t s, int64_t* launches);
// ---- Algorithm 2 on the whole grid (pa_lu_grid.cu), for large factors ----
// One triangular system in row form: row i's off-diagonal entries
// ci/va[rp[i] .. rp[i+1]) with va_ij = -T_ij / T_ii, and dinv_i = 1 / T_ii.
// order: the rows sorted by level (lower: row i depends on j < i; upper: on
// j > i), the sequence the grid kernel's warps take them in.
struct TriRows {
  const int32_t* rp;
  const int32_t* ci;
  const double* va;
  const double* dinv;
  const int32_t* order;
};
struct TriRowsHost {
  std::vector<int32_t> rp, ci, order;
  std::vector<double> va, dinv;
};
// Row form of a triangular CSR whose diagonal entries are present and non-zero
// (tri_analyse checks that first).
void tri_rows_host(int32_t n, const int32_t* rp, const int32_t* ci, const double* va, bool lower,
                   TriRowsHost* out);
struct LuGridParams {
  int32_t n;
  TriRows sys[4];            // L, U, U^T, L^T (lower, upper, lower, upper)
  const int32_t* p;          // row permutation of P A = L U Q^T (null = identity)
  double *x, *xmin, *m, *v, *dx, *w;
  double* y[4];              // the four solve vectors
  double* partials;          // [G][4]
  const double2* bias;
  double* L_trace; double* x_trace; int n_trace;
  RunState* st;
  int iters, t0;
  double beta1, beta2;
  long long timeout_ns;
};
int lu_grid_max_blocks();
cudaError_t launch_lu_grid(const LuGridParams& p, int G, cudaStream_t s, int64_t* launches);

// Host analysis for TriSys: checks triangularity and non-zero diagonals,
// computes the levels and builds the step lists.  lower: row i depends on
// columns j < i; else on j > i.  Returns an empty string or the reason the
// factor is unusable.
struct TriHost {
  int32_t nproc = 0, max_items = 0, max_ent = 0;
  std::vector<double> dinv, va;
  std::vector<int4> linfo, items;
  std::vector<int32_t> ci;
};
std::string tri_analyse(int32_t n, const int32_t* rp, const int32_t* ci, const double* va,
                        bool lower, TriHost* out);
// CSR of T^T; entries of each row in increasing (reverse = false) or
// decreasing (reverse = true) order of their source row.
void csr_transpose_host(int32_t n, const int32_t* rp, const int32_t* ci, const double* va,
                        bool reverse, std::vector<int32_t>* trp, std::vector<int32_t>* tci,
                        std::vector<double>* tva);

// Residual norms of an approximate solution and the bounds of Theorems 1-4
// into out[10] (device); part holds 3 * error_bound_blocks(max(n_rows,
// n_cols)) doubles.
constexpr int kErrorBoundMaxBlocks = 1216;
int error_bound_blocks(int64_t n);
cudaError_t launch_error_bounds(int32_t n_rows, int32_t n_cols, const int32_t* rp,
                                const int32_t* ci, const double* va, const double* x_hat,
                                const double* b, double kappa, double norm_a, double u,
                                double* part, double* out, cudaStream_t s, int64_t* launches);
// A := D_row^-1 A D_col^-1 in place, in the CSR of A and in that of A^T
// (power-of-two factors: exact).
cudaError_t launch_scale_csr(int32_t n_rows, int32_t n_cols, const int32_t* rp,
                             const int32_t* ci, double* va, const int32_t* rpt,
                             const int32_t* cit, double* vat, const double* d_row,
                             const double* d_col, cudaStream_t s, int64_t* launches);
// out[p] = (float) d[perm[p]] for p < n (permuted factors), and flags in
// *range_flag (bit 1) any factor outside the FP32 normal range.
cudaError_t launch_permute_factors(int32_t n, const int32_t* perm, const double* d, float* out,
                                   int* range_flag, cudaStream_t s, int64_t* launches);
// FP32 values of the sliced equilibrated matrix: val32[e] = (float)(val[e] /
// drow[row position] / dcol[column position]) for every slice entry of m.
cudaError_t launch_sell_scale32(const Sell& m, const float* d_rowpos, const float* d_colpos,
                                float* val32, cudaStream_t s, int64_t* launches);
cudaError_t launch_convert(int64_t n, const float* in, double* out, cudaStream_t s,
                           int64_t* launches);
cudaError_t launch_convert(int64_t n, const double* in, float* out, cudaStream_t s,
                           int64_t* launches);

// Persistent cooperative Projected Adam run (Algorithm 1) over a grid of G
// CTAs; dd selects compensated (double-double) products.
int persistent_max_blocks(int loss, bool dd, int* blocks_per_sm);
// The cluster variant: one thread-block cluster of G CTAs, synchronised by
// the hardware cluster barrier (plain FP64 products).
int persistent_cluster_max(int loss);
cudaError_t launch_persistent_cluster(const IterParams& p, int loss, int G, cudaStream_t s,
                                      int64_t* launches);
cudaError_t launch_persistent(const IterParams& p, int loss, bool dd, int G, cudaStream_t s,
                              int64_t* launches);

// The merged-phase persistent kernel: the normalisation of iteration t is
// folded into the product of iteration t+1 (one full grid barrier and one
// split barrier per iteration).  df selects the double-float variant
// (log-ratio loss only).  Internal status for a double-float run whose
// scalars left the range the variant supports (the caller reruns in FP64):
constexpr int kStatusDfRange = -100;
int merged_max_blocks(int loss, bool df);
cudaError_t launch_merged(const IterParams& p, int loss, bool df, int G, cudaStream_t s,
                          int64_t* launches);
// Double-float set-up: the largest and smallest non-zero binary exponents
// of |vals| (out[0] = max, out[1] = min; out must hold {INT_MIN, INT_MAX}),
// the split of 2^-k vals into (hi, lo) pairs, and vector conversions.
cudaError_t launch_exp_range(int64_t n, const double* vals, int* out, cudaStream_t s,
                             int64_t* launches);
cudaError_t launch_split_df(int64_t n, const double* in, int k, float2* out, cudaStream_t s,
                            int64_t* launches);
cudaError_t launch_join_df(int64_t n, const float2* in, double* out, cudaStream_t s,
                           int64_t* launches);

}  // namespace pa
