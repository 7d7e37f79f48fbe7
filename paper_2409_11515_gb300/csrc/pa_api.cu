// pa_api.cu -- host runtime behind include/pa.h: handles, argument and CSR
// validation, device memory, the start vector, launch orchestration of the
// persistent Projected Adam kernel, and result read-back.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <climits>
#include <mutex>
#include <string>
#include <chrono>
#include <map>
#include <vector>

#include "pa_device.cuh"
#include "pa_internal.h"
#include "pa_lu_cluster.h"

using namespace pa;

// NVTX range around each entry point (visible in Nsight timelines; free when
// no tool is attached: the header-only NVTX loads its injection library only
// when a profiler asks for it).
namespace {
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace

// ------------------------------------------------------------ errors --

static thread_local std::string g_err;

static pa_status fail(pa_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

static pa_status cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation)
    return fail(PA_ERR_OOM, "%s: out of device memory", what);
  return fail(PA_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                              \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

extern "C" const char* pa_last_error(void) { return g_err.c_str(); }

pa_status pa::set_error(pa_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

// --------------------------------------------------------- allocator --

static pa_alloc_fn g_alloc = nullptr;
static pa_free_fn g_free = nullptr;
static void* g_alloc_ctx = nullptr;

extern "C" void pa_set_allocator(pa_alloc_fn alloc, pa_free_fn free_fn, void* ctx) {
  g_alloc = alloc;
  g_free = free_fn;
  g_alloc_ctx = ctx;
}

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct pa_ctx {
  cudaStream_t stream = nullptr;
  pa_alloc_fn alloc = nullptr;
  pa_free_fn free_fn = nullptr;
  void* alloc_ctx = nullptr;
  pa_options opt{};
  int32_t n_rows = 0, n_cols = 0;
  int64_t nnz = 0;
  int64_t launches = 0;
  std::vector<DevBuf> bufs;  // everything allocated, freed in pa_destroy

  // matrix: CSR of A and of A^T (source order), and the sliced-ELL copies
  // P A Q^T (sa) and Q A^T P^T (st_) that the kernels iterate over
  int32_t *rp = nullptr, *ci = nullptr, *rpt = nullptr, *cit = nullptr;
  double *va = nullptr, *vat = nullptr;
  Sell sa, sq;

  // run buffers (sized for n = max(n_rows, n_cols))
  bool run_ready = false;
  double *X0 = nullptr, *X1 = nullptr, *X2 = nullptr, *Xinit = nullptr;
  double *m = nullptr, *v = nullptr, *y = nullptr, *ylo = nullptr, *dx = nullptr;
  double *partials = nullptr, *blockpart = nullptr;
  double *eb_part = nullptr, *eb_out = nullptr;  // pa_error_bounds scratch
  // Algorithm 2: the attached factors in level-scheduled form
  bool have_lu = false, have_min_lu = false, have_min_direct = false;
  TriSys lu_sys[4] = {};          // L, U, U^T, L^T
  TriRows lu_rows[4] = {};        // the same systems in row form (the grid kernel)
  double* lu_y4 = nullptr;        // the grid kernel's four solve vectors [4][n]
  double* lu_part = nullptr;      // its per-CTA partial sums
  int lu_part_G = 0;
  int lu_last_kernel = -1;        // 0: one CTA (level steps), 1: the grid (row waits), 2: a cluster
  LcSys lc_sys[4] = {};           // the four systems in the cluster kernel's form
  LcPlan lc_plan;                 // its cluster, vector slots and staging slots
  bool lc_ready = false;          // lc_sys built (for lc_plan)
  int lu_route = 0;               // the route of the next LU run: 0 one CTA, 1 grid, 2 cluster
  int32_t* lu_p = nullptr;        // row permutation (null = identity)
  std::vector<void*> lu_bufs;     // device arrays of the factors
  double* xmin_lu = nullptr;      // x_min of the latest LU-route run (source order)
  double *lu_w = nullptr, *lu_y = nullptr;  // s = P^T c, the solve vector (global fallback)
  LuParams* lu_params = nullptr;  // device copy of the latest run's parameters
  double *xmin_max = nullptr, *xmin_min = nullptr;
  RunState* st = nullptr;
  int G = 0;
  int32_t *part_a = nullptr, *part_t = nullptr, *dep = nullptr;
  // each CTA's slices dealt to its warps by cost, longest first to the least
  // loaded warp: warp w of CTA b takes list[woff[b (NW+1) + w] .. woff[.. + 1])
  int32_t *a_list = nullptr, *a_woff = nullptr, *t_list = nullptr, *t_woff = nullptr;
  std::vector<int32_t> wpa_h, wpt_h;  // host copies of the slice pointers
  unsigned* ready = nullptr;
  unsigned long long* cta_ns = nullptr;  // [2G] per-CTA busy time of the last run
  unsigned long long* cta_lat = nullptr; // [G] per-CTA phase-A completion latency
  int last_G = 0;
  int tuned_rounds = 0;                  // tuner rounds done for h->G
  double tune_best = INFINITY;           // fastest per-iteration time seen while tuning
  std::vector<int32_t> tune_best_a, tune_best_t;  // the partitions of that run
  cudaEvent_t tune_ev[2] = {nullptr, nullptr};
  float last_run_ms = 0.f;               // the latest timed grid run
  std::map<int, int> batch_kb;           // tuned restart-block width per k (batched engine)
  double2* bias = nullptr;
  int bias_cap = 0;
  bool have_max = false, have_min = false;
  double sigma_max = NAN, sigma_min = NAN;

  // power-of-two equilibration (source order, FP64) and the FP32 copies the
  // mixed-precision sigma_max kernel iterates over
  double *d_row = nullptr, *d_col = nullptr;
  double *tgt_row = nullptr, *tgt_col = nullptr;  // PA_EQ_TARGET: A_hat = D_r^-1 A D_c^-1
  float *drp32 = nullptr, *dcp32 = nullptr, *a_val32 = nullptr, *t_val32 = nullptr;
  float *X0f = nullptr, *X1f = nullptr, *X2f = nullptr, *Wf = nullptr;
  float *mf = nullptr, *vf = nullptr, *yf = nullptr, *dxf = nullptr;
  int64_t a_entries = 0, t_entries = 0;  // padded entries of the sliced copies

  // PA_DF64: values of 2^-df_k P A Q^T and its transpose as (hi, lo) float
  // pairs, the vectors in the same form, and the bias table as pairs
  bool df_ok = false;     // the matrix's exponent range fits the variant
  bool df_checked = false;  // the range was measured (and the values split if it fits)
  int df_k = 0;
  float2 *a_val2 = nullptr, *t_val2 = nullptr;
  float2 *XD0 = nullptr, *XD1 = nullptr, *XD2 = nullptr;
  float2 *ud = nullptr, *md = nullptr, *vd = nullptr, *yd = nullptr;
  float4* bias2 = nullptr;
  int df_fallbacks = 0;   // double-float runs redone in FP64 (range)
  int last_kernel = -1;   // kernel of the latest single-vector run (pa_last_run_info)
  int last_refreshes = 0;
  // the state pa_continue resumes: the latest FP64 run of the three-phase or
  // cluster kernel (x_T in X[cur], x_min in X[minb], m, v, the tracked minimum)
  struct Cont {
    bool valid = false;
    int mode = 0, t_done = 0, t_min = 0, have_best = 0, cur = 0, minb = 0, G = 0;
    bool cluster = false;
    double best_s = 0, best_q = 0, lr = 0, b1 = 0, b2 = 0, eps = 0;
  } cont;
  // the single-pass engine (PA_ENGINE_SINGLE): its partition (rows and x
  // positions alike), the owners of each window's columns (sp_dep), the CTAs
  // whose windows meet each CTA's positions (sp_rdep), its warp lists and the
  // per-CTA window plans, built for sp_G CTAs
  int sp_G = 0;
  int32_t *sp_part = nullptr, *sp_dep = nullptr, *sp_rdep = nullptr;
  int32_t *sp_list = nullptr, *sp_lwoff = nullptr;
  int32_t *sp_cmin = nullptr, *sp_woff = nullptr, *sp_goff = nullptr, *sp_gp = nullptr;
  int32_t* sp_gcol = nullptr;
  uint32_t* sp_ent = nullptr;
  double* sp_halo = nullptr;
  int64_t sp_window_cols = 0, sp_plan_entries = 0, sp_plan_slots = 0, sp_groups = 0;
  // the launch-shape tuner's choice for plain FP64 runs of the AUTO engine:
  // kernel (0 three-phase, 1 merged-phase, 6 single-pass) and CTAs; source 1
  // = this handle's trials, 2 = the cache of an earlier handle of the same
  // matrix; the trial candidates and their times
  int launch_kernel = -1, launch_G = 0, launch_source = 0;
  std::vector<std::array<int, 2>> launch_cands;
  std::vector<double> launch_ms;
};

static void* dev_alloc(pa_ctx* h, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~(size_t)255;
  void* p = nullptr;
  if (h->alloc) {
    p = h->alloc(bytes, (void*)h->stream, h->alloc_ctx);
  } else if (cudaMallocAsync(&p, bytes, h->stream) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) h->bufs.push_back({p, bytes});
  return p;
}

template <class T>
static pa_status alloc_n(pa_ctx* h, T** out, size_t count, const char* what) {
  *out = (T*)dev_alloc(h, sizeof(T) * count);
  if (!*out) return fail(PA_ERR_OOM, "out of device memory allocating %s (%zu bytes)", what,
                         sizeof(T) * count);
  return PA_OK;
}

static void dev_free(pa_ctx* h, void* p) {
  for (size_t i = 0; i < h->bufs.size(); ++i) {
    if (h->bufs[i].p == p) {
      if (h->free_fn) h->free_fn(p, h->bufs[i].bytes, (void*)h->stream, h->alloc_ctx);
      else cudaFreeAsync(p, h->stream);
      h->bufs.erase(h->bufs.begin() + i);
      return;
    }
  }
}

extern "C" void pa_options_default(pa_options* opt) {
  if (!opt) return;
  memset(opt, 0, sizeof *opt);
  opt->loss = PA_LOSS_LOGRATIO;
  opt->precision = PA_FP64;
  opt->equilibrate = PA_EQ_NONE;
  opt->engine = PA_ENGINE_AUTO;
  opt->barrier_timeout_ns = 2000000000LL;
  opt->fp64_tail = -1;
}

extern "C" void pa_destroy(pa_handle h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  for (auto& b : h->bufs) {
    if (h->free_fn) h->free_fn(b.p, b.bytes, (void*)h->stream, h->alloc_ctx);
    else cudaFreeAsync(b.p, h->stream);
  }
  cudaStreamSynchronize(h->stream);
  for (cudaEvent_t ev : h->tune_ev)
    if (ev) cudaEventDestroy(ev);
  delete h;
}

extern "C" int64_t pa_kernel_launches(pa_handle h) { return h ? h->launches : -1; }

// Sliced ELL copies P A Q^T and Q A^T P^T: P sorts the rows of A and Q the
// rows of A^T (the columns of A) by length inside kWindow-row windows.
static pa_status build_one_sell(pa_ctx* h, int32_t n_rows, const int32_t* rp, const int32_t* ci,
                                const double* va, const int32_t* lens, const int32_t* col_pos,
                                Sell* out) {
  pa_status st;
  const int32_t ns = sell_slices(n_rows);
  int32_t *widths = nullptr, *bsums = nullptr;
  if ((st = alloc_n(h, &out->wp, (size_t)ns + 1, "slice pointers")) ||
      (st = alloc_n(h, &widths, (size_t)ns + 1, "slice widths")) ||
      (st = alloc_n(h, &bsums, (size_t)scan_blocks((int64_t)ns + 1) + 1, "scan scratch")))
    return st;
  int64_t total = 0;
  cudaError_t e = launch_sell_build(n_rows, rp, ci, va, lens, col_pos, out, widths, bsums, &total,
                                    h->stream, &h->launches);
  if (e != cudaSuccess) return cuda_fail(e, "building slice widths");
  dev_free(h, widths);
  dev_free(h, bsums);
  if ((st = alloc_n(h, &out->col, (size_t)total + 32, "sliced columns")) ||
      (st = alloc_n(h, &out->val, (size_t)total + 32, "sliced values")))
    return st;
  if (out == &h->sa) h->a_entries = total; else h->t_entries = total;
  e = launch_sell_fill(n_rows, rp, ci, va, lens, col_pos, *out, h->stream, &h->launches);
  if (e != cudaSuccess) return cuda_fail(e, "filling the sliced matrix");
  return PA_OK;
}

static pa_status build_sell(pa_ctx* h) {
  pa_status st;
  int32_t *lens_a = nullptr, *lens_t = nullptr;
  if ((st = alloc_n(h, &lens_a, (size_t)h->n_rows, "row lengths")) ||
      (st = alloc_n(h, &lens_t, (size_t)h->n_cols, "column lengths")) ||
      (st = alloc_n(h, &h->sa.perm, (size_t)h->n_rows, "row permutation")) ||
      (st = alloc_n(h, &h->sa.pos, (size_t)h->n_rows, "row permutation")) ||
      (st = alloc_n(h, &h->sq.perm, (size_t)h->n_cols, "column permutation")) ||
      (st = alloc_n(h, &h->sq.pos, (size_t)h->n_cols, "column permutation")))
    return st;
  cudaError_t e;
  if ((e = launch_row_lengths(h->n_rows, h->rp, h->va, lens_a, h->stream, &h->launches)) ||
      (e = launch_row_lengths(h->n_cols, h->rpt, h->vat, lens_t, h->stream, &h->launches)) ||
      (e = launch_window_sort(h->n_rows, lens_a, h->sa.perm, h->sa.pos, h->stream, &h->launches)) ||
      (e = launch_window_sort(h->n_cols, lens_t, h->sq.perm, h->sq.pos, h->stream, &h->launches)))
    return cuda_fail(e, "sorting rows by length");
  // P A Q^T: rows of A in P order, column j of A lands at x position Q(j)
  if ((st = build_one_sell(h, h->n_rows, h->rp, h->ci, h->va, lens_a, h->sq.pos, &h->sa)))
    return st;
  // Q A^T P^T: rows of A^T in Q order, row i of A lands at y position P(i)
  if ((st = build_one_sell(h, h->n_cols, h->rpt, h->cit, h->vat, lens_t, h->sa.pos, &h->sq)))
    return st;
  if ((e = cudaStreamSynchronize(h->stream))) return cuda_fail(e, "building the sliced matrices");
  dev_free(h, lens_a);
  dev_free(h, lens_t);
  return PA_OK;
}

// Power-of-two equilibration D_r, D_c (source order), and for the mixed
// precision mode the permuted FP32 factors and FP32 values of the sliced
// copies of D_r^-1 A D_c^-1.
static pa_status build_equilibration(pa_ctx* h, bool fp32_copies) {
  pa_status st;
  if ((st = alloc_n(h, &h->d_row, (size_t)h->n_rows, "row scaling")) ||
      (st = alloc_n(h, &h->d_col, (size_t)h->n_cols, "column scaling")))
    return st;
  cudaError_t e = launch_equilibrate(h->n_rows, h->n_cols, h->rp, h->va, h->rpt, h->cit, h->vat,
                                     h->d_row, h->d_col, h->stream, &h->launches);
  if (e != cudaSuccess) return cuda_fail(e, "equilibrating");
  if (!fp32_copies) return PA_OK;
  int* flag = nullptr;
  if ((st = alloc_n(h, &h->drp32, (size_t)h->n_rows, "row scaling (FP32)")) ||
      (st = alloc_n(h, &h->dcp32, (size_t)h->n_cols, "column scaling (FP32)")) ||
      (st = alloc_n(h, &h->a_val32, (size_t)h->a_entries + 32, "FP32 values")) ||
      (st = alloc_n(h, &h->t_val32, (size_t)h->t_entries + 32, "FP32 values")) ||
      (st = alloc_n(h, &flag, 1, "flag")))
    return st;
  int hflag = 0;
  if ((e = cudaMemsetAsync(flag, 0, sizeof(int), h->stream)) ||
      (e = launch_permute_factors(h->n_rows, h->sa.perm, h->d_row, h->drp32, flag, h->stream,
                                  &h->launches)) ||
      (e = launch_permute_factors(h->n_cols, h->sq.perm, h->d_col, h->dcp32, flag, h->stream,
                                  &h->launches)) ||
      (e = launch_sell_scale32(h->sa, h->drp32, h->dcp32, h->a_val32, h->stream, &h->launches)) ||
      (e = launch_sell_scale32(h->sq, h->dcp32, h->drp32, h->t_val32, h->stream, &h->launches)) ||
      (e = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream)) ||
      (e = cudaStreamSynchronize(h->stream)))
    return cuda_fail(e, "building the FP32 equilibrated copies");
  dev_free(h, flag);
  if (hflag)
    return fail(PA_ERR_UNSUPPORTED,
                "mixed precision: an equilibration factor lies outside the FP32 normal range");
  return PA_OK;
}

// ---------------------------------------------------------- pa_create --

extern "C" pa_status pa_create(pa_handle* out, int32_t n_rows, int32_t n_cols, int64_t nnz,
                               const int32_t* row_ptr, const int32_t* col_idx, const double* vals,
                               int ptr_kind, const pa_options* opt, void* cuda_stream) {
  NvtxRange nvtx_range("pa_create");
  g_err.clear();
  if (!out) return fail(PA_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n_rows < 0 || n_cols < 0 || nnz < 0)
    return fail(PA_ERR_INVALID_ARG, "negative size (n_rows=%d n_cols=%d nnz=%lld)", n_rows, n_cols,
                (long long)nnz);
  if (n_rows == 0 || n_cols == 0)
    return fail(PA_ERR_INVALID_ARG, "empty matrix (%d x %d)", n_rows, n_cols);
  if (nnz > 2147483647LL) return fail(PA_ERR_INVALID_ARG, "nnz %lld exceeds int32 CSR", (long long)nnz);
  if (!row_ptr || (nnz > 0 && (!col_idx || !vals)))
    return fail(PA_ERR_INVALID_ARG, "NULL CSR array");
  if (ptr_kind != PA_HOST && ptr_kind != PA_DEVICE)
    return fail(PA_ERR_INVALID_ARG, "ptr_kind must be PA_HOST or PA_DEVICE");
  pa_options o;
  pa_options_default(&o);
  if (opt) o = *opt;
  if (o.barrier_timeout_ns <= 0) o.barrier_timeout_ns = 2000000000LL;
  if (o.loss != PA_LOSS_LOGRATIO && o.loss != PA_LOSS_QUADRATIC)
    return fail(PA_ERR_INVALID_ARG, "unknown loss %d", o.loss);
  if (o.precision != PA_FP64 && o.precision != PA_MIXED && o.precision != PA_DF64)
    return fail(PA_ERR_INVALID_ARG, "unknown precision mode %d", o.precision);
  if (o.engine < PA_ENGINE_AUTO || o.engine > PA_ENGINE_SINGLE)
    return fail(PA_ERR_INVALID_ARG, "unknown engine %d", o.engine);
  if (o.equilibrate != PA_EQ_NONE && o.equilibrate != PA_EQ_STORAGE &&
      o.equilibrate != PA_EQ_TARGET)
    return fail(PA_ERR_INVALID_ARG, "unknown equilibration mode %d", o.equilibrate);
  if (o.precision == PA_MIXED && o.loss != PA_LOSS_LOGRATIO)
    return fail(PA_ERR_UNSUPPORTED, "mixed precision supports the log-ratio loss only");
  if (o.autotune < 0) return fail(PA_ERR_INVALID_ARG, "autotune must be >= 0 (got %d)", o.autotune);
  // TARGET replaces A by A_hat once at creation; the handle then treats A_hat
  // like any input (MIXED adds its own STORAGE copies of it)
  const bool target = o.equilibrate == PA_EQ_TARGET;
  if (o.precision == PA_MIXED) o.equilibrate = PA_EQ_STORAGE;
  else if (target) o.equilibrate = PA_EQ_NONE;

  pa_ctx* h = new pa_ctx();
  h->stream = (cudaStream_t)cuda_stream;
  h->alloc = g_alloc;
  h->free_fn = g_free;
  h->alloc_ctx = g_alloc_ctx;
  h->opt = o;
  h->n_rows = n_rows;
  h->n_cols = n_cols;
  h->nnz = nnz;
  pa_status st = PA_OK;
  auto bail = [&](pa_status s) {
    pa_destroy(h);
    return s;
  };
  // +4 entries of padding on the nnz arrays keeps every vector load in bounds
  if ((st = alloc_n(h, &h->rp, (size_t)n_rows + 1, "row_ptr")) ||
      (st = alloc_n(h, &h->ci, (size_t)nnz + 4, "col_idx")) ||
      (st = alloc_n(h, &h->va, (size_t)nnz + 4, "values")) ||
      (st = alloc_n(h, &h->rpt, (size_t)n_cols + 1, "row_ptr of A^T")) ||
      (st = alloc_n(h, &h->cit, (size_t)nnz + 4, "col_idx of A^T")) ||
      (st = alloc_n(h, &h->vat, (size_t)nnz + 4, "values of A^T")))
    return bail(st);
  const cudaMemcpyKind kind = ptr_kind == PA_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(h->rp, row_ptr, sizeof(int32_t) * ((size_t)n_rows + 1), kind, h->stream)) ||
      (nnz && (e = cudaMemcpyAsync(h->ci, col_idx, sizeof(int32_t) * nnz, kind, h->stream))) ||
      (nnz && (e = cudaMemcpyAsync(h->va, vals, sizeof(double) * nnz, kind, h->stream))) ||
      (e = cudaMemsetAsync(h->ci + nnz, 0, sizeof(int32_t) * 4, h->stream)) ||
      (e = cudaMemsetAsync(h->va + nnz, 0, sizeof(double) * 4, h->stream)))
    return bail(cuda_fail(e, "copying the CSR arrays"));

  // validate on the device before any kernel walks the rows
  int* flag = nullptr;
  if ((st = alloc_n(h, &flag, 1, "flag"))) return bail(st);
  if ((e = cudaMemsetAsync(flag, 0, sizeof(int), h->stream)) ||
      (e = launch_validate_csr(n_rows, n_cols, nnz, h->rp, h->ci, flag, h->stream, &h->launches)))
    return bail(cuda_fail(e, "validating the CSR"));
  int hflag = 0;
  if ((e = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream)) ||
      (e = cudaStreamSynchronize(h->stream)))
    return bail(cuda_fail(e, "validating the CSR"));
  if (hflag) {
    return bail(fail(PA_ERR_INVALID_CSR, "invalid CSR:%s%s%s",
                     (hflag & 1) ? " row_ptr[0] != 0 or row_ptr[n_rows] != nnz;" : "",
                     (hflag & 2) ? " row_ptr decreases;" : "",
                     (hflag & 4) ? " column index out of range;" : ""));
  }
  dev_free(h, flag);

  // explicit CSR of A^T (stable: entries of each row of A^T in row order of A)
  int32_t *cursor = nullptr, *src = nullptr, *rowid = nullptr, *bsums = nullptr;
  if ((st = alloc_n(h, &cursor, (size_t)n_cols + 1, "transpose scratch")) ||
      (st = alloc_n(h, &src, (size_t)nnz + 1, "transpose scratch")) ||
      (st = alloc_n(h, &rowid, (size_t)nnz + 1, "transpose scratch")) ||
      (st = alloc_n(h, &bsums, (size_t)scan_blocks((int64_t)n_cols) + 1, "transpose scratch")))
    return bail(st);
  if ((e = launch_transpose(n_rows, n_cols, nnz, h->rp, h->ci, h->va, h->rpt, h->cit, h->vat,
                            cursor, src, rowid, bsums, nullptr, h->stream, &h->launches)) ||
      (e = cudaMemsetAsync(h->cit + nnz, 0, sizeof(int32_t) * 4, h->stream)) ||
      (e = cudaMemsetAsync(h->vat + nnz, 0, sizeof(double) * 4, h->stream)) ||
      (e = cudaStreamSynchronize(h->stream)))
    return bail(cuda_fail(e, "building the transpose"));
  dev_free(h, cursor);
  dev_free(h, src);
  dev_free(h, rowid);
  dev_free(h, bsums);
  if (target) {
    if ((st = alloc_n(h, &h->tgt_row, (size_t)n_rows, "row scaling")) ||
        (st = alloc_n(h, &h->tgt_col, (size_t)n_cols, "column scaling")))
      return bail(st);
    if ((e = launch_equilibrate(n_rows, n_cols, h->rp, h->va, h->rpt, h->cit, h->vat, h->tgt_row,
                                h->tgt_col, h->stream, &h->launches)) ||
        (e = launch_scale_csr(n_rows, n_cols, h->rp, h->ci, h->va, h->rpt, h->cit, h->vat,
                              h->tgt_row, h->tgt_col, h->stream, &h->launches)))
      return bail(cuda_fail(e, "equilibrating the target matrix"));
  }
  if ((st = build_sell(h))) return bail(st);
  if (o.equilibrate == PA_EQ_STORAGE &&
      (st = build_equilibration(h, o.precision == PA_MIXED)))
    return bail(st);
  *out = h;
  return PA_OK;
}

// ------------------------------------------------------------- runs --

// PA_DF64 set-up: the binary exponent range of the sliced values decides
// whether the double-float variant applies (2^-k A with max |a| in [1/2, 1)
// must keep every non-zero above 2^-100, so that its low part stays a normal
// float); if so, the (hi, lo) copies of both sliced matrices and the vectors.
// The double-float values (PA_DF64): the exponent range of the sliced
// values decides whether the variant can take the matrix (df_ok); if so, the
// values of 2^-k P A Q^T and of its transpose as (hi, lo) pairs.  Once per
// handle; shared by the single-vector and the batched kernels.
static pa_status build_df_values(pa_ctx* h) {
  if (h->df_checked) return PA_OK;
  pa_status st;
  int* rng = nullptr;
  if ((st = alloc_n(h, &rng, 2, "exponent range"))) return st;
  const int init[2] = {INT_MIN, INT_MAX};
  int got[2] = {0, 0};
  cudaError_t e;
  if ((e = cudaMemcpyAsync(rng, init, sizeof init, cudaMemcpyHostToDevice, h->stream)) ||
      (e = launch_exp_range(h->a_entries, h->sa.val, rng, h->stream, &h->launches)) ||
      (e = cudaMemcpyAsync(got, rng, sizeof got, cudaMemcpyDeviceToHost, h->stream)) ||
      (e = cudaStreamSynchronize(h->stream)))
    return cuda_fail(e, "measuring the value range");
  dev_free(h, rng);
  h->df_ok = false;
  h->df_checked = true;
  if (h->opt.loss != PA_LOSS_LOGRATIO || got[0] == INT_MIN || got[0] >= 2047 || got[1] < 1 ||
      got[0] - got[1] > 99)
    return PA_OK;  // runs use the FP64 kernels
  h->df_k = got[0] - 1022;  // 2^-k max|a| lies in [1/2, 1)
  if (h->df_k < -400 || h->df_k > 400) return PA_OK;
  if ((st = alloc_n(h, &h->a_val2, (size_t)h->a_entries + 32, "values (double-float)")) ||
      (st = alloc_n(h, &h->t_val2, (size_t)h->t_entries + 32, "values (double-float)")))
    return st;
  if ((e = launch_split_df(h->a_entries, h->sa.val, h->df_k, h->a_val2, h->stream, &h->launches)) ||
      (e = launch_split_df(h->t_entries, h->sq.val, h->df_k, h->t_val2, h->stream, &h->launches)))
    return cuda_fail(e, "splitting the values");
  h->df_ok = true;
  return PA_OK;
}

// The values and the single-vector kernel's double-float vectors.
static pa_status build_df(pa_ctx* h) {
  pa_status st;
  if ((st = build_df_values(h)) || !h->df_ok) return st;
  const size_t n = (size_t)std::max(h->n_rows, h->n_cols);
  if ((st = alloc_n(h, &h->XD0, n, "iterate (double-float)")) ||
      (st = alloc_n(h, &h->XD1, n, "iterate (double-float)")) ||
      (st = alloc_n(h, &h->XD2, n, "iterate (double-float)")) ||
      (st = alloc_n(h, &h->ud, n, "u (double-float)")) ||
      (st = alloc_n(h, &h->md, n, "first moment (double-float)")) ||
      (st = alloc_n(h, &h->vd, n, "second moment (double-float)")) ||
      (st = alloc_n(h, &h->yd, (size_t)std::max(h->n_rows, 1), "A x (double-float)")))
    return st;
  return PA_OK;
}

static pa_status ensure_run_buffers(pa_ctx* h) {
  if (h->run_ready) return PA_OK;
  const size_t n = (size_t)std::max(h->n_rows, h->n_cols);
  pa_status st;
  if ((st = alloc_n(h, &h->X0, n, "iterate")) || (st = alloc_n(h, &h->X1, n, "iterate")) ||
      (st = alloc_n(h, &h->X2, n, "iterate")) || (st = alloc_n(h, &h->Xinit, n, "x_init")) ||
      (st = alloc_n(h, &h->m, n, "first moment")) || (st = alloc_n(h, &h->v, n, "second moment")) ||
      (st = alloc_n(h, &h->y, (size_t)h->n_rows, "A x")) ||
      (st = alloc_n(h, &h->dx, n, "step")) ||
      (st = alloc_n(h, &h->xmin_max, (size_t)h->n_cols, "x_min")) ||
      (st = alloc_n(h, &h->xmin_min, (size_t)h->n_cols, "x_min")) ||
      (st = alloc_n(h, &h->st, 1, "run state")) ||
      (st = alloc_n(h, &h->blockpart, (size_t)2 * 152 * 8 + 64, "block partials")))
    return st;
  if (h->opt.precision == PA_MIXED &&
      ((st = alloc_n(h, &h->ylo, (size_t)h->n_rows, "A x (low part)")) ||
       (st = alloc_n(h, &h->X0f, n, "iterate (FP32)")) || (st = alloc_n(h, &h->X1f, n, "iterate (FP32)")) ||
       (st = alloc_n(h, &h->X2f, n, "iterate (FP32)")) || (st = alloc_n(h, &h->Wf, n, "D_c x (FP32)")) ||
       (st = alloc_n(h, &h->mf, n, "first moment (FP32)")) ||
       (st = alloc_n(h, &h->vf, n, "second moment (FP32)")) ||
       (st = alloc_n(h, &h->yf, (size_t)h->n_rows, "A x (FP32)")) ||
       (st = alloc_n(h, &h->dxf, n, "step (FP32)"))))
    return st;
  if (h->opt.precision == PA_DF64 && (st = build_df(h))) return st;
  h->run_ready = true;
  return PA_OK;
}

static int choose_grid(pa_ctx* h, int* maxG_out) {
  int per = 0;
  int maxG = persistent_max_blocks(h->opt.loss, false, &per);
  maxG = std::min(maxG, merged_max_blocks(h->opt.loss, false));
  if (h->df_ok) maxG = std::min(maxG, merged_max_blocks(PA_LOSS_LOGRATIO, true));
  if (h->opt.precision == PA_MIXED) {
    maxG = std::min(maxG, persistent_max_blocks(h->opt.loss, true, &per));
    maxG = std::min(maxG, persistent32_max_blocks(&per));
  }
  if (maxG_out) *maxG_out = maxG;
  if (maxG <= 0) return -1;
  const int64_t n = std::max(h->n_rows, h->n_cols);
  const int64_t slices = std::max<int64_t>(1, std::min(h->sa.n_slices, h->sq.n_slices));
  int64_t want = (n + 2047) / 2048;  // about four rows per thread
  if (h->opt.grid_blocks > 0) want = h->opt.grid_blocks;  // an explicit request
  want = std::max<int64_t>(1, std::min(want, slices));
  return (int)std::min<int64_t>(want, maxG);
}

// Deal each CTA's slices [part[b], part[b+1]) to its NW warps: slices by
// decreasing cost 32 (width + row_weight), each to the warp with the least
// cost so far (ties: the lower warp); every warp then takes its slices in
// increasing order.  Deterministic, so the per-thread partial sums keep a
// fixed order.  Round-robin dealing left the slowest warp of a CTA with
// 1.2-1.3x the mean work on the hydro operators (rows of 1, 3, 6 and 11
// entries sorted within windows).
static void deal_slices(const std::vector<int32_t>& part, const std::vector<int32_t>& wp,
                        int row_weight, int NW, std::vector<int32_t>* list,
                        std::vector<int32_t>* woff) {
  const int G = (int)part.size() - 1;
  list->assign((size_t)part[G], 0);
  woff->assign((size_t)G * (NW + 1), 0);
  std::vector<int32_t> idx;
  std::vector<std::vector<int32_t>> per(NW);
  std::vector<long long> load(NW);
  for (int b = 0; b < G; ++b) {
    idx.clear();
    for (int32_t sl = part[b]; sl < part[b + 1]; ++sl) idx.push_back(sl);
    std::stable_sort(idx.begin(), idx.end(), [&](int32_t x, int32_t y) {
      return wp[x + 1] - wp[x] > wp[y + 1] - wp[y];
    });
    for (int w = 0; w < NW; ++w) {
      per[w].clear();
      load[w] = 0;
    }
    for (int32_t sl : idx) {
      int best = 0;
      for (int w = 1; w < NW; ++w)
        if (load[w] < load[best]) best = w;
      per[best].push_back(sl);
      load[best] += 32ll * (wp[sl + 1] - wp[sl] + row_weight);
    }
    int32_t pos = part[b];
    for (int w = 0; w < NW; ++w) {
      std::sort(per[w].begin(), per[w].end());
      (*woff)[(size_t)b * (NW + 1) + w] = pos;
      for (int32_t sl : per[w]) (*list)[pos++] = sl;
    }
    (*woff)[(size_t)b * (NW + 1) + NW] = pos;
  }
}

// The warp slice lists of the current partitions (after ensure_partitions
// or a tuner round).
static pa_status build_warp_lists(pa_ctx* h) {
  const int G = h->G, NW = kBlock / 32;
  cudaError_t e;
  if (h->wpa_h.empty()) {
    h->wpa_h.resize((size_t)h->sa.n_slices + 1);
    h->wpt_h.resize((size_t)h->sq.n_slices + 1);
    if ((e = cudaMemcpyAsync(h->wpa_h.data(), h->sa.wp, sizeof(int32_t) * h->wpa_h.size(), cudaMemcpyDeviceToHost, h->stream)) ||
        (e = cudaMemcpyAsync(h->wpt_h.data(), h->sq.wp, sizeof(int32_t) * h->wpt_h.size(), cudaMemcpyDeviceToHost, h->stream)))
      return cuda_fail(e, "reading the slice pointers");
  }
  std::vector<int32_t> pa_((size_t)G + 1), pt_((size_t)G + 1);
  if ((e = cudaMemcpyAsync(pa_.data(), h->part_a, sizeof(int32_t) * pa_.size(), cudaMemcpyDeviceToHost, h->stream)) ||
      (e = cudaMemcpyAsync(pt_.data(), h->part_t, sizeof(int32_t) * pt_.size(), cudaMemcpyDeviceToHost, h->stream)) ||
      (e = cudaStreamSynchronize(h->stream)))
    return cuda_fail(e, "reading the partitions");
  std::vector<int32_t> la, wa, lt, wt;
  deal_slices(pa_, h->wpa_h, 2, NW, &la, &wa);
  deal_slices(pt_, h->wpt_h, 30, NW, &lt, &wt);
  pa_status st;
  if (!h->a_list) {
    if ((st = alloc_n(h, &h->a_list, std::max<size_t>(la.size(), 1), "warp slice lists")) ||
        (st = alloc_n(h, &h->t_list, std::max<size_t>(lt.size(), 1), "warp slice lists")))
      return st;
  }
  if (h->a_woff) dev_free(h, h->a_woff);
  if (h->t_woff) dev_free(h, h->t_woff);
  h->a_woff = h->t_woff = nullptr;
  if ((st = alloc_n(h, &h->a_woff, wa.size(), "warp slice lists")) ||
      (st = alloc_n(h, &h->t_woff, wt.size(), "warp slice lists")))
    return st;
  if ((!la.empty() && (e = cudaMemcpyAsync(h->a_list, la.data(), sizeof(int32_t) * la.size(), cudaMemcpyHostToDevice, h->stream))) ||
      (!lt.empty() && (e = cudaMemcpyAsync(h->t_list, lt.data(), sizeof(int32_t) * lt.size(), cudaMemcpyHostToDevice, h->stream))) ||
      (e = cudaMemcpyAsync(h->a_woff, wa.data(), sizeof(int32_t) * wa.size(), cudaMemcpyHostToDevice, h->stream)) ||
      (e = cudaMemcpyAsync(h->t_woff, wt.data(), sizeof(int32_t) * wt.size(), cudaMemcpyHostToDevice, h->stream)) ||
      (e = cudaStreamSynchronize(h->stream)))  // the host vectors are pageable
    return cuda_fail(e, "uploading the warp slice lists");
  return PA_OK;
}

static pa_status ensure_partitions(pa_ctx* h, int G) {
  if (h->G == G && h->part_a) return PA_OK;
  if (h->part_a) dev_free(h, h->part_a);
  if (h->part_t) dev_free(h, h->part_t);
  if (h->partials) dev_free(h, h->partials);
  if (h->dep) dev_free(h, h->dep);
  if (h->ready) dev_free(h, h->ready);
  if (h->cta_ns) dev_free(h, h->cta_ns);
  if (h->cta_lat) dev_free(h, h->cta_lat);
  h->cta_lat = nullptr;
  h->part_a = h->part_t = h->dep = nullptr;
  h->partials = nullptr;
  h->ready = nullptr;
  h->cta_ns = nullptr;
  pa_status st;
  if ((st = alloc_n(h, &h->part_a, (size_t)G + 1, "partition")) ||
      (st = alloc_n(h, &h->part_t, (size_t)G + 1, "partition")) ||
      (st = alloc_n(h, &h->dep, (size_t)2 * G, "dependencies")) ||
      (st = alloc_n(h, &h->ready, (size_t)G, "ready flags")) ||
      (st = alloc_n(h, &h->cta_ns, (size_t)2 * G, "CTA timers")) ||
      (st = alloc_n(h, &h->cta_lat, (size_t)G, "CTA timers")) ||
      (st = alloc_n(h, &h->partials, (size_t)G * kPartSlots, "partials")))
    return st;
  cudaError_t e;
  // phase A rows weigh their padded entries plus 2; phase B/C rows carry the
  // Adam update as well (about 30 FP64 operations), hence the heavier weight.
  if ((e = launch_partition(h->sa.wp, h->sa.n_slices, G, 2, h->part_a, h->stream, &h->launches)) ||
      (e = launch_partition(h->sq.wp, h->sq.n_slices, G, 30, h->part_t, h->stream, &h->launches)))
    return cuda_fail(e, "partitioning slices");
  if ((e = launch_dependencies(h->sa.wp, h->sa.col, h->sa.val, h->part_a, h->part_t, G, h->dep,
                               h->stream, &h->launches)))
    return cuda_fail(e, "finding neighbour dependencies");
  h->G = G;
  h->tuned_rounds = 0;
  h->tune_best = INFINITY;
  return build_warp_lists(h);
}

// Re-split one partition at equal measured cost.  CTA b spent busy[b] on
// slices [part[b], part[b+1]); its time is spread over those slices in
// proportion to the cost model u(s) = 32 (w(s) + row_weight), and the new
// boundaries cut the cumulative estimate into G equal parts.
static void resplit(std::vector<int32_t>& part, const std::vector<int32_t>& wp,
                    const std::vector<double>& busy, int row_weight) {
  const int G = (int)part.size() - 1;
  const int ns = (int)wp.size() - 1;
  std::vector<double> cost(ns);
  for (int b = 0; b < G; ++b) {
    double U = 0;
    for (int s = part[b]; s < part[b + 1]; ++s) U += 32.0 * (wp[s + 1] - wp[s] + row_weight);
    const double tau = U > 0 ? busy[b] / U : 0.0;
    for (int s = part[b]; s < part[b + 1]; ++s) cost[s] = tau * 32.0 * (wp[s + 1] - wp[s] + row_weight);
  }
  double tot = 0;
  for (double c : cost) tot += c;
  if (!(tot > 0)) return;
  std::vector<int32_t> np(G + 1);
  np[0] = 0;
  np[G] = ns;
  double acc = 0;
  int s = 0;
  for (int b = 1; b < G; ++b) {
    const double target = tot * b / G;
    while (s < ns && acc + cost[s] < target) acc += cost[s++];
    np[b] = std::max(np[b - 1], s);
  }
  part = np;
}

// One round of the partition tuner, from the per-CTA timers of the last run
// and its time per iteration.  Every round but the last re-splits at equal
// measured cost; the last installs the fastest partition seen over the
// rounds (the cost-model start included), so one noisy measurement cannot
// leave a bad split behind.
static pa_status tune_partitions(pa_ctx* h, double t_iter) {
  const int G = h->G;
  std::vector<unsigned long long> t((size_t)2 * G), lat((size_t)G);
  std::vector<int32_t> pa_((size_t)G + 1), pt_((size_t)G + 1);
  std::vector<int32_t> wpa((size_t)h->sa.n_slices + 1), wpt((size_t)h->sq.n_slices + 1);
  cudaError_t e;
  if ((e = cudaMemcpyAsync(t.data(), h->cta_ns, sizeof(unsigned long long) * t.size(), cudaMemcpyDeviceToHost, h->stream)) ||
      (e = cudaMemcpyAsync(lat.data(), h->cta_lat, sizeof(unsigned long long) * lat.size(), cudaMemcpyDeviceToHost, h->stream)) ||
      (e = cudaMemcpyAsync(pa_.data(), h->part_a, sizeof(int32_t) * pa_.size(), cudaMemcpyDeviceToHost, h->stream)) ||
      (e = cudaMemcpyAsync(pt_.data(), h->part_t, sizeof(int32_t) * pt_.size(), cudaMemcpyDeviceToHost, h->stream)) ||
      (e = cudaMemcpyAsync(wpa.data(), h->sa.wp, sizeof(int32_t) * wpa.size(), cudaMemcpyDeviceToHost, h->stream)) ||
      (e = cudaMemcpyAsync(wpt.data(), h->sq.wp, sizeof(int32_t) * wpt.size(), cudaMemcpyDeviceToHost, h->stream)) ||
      (e = cudaStreamSynchronize(h->stream)))
    return cuda_fail(e, "reading the run profile for the tuner");
  if (t_iter < h->tune_best) {
    h->tune_best = t_iter;
    h->tune_best_a = pa_;
    h->tune_best_t = pt_;
  }
  ++h->tuned_rounds;
  if (h->tuned_rounds < h->opt.autotune) {
    // phase A is split by how late each CTA's y is ready (its phase C, its
    // wait for neighbours and its phase A), phases B and C by busy time
    std::vector<double> ba(G), bb(G);
    bool have_lat = true;
    for (int b = 0; b < G; ++b) have_lat = have_lat && lat[b] > 0;
    for (int b = 0; b < G; ++b) {
      ba[b] = have_lat ? (double)lat[b] : (double)t[2 * b];
      bb[b] = (double)t[2 * b + 1];
    }
    resplit(pa_, wpa, ba, 2);
    resplit(pt_, wpt, bb, 30);
  } else {
    pa_ = h->tune_best_a;
    pt_ = h->tune_best_t;
  }
  if ((e = cudaMemcpyAsync(h->part_a, pa_.data(), sizeof(int32_t) * pa_.size(), cudaMemcpyHostToDevice, h->stream)) ||
      (e = cudaMemcpyAsync(h->part_t, pt_.data(), sizeof(int32_t) * pt_.size(), cudaMemcpyHostToDevice, h->stream)) ||
      (e = launch_dependencies(h->sa.wp, h->sa.col, h->sa.val, h->part_a, h->part_t, G, h->dep,
                               h->stream, &h->launches)) ||
      (e = cudaStreamSynchronize(h->stream)))
    return cuda_fail(e, "applying the tuned partition");
  return build_warp_lists(h);
}

// The single-pass engine's structures for G CTAs.  The partition cuts the
// slices of P A Q^T at equal cost 32 (w(s) + 15) (each entry is used twice:
// y = A x and its column's window sum; the 15 stands for the per-position
// Adam work), and CTA b owns rows and x positions [32 part[b], 32 part[b+1]).
// The plan of CTA b lists, for each column c of its window [cmin_b, cmax_b]
// (the columns its rows touch), the block's entries in column c by
// increasing row, each as (row - 32 part[b]) << 8 | slot k of the entry in
// its row.  The columns with entries are sorted by entry count (stable) and
// cut into groups of 32, one column per lane, stored column-major like the
// slices of the matrix, so a warp's lanes take columns of equal length.
// Built on the host from the sliced copy, so it is deterministic.
static pa_status ensure_single(pa_ctx* h, int G) {
  if (h->sp_G == G && h->sp_part) return PA_OK;
  if (h->n_rows != h->n_cols)
    return fail(PA_ERR_UNSUPPORTED, "the single-pass engine needs a square matrix (%d x %d)",
                h->n_rows, h->n_cols);
  for (void* q : {(void*)h->sp_part, (void*)h->sp_dep, (void*)h->sp_rdep, (void*)h->sp_list,
                  (void*)h->sp_lwoff, (void*)h->sp_cmin, (void*)h->sp_woff, (void*)h->sp_goff,
                  (void*)h->sp_gp, (void*)h->sp_gcol, (void*)h->sp_ent, (void*)h->sp_halo})
    if (q) dev_free(h, q);
  h->sp_part = h->sp_dep = h->sp_rdep = h->sp_list = h->sp_lwoff = nullptr;
  h->sp_cmin = h->sp_woff = h->sp_goff = h->sp_gp = h->sp_gcol = nullptr;
  h->sp_ent = nullptr;
  h->sp_halo = nullptr;
  h->sp_G = 0;
  const int ns = h->sa.n_slices, n = h->n_cols;
  pa_status st;
  if ((st = alloc_n(h, &h->sp_part, (size_t)G + 1, "single-pass partition")) ||
      (st = alloc_n(h, &h->sp_dep, (size_t)2 * G, "single-pass partition")))
    return st;
  cudaError_t e;
  if ((e = launch_partition(h->sa.wp, ns, G, 15, h->sp_part, h->stream, &h->launches)) ||
      (e = launch_dependencies(h->sa.wp, h->sa.col, h->sa.val, h->sp_part, h->sp_part, G,
                               h->sp_dep, h->stream, &h->launches)))
    return cuda_fail(e, "partitioning for the single-pass engine");
  // the sliced copy on the host
  if (h->wpa_h.empty()) {
    h->wpa_h.resize((size_t)ns + 1);
    h->wpt_h.resize((size_t)h->sq.n_slices + 1);
    if ((e = cudaMemcpyAsync(h->wpa_h.data(), h->sa.wp, sizeof(int32_t) * h->wpa_h.size(), cudaMemcpyDeviceToHost, h->stream)) ||
        (e = cudaMemcpyAsync(h->wpt_h.data(), h->sq.wp, sizeof(int32_t) * h->wpt_h.size(), cudaMemcpyDeviceToHost, h->stream)))
      return cuda_fail(e, "reading the slice pointers");
  }
  const std::vector<int32_t>& wp = h->wpa_h;
  const size_t total = (size_t)32 * wp[ns];
  std::vector<int32_t> part((size_t)G + 1), col(total);
  std::vector<double> val(total);
  if ((e = cudaMemcpyAsync(part.data(), h->sp_part, sizeof(int32_t) * part.size(), cudaMemcpyDeviceToHost, h->stream)) ||
      (total && (e = cudaMemcpyAsync(col.data(), h->sa.col, sizeof(int32_t) * total, cudaMemcpyDeviceToHost, h->stream))) ||
      (total && (e = cudaMemcpyAsync(val.data(), h->sa.val, sizeof(double) * total, cudaMemcpyDeviceToHost, h->stream))) ||
      (e = cudaStreamSynchronize(h->stream)))
    return cuda_fail(e, "reading the sliced matrix");
  for (int s = 0; s < ns; ++s)
    if (wp[s + 1] - wp[s] > 255)
      return fail(PA_ERR_UNSUPPORTED, "the single-pass engine takes rows of at most 255 entries");
  // windows
  std::vector<int32_t> cmin((size_t)G), woff((size_t)G + 1, 0), rdep((size_t)2 * G);
  for (int b = 0; b < G; ++b) {
    int32_t lo = INT32_MAX, hi = -1;
    for (int s = part[b]; s < part[b + 1]; ++s)
      for (size_t e2 = (size_t)32 * wp[s]; e2 < (size_t)32 * wp[s + 1]; ++e2)
        if (val[e2] != 0.0) {
          lo = std::min(lo, col[e2]);
          hi = std::max(hi, col[e2]);
        }
    cmin[b] = hi < 0 ? 0 : lo;
    const int64_t w = hi < 0 ? 0 : (int64_t)hi - lo + 1;
    if ((int64_t)woff[b] + w > INT32_MAX - 1)
      return fail(PA_ERR_UNSUPPORTED, "single-pass windows exceed 2^31 columns");
    woff[b + 1] = woff[b] + (int32_t)w;
  }
  const size_t nwin = (size_t)woff[G];
  // entries per window column, then the entries in row order
  std::vector<int32_t> cptr(nwin + 1, 0);
  for (int b = 0; b < G; ++b)
    for (int s = part[b]; s < part[b + 1]; ++s)
      for (size_t e2 = (size_t)32 * wp[s]; e2 < (size_t)32 * wp[s + 1]; ++e2)
        if (val[e2] != 0.0) ++cptr[(size_t)woff[b] + (col[e2] - cmin[b]) + 1];
  for (size_t w = 0; w < nwin; ++w) cptr[w + 1] += cptr[w];
  const size_t nent = (size_t)cptr[nwin];
  std::vector<uint32_t> bucket(std::max<size_t>(nent, 1));
  {
    std::vector<int32_t> fill(cptr.begin(), cptr.end() - 1);
    for (int b = 0; b < G; ++b)
      for (int s = part[b]; s < part[b + 1]; ++s) {
        const int w = wp[s + 1] - wp[s];
        for (int l = 0; l < 32; ++l)  // rows of the slice in order, each row's entries in order
          for (int k = 0; k < w; ++k) {
            const size_t e2 = (size_t)32 * (wp[s] + k) + l;
            if (val[e2] == 0.0) continue;
            const uint32_t rl = (uint32_t)(32 * (s - part[b]) + l);
            bucket[(size_t)fill[(size_t)woff[b] + (col[e2] - cmin[b])]++] = (rl << 8) | (uint32_t)k;
          }
      }
  }
  // per CTA: the window columns that have entries, by decreasing count
  // (stable), in groups of 32 stored column-major and padded with kPlanPad
  std::vector<int32_t> goff((size_t)G + 1, 0), gp(1, 0), gcol;
  std::vector<uint32_t> ent;
  std::vector<int32_t> order;
  for (int b = 0; b < G; ++b) {
    const int32_t W = woff[b + 1] - woff[b];
    auto cnt = [&](int32_t w) { return cptr[(size_t)woff[b] + w + 1] - cptr[(size_t)woff[b] + w]; };
    order.clear();
    for (int32_t w = 0; w < W; ++w)
      if (cnt(w) > 0) order.push_back(w);
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return cnt(x) > cnt(y); });
    for (size_t g0 = 0; g0 < order.size(); g0 += 32) {
      const int width = cnt(order[g0]);
      const size_t base = ent.size();
      ent.resize(base + (size_t)32 * width, kPlanPad);
      for (int l = 0; l < 32; ++l) {
        if (g0 + l >= order.size()) {
          gcol.push_back(-1);
          continue;
        }
        const int32_t w = order[g0 + l];
        gcol.push_back(w);
        const size_t c0 = (size_t)cptr[(size_t)woff[b] + w];
        for (int k = 0; k < cnt(w); ++k) ent[base + (size_t)32 * k + l] = bucket[c0 + k];
      }
      gp.push_back(gp.back() + width);
    }
    goff[b + 1] = (int32_t)(gp.size() - 1);
  }
  if (ent.empty()) ent.push_back(kPlanPad);
  if (gcol.empty()) gcol.push_back(-1);
  // the CTAs whose windows meet each CTA's own positions
  for (int c = 0; c < G; ++c) {
    const int64_t p0 = std::min<int64_t>(32ll * part[c], n), p1 = std::min<int64_t>(32ll * part[c + 1], n);
    int lo = 1, hi = 0;
    for (int b = 0; b < G && p0 < p1; ++b) {
      const int64_t w0 = cmin[b], w1 = (int64_t)cmin[b] + (woff[b + 1] - woff[b]);
      if (w0 < p1 && p0 < w1) {
        if (lo > hi) lo = b;
        hi = b;
      }
    }
    rdep[2 * c] = lo;
    rdep[2 * c + 1] = hi;
  }
  std::vector<int32_t> list, lwoff;
  deal_slices(part, wp, 15, kBlock / 32, &list, &lwoff);
  if ((st = alloc_n(h, &h->sp_rdep, rdep.size(), "single-pass plan")) ||
      (st = alloc_n(h, &h->sp_list, std::max<size_t>(list.size(), 1), "single-pass plan")) ||
      (st = alloc_n(h, &h->sp_lwoff, lwoff.size(), "single-pass plan")) ||
      (st = alloc_n(h, &h->sp_cmin, cmin.size(), "single-pass plan")) ||
      (st = alloc_n(h, &h->sp_woff, woff.size(), "single-pass plan")) ||
      (st = alloc_n(h, &h->sp_goff, goff.size(), "single-pass plan")) ||
      (st = alloc_n(h, &h->sp_gp, gp.size(), "single-pass plan")) ||
      (st = alloc_n(h, &h->sp_gcol, gcol.size(), "single-pass plan")) ||
      (st = alloc_n(h, &h->sp_ent, ent.size(), "single-pass plan")) ||
      (st = alloc_n(h, &h->sp_halo, std::max<size_t>(nwin, 1), "single-pass halo")))
    return st;
  if ((e = cudaMemcpyAsync(h->sp_rdep, rdep.data(), sizeof(int32_t) * rdep.size(), cudaMemcpyHostToDevice, h->stream)) ||
      (!list.empty() && (e = cudaMemcpyAsync(h->sp_list, list.data(), sizeof(int32_t) * list.size(), cudaMemcpyHostToDevice, h->stream))) ||
      (e = cudaMemcpyAsync(h->sp_lwoff, lwoff.data(), sizeof(int32_t) * lwoff.size(), cudaMemcpyHostToDevice, h->stream)) ||
      (e = cudaMemcpyAsync(h->sp_cmin, cmin.data(), sizeof(int32_t) * cmin.size(), cudaMemcpyHostToDevice, h->stream)) ||
      (e = cudaMemcpyAsync(h->sp_woff, woff.data(), sizeof(int32_t) * woff.size(), cudaMemcpyHostToDevice, h->stream)) ||
      (e = cudaMemcpyAsync(h->sp_goff, goff.data(), sizeof(int32_t) * goff.size(), cudaMemcpyHostToDevice, h->stream)) ||
      (e = cudaMemcpyAsync(h->sp_gp, gp.data(), sizeof(int32_t) * gp.size(), cudaMemcpyHostToDevice, h->stream)) ||
      (e = cudaMemcpyAsync(h->sp_gcol, gcol.data(), sizeof(int32_t) * gcol.size(), cudaMemcpyHostToDevice, h->stream)) ||
      (e = cudaMemsetAsync(h->sp_halo, 0, sizeof(double) * std::max<size_t>(nwin, 1), h->stream)) ||
      (e = cudaMemcpyAsync(h->sp_ent, ent.data(), sizeof(uint32_t) * ent.size(), cudaMemcpyHostToDevice, h->stream)) ||
      (e = cudaStreamSynchronize(h->stream)))  // the host vectors are pageable
    return cuda_fail(e, "uploading the single-pass plan");
  h->sp_window_cols = (int64_t)nwin;
  h->sp_plan_entries = (int64_t)nent;
  h->sp_plan_slots = (int64_t)ent.size();
  h->sp_groups = (int64_t)goff[G];
  h->sp_G = G;
  return PA_OK;
}

// The single-pass engine's fields of IterParams.
static void single_params(pa_ctx* h, IterParams* p) {
  p->part_a = h->sp_part;
  p->part_t = h->sp_part;
  p->dep = h->sp_dep;
  p->a_list = h->sp_list;
  p->a_woff = h->sp_lwoff;
  p->sp_cmin = h->sp_cmin;
  p->sp_woff = h->sp_woff;
  p->sp_goff = h->sp_goff;
  p->sp_gp = h->sp_gp;
  p->sp_gcol = h->sp_gcol;
  p->sp_ent = h->sp_ent;
  p->sp_halo = h->sp_halo;
  p->sp_rdep = h->sp_rdep;
}

// Per-iteration Adam scalars: the step lr m_hat / (sqrt(v_hat) + eps) with
// m_hat = m / (1 - b1^t), v_hat = v / (1 - b2^t) equals K1 m / (sqrt(v) + K2)
// with K1 = lr sqrt(1 - b2^t) / (1 - b1^t) and K2 = eps sqrt(1 - b2^t).
static pa_status ensure_bias(pa_ctx* h, int iters, double lr, double b1, double b2, double eps) {
  std::vector<double2> tab((size_t)std::max(iters, 1));
  for (int t = 1; t <= iters; ++t) {
    const double r2 = sqrt(1.0 - pow(b2, (double)t));
    tab[t - 1] = make_double2(lr * r2 / (1.0 - pow(b1, (double)t)), eps * r2);
  }
  if (h->bias_cap < iters) {
    if (h->bias) dev_free(h, h->bias);
    h->bias = nullptr;
    pa_status st;
    if ((st = alloc_n(h, &h->bias, (size_t)std::max(iters, 1), "bias table"))) return st;
    h->bias_cap = iters;
  }
  if (iters > 0) {
    cudaError_t e = cudaMemcpyAsync(h->bias, tab.data(), sizeof(double2) * iters,
                                    cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // tab is pageable host memory
    if (e != cudaSuccess) return cuda_fail(e, "uploading the bias corrections");
  }
  if (h->df_ok && iters > 0) {
    // the same constants as double-word pairs: hi = float(K), lo = float(K - hi)
    std::vector<float4> t2((size_t)iters);
    for (int t = 0; t < iters; ++t) {
      const float k1 = (float)tab[t].x, k2 = (float)tab[t].y;
      t2[t] = make_float4(k1, (float)(tab[t].x - (double)k1), k2, (float)(tab[t].y - (double)k2));
    }
    if (h->bias2) dev_free(h, h->bias2);
    h->bias2 = nullptr;
    pa_status st;
    if ((st = alloc_n(h, &h->bias2, (size_t)iters, "bias table (double-float)"))) return st;
    cudaError_t e = cudaMemcpyAsync(h->bias2, t2.data(), sizeof(float4) * iters,
                                    cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "uploading the bias corrections");
  }
  return PA_OK;
}

static pa_status check_hyper(int iters, double lr, double b1, double b2, double eps) {
  if (iters < 0) return fail(PA_ERR_INVALID_ARG, "iters < 0");
  if (!(lr > 0) || !isfinite(lr)) return fail(PA_ERR_INVALID_ARG, "lr must be finite and > 0");
  if (!(b1 >= 0 && b1 < 1) || !(b2 >= 0 && b2 < 1))
    return fail(PA_ERR_INVALID_ARG, "beta1, beta2 must lie in [0, 1)");
  if (!(eps >= 0) || !isfinite(eps)) return fail(PA_ERR_INVALID_ARG, "eps must be finite and >= 0");
  return PA_OK;
}

static pa_status status_error(const RunState* rs) {
  if (rs->status == PA_ERR_TIMEOUT)
    return fail(PA_ERR_TIMEOUT, "a grid barrier wait ran out of time (barrier %d)", rs->timeout_site);
  if (rs->status == PA_ERR_NONFINITE) return fail(PA_ERR_NONFINITE, "a NaN or Inf reached a reduction");
  return PA_OK;
}

// One FP64 launch of the persistent kernel: `iters` iterations continuing at
// iteration t0 + 1 (the bias table is indexed from there).  With fresh_state
// X0 = Xinit and m = v = 0; otherwise X0, m and v hold the state to continue
// from.  Then sigma of the tracked minimiser; the run state comes back in *out.
static pa_status fp64_run(pa_ctx* h, pa_mode mode, int iters, int t0, bool fresh_state, bool dd,
                          double b1, double b2, double eps, int G, int maxG, double* L_trace_dev,
                          double* x_trace_dev, int n_trace, RunState* out, bool cluster = false,
                          int kernel = 0, const pa_ctx::Cont* cont = nullptr) {
  // kernel: 0 = the three-phase k_persistent, 1 = the merged-phase kernel in
  // FP64, 2 = the merged-phase kernel in double-float, 6 = the single-pass
  // kernel (k_single)
  const size_t n = (size_t)h->n_cols;
  cudaError_t e = cudaSuccess;
  if (fresh_state &&
      ((e = cudaMemcpyAsync(h->X0, h->Xinit, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream)) ||
       (e = cudaMemsetAsync(h->m, 0, sizeof(double) * n, h->stream)) ||
       (e = cudaMemsetAsync(h->v, 0, sizeof(double) * n, h->stream))))
    return cuda_fail(e, "preparing the run");
  if ((e = cudaMemsetAsync(h->st, 0, sizeof(RunState), h->stream)) ||
      (e = cudaMemsetAsync(h->ready, 0, sizeof(unsigned) * G, h->stream)))
    return cuda_fail(e, "preparing the run");
  IterParams p{};
  p.n_rows = h->n_rows;
  p.n_cols = h->n_cols;
  p.a_wp = h->sa.wp; p.a_col = h->sa.col; p.a_val = h->sa.val;
  p.t_wp = h->sq.wp; p.t_col = h->sq.col; p.t_val = h->sq.val;
  p.part_a = h->part_a; p.part_t = h->part_t;
  p.a_list = h->a_list; p.a_woff = h->a_woff; p.t_list = h->t_list; p.t_woff = h->t_woff;
  p.X0 = h->X0; p.X1 = h->X1; p.X2 = h->X2;
  p.m = h->m; p.v = h->v; p.y = h->y; p.ylo = h->ylo; p.dx = h->dx;
  p.partials = h->partials;
  p.ready = h->ready;
  p.cta_ns = h->cta_ns;
  p.cta_lat = h->cta_lat;
  h->last_G = G;
  p.dep = h->dep;
  p.bias = h->bias;
  p.L_trace = L_trace_dev;
  p.x_trace = x_trace_dev;
  p.n_trace = n_trace;
  p.st = h->st;
  p.iters = iters;
  p.t0 = t0;
  p.mode = mode;
  p.ablation = h->opt.ablation;
  p.beta1 = b1; p.beta2 = b2; p.eps = eps;
  p.omb1 = 1.0 - b1;
  p.w2 = (1.0 - b2) / ((1.0 - b1) * (1.0 - b1));
  p.timeout_ns = h->opt.barrier_timeout_ns;
  p.skip_arrival = h->opt.debug_skip_arrival;
  p.u = h->dx;
  p.s_scale = 1.0;
  if (cont) {  // continue a run: x_T in X0, x_min in X1, m and v as left
    p.init_have_best = cont->have_best;
    p.init_best_s = cont->best_s;
    p.init_best_q = cont->best_q;
    p.init_t_min = cont->t_min;
    p.init_minb = 1;
    p.t_min_base = cont->t_done;
  }
  if (kernel == 2) {
    p.a_val2 = h->a_val2; p.t_val2 = h->t_val2;
    p.XD0 = h->XD0; p.XD1 = h->XD1; p.XD2 = h->XD2;
    p.ud = h->ud; p.md = h->md; p.vd = h->vd; p.yd = h->yd;
    p.bias2 = h->bias2;
    p.s_scale = ldexp(1.0, 2 * h->df_k);
    if (!fresh_state) return fail(PA_ERR_UNSUPPORTED, "double-float runs start from x_init");
    if ((e = launch_split_df((int64_t)n, h->X0, 0, h->XD0, h->stream, &h->launches)) ||
        (e = cudaMemsetAsync(h->md, 0, sizeof(float2) * n, h->stream)) ||
        (e = cudaMemsetAsync(h->vd, 0, sizeof(float2) * n, h->stream)))
      return cuda_fail(e, "preparing the run");
  }
  if (kernel == 6) single_params(h, &p);
  if (cluster) e = launch_persistent_cluster(p, h->opt.loss, G, h->stream, &h->launches);
  else if (kernel == 0) e = launch_persistent(p, h->opt.loss, dd, G, h->stream, &h->launches);
  else if (kernel == 6) e = launch_single(p, h->opt.loss, G, h->stream, &h->launches);
  else e = launch_merged(p, h->opt.loss, kernel == 2, G, h->stream, &h->launches);
  if (e == cudaErrorCooperativeLaunchTooLarge)
    return fail(PA_ERR_LAUNCH, "cooperative grid of %d CTAs does not fit (max %d)", G, maxG);
  if (e != cudaSuccess) return cuda_fail(e, "launching the persistent kernel");
  if (kernel == 2) {
    // x_min and the last iterate back to FP64 in the buffers the rest reads
    RunState rs{};
    if ((e = cudaMemcpyAsync(&rs, h->st, sizeof(RunState), cudaMemcpyDeviceToHost, h->stream)) ||
        (e = cudaStreamSynchronize(h->stream)))
      return cuda_fail(e, "running Projected Adam");
    if (rs.status == kStatusDfRange) {  // outside the variant's range: the run again in FP64
      ++h->df_fallbacks;
      if ((e = cudaMemcpyAsync(h->X0, h->Xinit, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream)))
        return cuda_fail(e, "preparing the run");
      return fp64_run(h, mode, iters, t0, fresh_state, dd, b1, b2, eps, G, maxG, L_trace_dev,
                      x_trace_dev, n_trace, out, false, 1);
    }
    float2* xd[3] = {h->XD0, h->XD1, h->XD2};
    double* x64[3] = {h->X0, h->X1, h->X2};
    for (int k : {rs.minb, rs.cur})
      if (k >= 0 && k < 3 && (e = launch_join_df((int64_t)n, xd[k], x64[k], h->stream, &h->launches)))
        return cuda_fail(e, "converting the iterates");
  }
  if ((e = launch_sigma(h->sa, h->n_cols, h->X0, h->X1, h->X2, 1, h->st, h->blockpart, dd,
                        h->stream, &h->launches)))
    return cuda_fail(e, "launching the sigma kernel");
  if ((e = cudaMemcpyAsync(out, h->st, sizeof(RunState), cudaMemcpyDeviceToHost, h->stream)) ||
      (e = cudaStreamSynchronize(h->stream)))
    return cuda_fail(e, "running Projected Adam");
  h->last_kernel = cluster ? 3 : kernel;
  h->last_refreshes = (kernel == 1 || kernel == 2) ? out->refreshes : 0;
  return PA_OK;
}

static float* pick32h(pa_ctx* h, int k) { return k == 0 ? h->X0f : (k == 1 ? h->X1f : h->X2f); }
static double* pick64h(pa_ctx* h, int k) { return k == 0 ? h->X0 : (k == 1 ? h->X1 : h->X2); }

// Mixed-precision sigma_max: FP32 stage (iters - tail iterations), then the
// FP64 tail from the converted FP32 state.  x_min is the tracked minimiser of
// whichever stage scores the larger sigma in FP64.
static pa_status mixed_max_run(pa_ctx* h, int iters, double b1, double b2, double eps, int G,
                               int maxG, double* L_trace_dev, RunState* out) {
  const int tail = h->opt.fp64_tail < 0 ? iters / 10 : std::min(h->opt.fp64_tail, iters);
  const int t32 = iters - tail;
  const size_t n = (size_t)h->n_cols;
  cudaError_t e;
  // ---- FP32 stage
  if ((e = launch_convert((int64_t)n, h->Xinit, h->X0f, h->stream, &h->launches)) ||
      (e = cudaMemsetAsync(h->mf, 0, sizeof(float) * n, h->stream)) ||
      (e = cudaMemsetAsync(h->vf, 0, sizeof(float) * n, h->stream)) ||
      (e = cudaMemsetAsync(h->st, 0, sizeof(RunState), h->stream)) ||
      (e = cudaMemsetAsync(h->ready, 0, sizeof(unsigned) * G, h->stream)))
    return cuda_fail(e, "preparing the FP32 stage");
  IterParams32 q{};
  q.n_rows = h->n_rows;
  q.n_cols = h->n_cols;
  q.a_wp = h->sa.wp; q.a_col = h->sa.col; q.a_val = h->a_val32;
  q.t_wp = h->sq.wp; q.t_col = h->sq.col; q.t_val = h->t_val32;
  q.dr = h->drp32; q.dc = h->dcp32;
  q.part_a = h->part_a; q.part_t = h->part_t; q.dep = h->dep;
  q.X0 = h->X0f; q.X1 = h->X1f; q.X2 = h->X2f; q.W = h->Wf;
  q.m = h->mf; q.v = h->vf; q.y = h->yf; q.dx = h->dxf;
  q.partials = h->partials;
  q.ready = h->ready;
  q.cta_ns = h->cta_ns;
  q.bias = h->bias;
  q.L_trace = L_trace_dev;
  q.st = h->st;
  q.iters = t32;
  q.ablation = h->opt.ablation;
  q.beta1 = b1; q.beta2 = b2;
  q.omb1 = 1.0 - b1;
  q.w2 = (1.0 - b2) / ((1.0 - b1) * (1.0 - b1));
  q.timeout_ns = h->opt.barrier_timeout_ns;
  q.skip_arrival = h->opt.debug_skip_arrival;
  h->last_G = G;
  e = launch_persistent32(q, G, h->stream, &h->launches);
  if (e == cudaErrorCooperativeLaunchTooLarge)
    return fail(PA_ERR_LAUNCH, "cooperative grid of %d CTAs does not fit (max %d)", G, maxG);
  if (e != cudaSuccess) return cuda_fail(e, "launching the FP32 persistent kernel");
  RunState r32{};
  if ((e = cudaMemcpyAsync(&r32, h->st, sizeof(RunState), cudaMemcpyDeviceToHost, h->stream)) ||
      (e = cudaStreamSynchronize(h->stream)))
    return cuda_fail(e, "running the FP32 stage");
  pa_status st;
  if ((st = status_error(&r32))) return st;
  // candidate 1: the FP32 stage's tracked minimiser, scored in FP64 (in X1)
  if ((e = launch_convert((int64_t)n, pick32h(h, r32.minb), h->X1, h->stream, &h->launches)) ||
      (e = launch_sigma(h->sa, h->n_cols, h->X1, h->X1, h->X1, 0, h->st, h->blockpart, false,
                        h->stream, &h->launches)))
    return cuda_fail(e, "scoring the FP32 stage");
  double sig32 = 0;
  if ((e = cudaMemcpyAsync(&sig32, &h->st->sigma, sizeof(double), cudaMemcpyDeviceToHost, h->stream)) ||
      (e = cudaStreamSynchronize(h->stream)))
    return cuda_fail(e, "scoring the FP32 stage");
  if ((e = launch_unpermute(h->n_cols, 1, h->sq.pos, h->X1, h->xmin_max, h->stream, &h->launches)))
    return cuda_fail(e, "keeping x_min");
  *out = r32;
  out->sigma = sig32;
  out->cur = 0;
  // the last FP32 iterate, in FP64, continues (or is x_last when there is no tail)
  if ((e = launch_convert((int64_t)n, pick32h(h, r32.cur), h->X0, h->stream, &h->launches)))
    return cuda_fail(e, "converting the FP32 state");
  if (tail == 0 || r32.status != PA_OK) return (pa_status)r32.status;
  // ---- FP64 tail near convergence
  if ((e = launch_convert((int64_t)n, h->mf, h->m, h->stream, &h->launches)) ||
      (e = launch_convert((int64_t)n, h->vf, h->v, h->stream, &h->launches)))
    return cuda_fail(e, "converting the FP32 state");
  RunState r64{};
  if ((st = fp64_run(h, PA_SIGMA_MAX, tail, t32, false, false, b1, b2, eps, G, maxG,
                     L_trace_dev ? L_trace_dev + t32 : nullptr, nullptr, 0, &r64)))
    return st;
  if ((st = status_error(&r64))) return st;
  out->iters_run = r32.iters_run + r64.iters_run;
  out->cur = r64.cur;
  out->L_last = r64.L_last;
  out->status = r64.status;
  if (r64.sigma > sig32) {  // the FP64 tail found the better iterate
    out->sigma = r64.sigma;
    out->L_min = r64.L_min;
    out->t_min = t32 + r64.t_min;
    out->minb = r64.minb;
    if ((e = launch_unpermute(h->n_cols, 1, h->sq.pos, pick64h(h, r64.minb), h->xmin_max,
                              h->stream, &h->launches)))
      return cuda_fail(e, "keeping x_min");
  }
  return (pa_status)out->status;
}

// The launch-shape tuner (autotune > 0, plain FP64 runs of the AUTO engine
// on a grid of more than 16 CTAs, no explicit grid size): short timed runs
// of the three-phase kernel with two and with one CTA per SM, the
// merged-phase kernel and the single-pass kernel (when the matrix suits it),
// each from x_init; the fastest is kept for the handle and, under the
// matrix's structural signature, for later handles of the same matrix.
// The choice sets the order of the reductions, like the partition tuner.
static std::mutex g_launch_mu;
static std::map<std::array<int64_t, 6>, std::array<int, 2>> g_launch_cache;

static pa_status tune_launch(pa_ctx* h, pa_mode mode, int iters, double b1, double b2, double eps,
                             int Gdef, int maxG) {
  if (h->launch_kernel >= 0) return PA_OK;
  const std::array<int64_t, 6> key = {h->n_rows, h->n_cols, h->nnz, h->sa.n_slices,
                                      h->a_entries, h->t_entries};
  {
    std::lock_guard<std::mutex> lk(g_launch_mu);
    auto it = g_launch_cache.find(key);
    if (it != g_launch_cache.end()) {
      h->launch_kernel = it->second[0];
      h->launch_G = it->second[1];
      h->launch_source = 2;
      return PA_OK;
    }
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  std::vector<std::array<int, 2>> cands = {{0, Gdef}};
  if (Gdef > sms && sms > 16) cands.push_back({0, sms});
  const int gm = merged_max_blocks(h->opt.loss, false);
  if (gm > 16) cands.push_back({1, std::min(Gdef, gm)});
  const int gs = single_max_blocks(h->opt.loss);
  if (h->n_rows == h->n_cols && gs > 16) cands.push_back({6, std::min(Gdef, gs)});
  const int trial = std::min(iters, 40);
  cudaError_t e;
  for (cudaEvent_t& ev : h->tune_ev)
    if (!ev && (e = cudaEventCreate(&ev))) return cuda_fail(e, "creating the tuner's events");
  h->launch_cands.clear();
  h->launch_ms.clear();
  double best = INFINITY;
  std::array<int, 2> pick = cands[0];
  for (const auto& c : cands) {
    pa_status st;
    if ((st = ensure_partitions(h, c[1]))) return st;
    if (c[0] == 6 && (st = ensure_single(h, c[1]))) {
      if (st != PA_ERR_UNSUPPORTED) return st;
      g_err.clear();  // the single-pass engine does not take this matrix
      continue;
    }
    RunState rs{};
    float ms = 0.f;
    if ((e = cudaEventRecord(h->tune_ev[0], h->stream))) return cuda_fail(e, "timing a trial");
    if ((st = fp64_run(h, mode, trial, 0, true, false, b1, b2, eps, c[1], maxG, nullptr, nullptr,
                       0, &rs, false, c[0])))
      return st;
    if ((e = cudaEventRecord(h->tune_ev[1], h->stream)) ||
        (e = cudaEventSynchronize(h->tune_ev[1])) ||
        (e = cudaEventElapsedTime(&ms, h->tune_ev[0], h->tune_ev[1])))
      return cuda_fail(e, "timing a trial");
    h->launch_cands.push_back(c);
    h->launch_ms.push_back(ms);
    if (ms < best) {
      best = ms;
      pick = c;
    }
  }
  h->launch_kernel = pick[0];
  h->launch_G = pick[1];
  h->launch_source = 1;
  std::lock_guard<std::mutex> lk(g_launch_mu);
  g_launch_cache[key] = pick;
  return PA_OK;
}

// One Algorithm 1 run from the device vector h->Xinit.
static pa_status run_one(pa_ctx* h, pa_mode mode, int iters, double lr, double b1, double b2,
                         double eps, double* L_trace_dev, double* x_trace_dev, int n_trace,
                         RunState* out) {
  if (mode == PA_SIGMA_MIN && h->n_rows < h->n_cols)
    return fail(PA_ERR_NOT_SQUARE, "sigma_min needs n_rows >= n_cols (%d x %d)", h->n_rows,
                h->n_cols);
  const bool mixed = h->opt.precision == PA_MIXED;
  if (mixed && mode == PA_SIGMA_MAX && x_trace_dev)
    return fail(PA_ERR_INVALID_ARG, "x traces are not available for the mixed-precision sigma_max");
  int maxG = 0;
  int G = choose_grid(h, &maxG);
  if (G <= 0) return fail(PA_ERR_LAUNCH, "the persistent kernel does not fit on this GPU");
  // the cluster engine: one thread-block cluster with hardware barriers, for
  // plain FP64 runs of matrices that would use at most 16 CTAs anyway
  bool cluster = false;
  const bool df = h->opt.precision == PA_DF64 && h->df_ok;
  const bool single = h->opt.engine == PA_ENGINE_SINGLE;
  if (single) {
    if (h->opt.precision != PA_FP64)
      return fail(PA_ERR_UNSUPPORTED, "the single-pass engine runs in FP64 only");
    const int gs = single_max_blocks(h->opt.loss);
    if (gs <= 0) return fail(PA_ERR_LAUNCH, "the single-pass kernel does not fit on this GPU");
    G = std::min(G, gs);
    maxG = std::min(maxG, gs);
  }
  if (!mixed && !df && !single && h->opt.engine != PA_ENGINE_GRID && h->opt.engine != PA_ENGINE_MERGED &&
      h->opt.debug_skip_arrival == 0 && (h->opt.engine == PA_ENGINE_CLUSTER || G <= 16)) {
    const int cmax = persistent_cluster_max(h->opt.loss);
    const int slices = std::max(1, std::min(h->sa.n_slices, h->sq.n_slices));
    int Gc = std::min(std::min(cmax, 16), slices);
    if (h->opt.grid_blocks > 0) Gc = std::min(Gc, h->opt.grid_blocks);
    if (Gc >= 1) {
      cluster = true;
      G = Gc;
    }
  }
  pa_status st;
  if ((st = ensure_bias(h, iters, lr, b1, b2, eps))) return st;
  // the merged-phase kernel in double-float for PA_DF64 (when the matrix
  // fits it) and in FP64 on request; the single-pass kernel on request;
  // the launch-shape tuner's choice for tuned plain FP64 runs; otherwise the
  // three-phase kernel
  int kernel = 0;
  if (single) kernel = 6;
  else if (!cluster && !mixed) {
    if (h->opt.precision == PA_DF64 && h->df_ok) kernel = 2;
    else if (h->opt.engine == PA_ENGINE_MERGED) kernel = 1;
    else if (h->opt.precision == PA_FP64 && h->opt.engine == PA_ENGINE_AUTO &&
             h->opt.autotune > 0 && iters >= 20 &&
             h->opt.grid_blocks == 0 && h->opt.debug_skip_arrival == 0) {
      if ((st = tune_launch(h, mode, iters, b1, b2, eps, G, maxG))) return st;
      kernel = h->launch_kernel;
      G = h->launch_G;
    }
  }
  if ((st = ensure_partitions(h, G))) return st;
  if (kernel == 6 && (st = ensure_single(h, G))) return st;
  if (mixed && mode == PA_SIGMA_MAX) {
    h->cont.valid = false;
    if ((st = mixed_max_run(h, iters, b1, b2, eps, G, maxG, L_trace_dev, out)) < 0) return st;
  } else {
    const bool tuning = !cluster && !mixed && kernel != 6 && h->opt.autotune > 0 &&
                        h->tuned_rounds < h->opt.autotune && iters >= 20;
    cudaError_t e;
    if (tuning) {
      for (cudaEvent_t& ev : h->tune_ev)
        if (!ev && (e = cudaEventCreate(&ev))) return cuda_fail(e, "creating the tuner's events");
      if ((e = cudaEventRecord(h->tune_ev[0], h->stream))) return cuda_fail(e, "timing the run");
    }
    if ((st = fp64_run(h, mode, iters, 0, true, mixed, b1, b2, eps, G, maxG, L_trace_dev,
                       x_trace_dev, n_trace, out, cluster, kernel)))
      return st;
    if (tuning) {
      float ms = 0.f;
      if ((e = cudaEventRecord(h->tune_ev[1], h->stream)) ||
          (e = cudaEventSynchronize(h->tune_ev[1])) ||
          (e = cudaEventElapsedTime(&ms, h->tune_ev[0], h->tune_ev[1])))
        return cuda_fail(e, "timing the run");
      h->last_run_ms = ms;
    }
    double* keep = mode == PA_SIGMA_MAX ? h->xmin_max : h->xmin_min;
    e = launch_unpermute(h->n_cols, 1, h->sq.pos, pick64h(h, out->minb), keep, h->stream,
                         &h->launches);
    if (e != cudaSuccess) return cuda_fail(e, "keeping x_min");
    h->cont.valid = false;
    if ((st = status_error(out))) return st;
    if (kernel == 0 && !mixed && out->status == PA_OK) {
      pa_ctx::Cont& c = h->cont;
      c.valid = true;
      c.mode = mode;
      c.t_done = out->iters_run;
      c.t_min = out->t_min;
      c.have_best = out->have_best;
      c.best_s = out->best_s;
      c.best_q = out->best_q;
      c.cur = out->cur;
      c.minb = out->minb;
      c.G = G;
      c.cluster = cluster;
      c.lr = lr; c.b1 = b1; c.b2 = b2; c.eps = eps;
    }
  }
  if (mode == PA_SIGMA_MAX) { h->sigma_max = out->sigma; h->have_max = true; }
  else { h->sigma_min = out->sigma; h->have_min = true; h->have_min_direct = true; }
  // the partition tuner learns from plain FP64 grid-engine runs long enough
  // to time (the FP32 and compensated kernels have other cost profiles)
  if (!cluster && !mixed && h->last_kernel != 6 && h->opt.autotune > 0 &&
      h->tuned_rounds < h->opt.autotune && iters >= 20 &&
      (st = tune_partitions(h, h->last_run_ms / iters)))
    return st;
  return (pa_status)out->status;
}

// ------------------------------------------------ Algorithm 2 (LU route) --

static pa_status free_lu(pa_ctx* h) {
  for (void* b : h->lu_bufs) dev_free(h, b);
  h->lu_bufs.clear();
  h->have_lu = false;
  h->lc_ready = false;
  h->lu_p = nullptr;
  return PA_OK;
}

template <typename T>
static pa_status upload(pa_ctx* h, const std::vector<T>& v, T** out, const char* what) {
  pa_status st = alloc_n(h, out, std::max<size_t>(v.size(), 1), what);
  if (st) return st;
  h->lu_bufs.push_back((void*)*out);
  if (!v.empty()) {
    cudaError_t e = cudaMemcpyAsync(*out, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice,
                                    h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // v is pageable
    if (e != cudaSuccess) return cuda_fail(e, what);
  }
  return PA_OK;
}

template <typename T>
static pa_status to_host(pa_ctx* h, const T* src, size_t count, int kind, std::vector<T>* out) {
  out->resize(count);
  if (count == 0) return PA_OK;
  if (kind == PA_HOST) {
    std::copy(src, src + count, out->begin());
    return PA_OK;
  }
  cudaError_t e = cudaMemcpyAsync(out->data(), src, sizeof(T) * count, cudaMemcpyDeviceToHost,
                                  h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? PA_OK : cuda_fail(e, "reading the LU factors");
}

static pa_status upload_rows(pa_ctx* h, const TriRowsHost& t, TriRows* out) {
  int32_t *rp, *ci, *order;
  double *va, *dinv;
  pa_status st;
  if ((st = upload(h, t.rp, &rp, "LU rows")) || (st = upload(h, t.ci, &ci, "LU rows")) ||
      (st = upload(h, t.va, &va, "LU rows")) || (st = upload(h, t.dinv, &dinv, "LU rows")) ||
      (st = upload(h, t.order, &order, "LU rows")))
    return st;
  *out = TriRows{rp, ci, va, dinv, order};
  return PA_OK;
}

static pa_status upload_tri(pa_ctx* h, const TriHost& t, TriSys* out) {
  double *dinv, *va;
  int4 *linfo, *items;
  int32_t* ci;
  pa_status st;
  if ((st = upload(h, t.dinv, &dinv, "LU factor")) || (st = upload(h, t.linfo, &linfo, "LU steps")) ||
      (st = upload(h, t.items, &items, "LU steps")) || (st = upload(h, t.ci, &ci, "LU factor")) ||
      (st = upload(h, t.va, &va, "LU factor")))
    return st;
  *out = TriSys{t.nproc, t.max_items, t.max_ent, dinv, linfo, items, ci, va};
  return PA_OK;
}

// Whether the LU route runs on a cluster (once its form is built): engine
// CLUSTER, or AUTO when the solve vector does not fit one CTA's shared memory
// or the factors have kLuClusterMinRows rows or more.
static bool lu_on_cluster(const pa_ctx* h, const LuParams& p) {
  return h->opt.engine == PA_ENGINE_CLUSTER ||
         (h->opt.engine != PA_ENGINE_GRID && (p.smem_mode == 0 || p.n >= kLuClusterMinRows));
}

static bool is_permutation(const std::vector<int32_t>& p, int32_t n) {
  std::vector<char> seen((size_t)n, 0);
  for (int32_t v : p) {
    if (v < 0 || v >= n || seen[v]) return false;
    seen[v] = 1;
  }
  return true;
}

extern "C" pa_status pa_attach_lu(pa_handle h, const int32_t* l_row_ptr, const int32_t* l_col,
                                  const double* l_val, const int32_t* u_row_ptr,
                                  const int32_t* u_col, const double* u_val, const int32_t* p,
                                  const int32_t* q, int ptr_kind) {
  NvtxRange nvtx_range("pa_attach_lu");
  g_err.clear();
  if (!h || !l_row_ptr || !u_row_ptr) return fail(PA_ERR_INVALID_ARG, "NULL handle or row_ptr");
  if (h->n_rows != h->n_cols)
    return fail(PA_ERR_NOT_SQUARE, "the LU route needs a square matrix (%d x %d)", h->n_rows, h->n_cols);
  if (ptr_kind != PA_HOST && ptr_kind != PA_DEVICE)
    return fail(PA_ERR_INVALID_ARG, "ptr_kind must be PA_HOST or PA_DEVICE");
  const int32_t n = h->n_rows;
  pa_status st;
  std::vector<int32_t> lrp, urp, lci, uci, pp, qq;
  std::vector<double> lva, uva;
  if ((st = to_host(h, l_row_ptr, (size_t)n + 1, ptr_kind, &lrp)) ||
      (st = to_host(h, u_row_ptr, (size_t)n + 1, ptr_kind, &urp)))
    return st;
  for (const auto* rp : {&lrp, &urp}) {
    if ((*rp)[0] != 0) return fail(PA_ERR_INVALID_ARG, "factor row_ptr[0] != 0");
    for (int32_t i = 0; i < n; ++i)
      if ((*rp)[i + 1] < (*rp)[i]) return fail(PA_ERR_INVALID_ARG, "factor row_ptr decreases");
  }
  if ((lrp[n] > 0 && (!l_col || !l_val)) || (urp[n] > 0 && (!u_col || !u_val)))
    return fail(PA_ERR_INVALID_ARG, "NULL factor arrays");
  if ((st = to_host(h, l_col, (size_t)lrp[n], ptr_kind, &lci)) ||
      (st = to_host(h, l_val, (size_t)lrp[n], ptr_kind, &lva)) ||
      (st = to_host(h, u_col, (size_t)urp[n], ptr_kind, &uci)) ||
      (st = to_host(h, u_val, (size_t)urp[n], ptr_kind, &uva)) ||
      (p && (st = to_host(h, p, (size_t)n, ptr_kind, &pp))) ||
      (q && (st = to_host(h, q, (size_t)n, ptr_kind, &qq))))
    return st;
  if ((p && !is_permutation(pp, n)) || (q && !is_permutation(qq, n)))
    return fail(PA_ERR_INVALID_ARG, "p or q is not a permutation of 0..n-1");
  // the four systems: L t = w, U u = t, U^T a = u (rows of U^T: increasing
  // source row), L^T c = a (rows of L^T: decreasing source row, the order in
  // which back substitution meets them)
  std::vector<int32_t> utrp, utci, ltrp, ltci;
  std::vector<double> utva, ltva;
  csr_transpose_host(n, urp.data(), uci.data(), uva.data(), false, &utrp, &utci, &utva);
  csr_transpose_host(n, lrp.data(), lci.data(), lva.data(), true, &ltrp, &ltci, &ltva);
  TriHost tl, tu, tut, tlt;
  std::string why;
  if (!(why = tri_analyse(n, lrp.data(), lci.data(), lva.data(), true, &tl)).empty())
    return fail(PA_ERR_INVALID_ARG, "L: %s", why.c_str());
  if (!(why = tri_analyse(n, urp.data(), uci.data(), uva.data(), false, &tu)).empty())
    return fail(PA_ERR_INVALID_ARG, "U: %s", why.c_str());
  if (!(why = tri_analyse(n, utrp.data(), utci.data(), utva.data(), true, &tut)).empty())
    return fail(PA_ERR_INVALID_ARG, "U^T: %s", why.c_str());
  if (!(why = tri_analyse(n, ltrp.data(), ltci.data(), ltva.data(), false, &tlt)).empty())
    return fail(PA_ERR_INVALID_ARG, "L^T: %s", why.c_str());
  // q only relabels u: ||r|| = ||Q u|| = ||u|| and s needs Q^T r = u, so the
  // iteration never applies it (it is checked above for the caller's sake)
  free_lu(h);
  if ((st = upload_tri(h, tl, &h->lu_sys[0])) || (st = upload_tri(h, tu, &h->lu_sys[1])) ||
      (st = upload_tri(h, tut, &h->lu_sys[2])) || (st = upload_tri(h, tlt, &h->lu_sys[3])) ||
      (p && (st = upload(h, pp, &h->lu_p, "LU permutation"))))
    return (free_lu(h), st);
  {  // the cluster kernel's form, where that kernel may run (lu_on_cluster)
    LuParams probe{};
    probe.n = n;
    probe.L = h->lu_sys[0];
    probe.U = h->lu_sys[1];
    probe.Ut = h->lu_sys[2];
    probe.Lt = h->lu_sys[3];
    lu_layout(&probe);
    if (lu_on_cluster(h, probe) && lu_cluster_plan(n, &h->lc_plan)) {
      const TriHost* ts[4] = {&tl, &tu, &tut, &tlt};
      LcHost c;
      for (int k = 0; k < 4; ++k) {
        lc_build(*ts[k], h->lc_plan.lgC, h->lc_plan.cap, &c);
        int4 *stream, *batch;
        int32_t* bbase;
        uint8_t* fin0;
        if ((st = upload(h, c.stream, &stream, "LU cluster steps")) ||
            (st = upload(h, c.batch, &batch, "LU cluster steps")) ||
            (st = upload(h, c.bbase, &bbase, "LU cluster steps")) ||
            (st = upload(h, c.fin0, &fin0, "LU cluster steps")))
          return (free_lu(h), st);
        h->lc_sys[k] = LcSys{c.nproc, stream, batch, bbase, fin0, h->lu_sys[k].dinv};
      }
      h->lc_ready = true;
    }
    h->lu_route = h->lc_ready && lu_on_cluster(h, probe)
                      ? 2
                      : (h->opt.engine == PA_ENGINE_GRID || probe.smem_mode == 0 ||
                                 h->opt.engine == PA_ENGINE_CLUSTER
                             ? 1
                             : 0);
  }
  {  // the row form for the grid kernel
    TriRowsHost r;
    const int32_t* rps[4] = {lrp.data(), urp.data(), utrp.data(), ltrp.data()};
    const int32_t* cis[4] = {lci.data(), uci.data(), utci.data(), ltci.data()};
    const double* vas[4] = {lva.data(), uva.data(), utva.data(), ltva.data()};
    for (int k = 0; k < 4; ++k) {
      tri_rows_host(n, rps[k], cis[k], vas[k], k % 2 == 0, &r);
      if ((st = upload_rows(h, r, &h->lu_rows[k]))) return (free_lu(h), st);
    }
    if ((st = alloc_n(h, &h->lu_y4, (size_t)4 * n, "LU solve vectors"))) return (free_lu(h), st);
    h->lu_bufs.push_back(h->lu_y4);
  }
  if (!h->xmin_lu &&
      ((st = alloc_n(h, &h->xmin_lu, (size_t)n, "x_min")) ||
       (st = alloc_n(h, &h->lu_w, (size_t)n, "LU vectors")) ||
       (st = alloc_n(h, &h->lu_y, (size_t)n, "LU vectors"))))
    return (free_lu(h), st);
  h->have_lu = true;
  return PA_OK;
}

// Algorithm 1 on A^{-1} from x0 (device, source order, n entries); x_last
// stays in h->dx's sibling buffer X0.  sigma_min(A) = 1 / ||A^{-1} x_min||.
static pa_status lu_run(pa_ctx* h, const double* x0, int iters, double lr, double b1, double b2,
                        double eps, double* L_trace_dev, double* x_trace_dev, int n_trace,
                        RunState* out) {
  if (!h->have_lu) return fail(PA_ERR_INVALID_ARG, "no LU factors attached (pa_attach_lu)");
  h->cont.valid = false;  // the LU route reuses the iterate and moment buffers
  pa_status st;
  if ((st = ensure_bias(h, iters, lr, b1, b2, eps))) return st;
  const size_t n = (size_t)h->n_cols;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(h->X0, x0, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream)) ||
      (e = cudaMemcpyAsync(h->xmin_lu, x0, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream)) ||
      (e = cudaMemsetAsync(h->m, 0, sizeof(double) * n, h->stream)) ||
      (e = cudaMemsetAsync(h->v, 0, sizeof(double) * n, h->stream)) ||
      (e = cudaMemsetAsync(h->st, 0, sizeof(RunState), h->stream)))
    return cuda_fail(e, "preparing the LU-route run");
  LuParams p{};
  p.n = h->n_rows;
  p.L = h->lu_sys[0];
  p.U = h->lu_sys[1];
  p.Ut = h->lu_sys[2];
  p.Lt = h->lu_sys[3];
  p.p = h->lu_p;
  p.x = h->X0;
  p.xmin = h->xmin_lu;
  p.m = h->m;
  p.v = h->v;
  p.dx = h->dx;
  p.w = h->lu_w;
  p.y = h->lu_y;
  p.bias = h->bias;
  p.L_trace = L_trace_dev;
  p.x_trace = x_trace_dev;
  p.n_trace = n_trace;
  p.st = h->st;
  p.iters = iters;
  p.t0 = 0;
  p.beta1 = b1;
  p.beta2 = b2;
  const size_t smem = lu_layout(&p);
  // the route chosen when the factors were attached (h->lu_route): one CTA
  // stepping through the levels while the solve vector fits in its shared
  // memory and the factors are small; past that, one cluster with the solve
  // vector in distributed shared memory while it fits there, else the whole
  // grid (engine GRID forces the grid; CLUSTER the cluster when the vector
  // fits)
  const bool cluster = h->lu_route == 2, grid = h->lu_route == 1;
  const int C = cluster ? 1 << h->lc_plan.lgC : 0;
  h->lu_last_kernel = cluster ? 2 : (grid ? 1 : 0);
  if (grid || cluster) {
    const int G = cluster ? C : lu_grid_max_blocks();
    if (G <= 0) return fail(PA_ERR_LAUNCH, "the LU grid kernel does not fit on this GPU");
    if (h->lu_part_G < G) {
      if (h->lu_part) dev_free(h, h->lu_part);
      h->lu_part = nullptr;
      if ((st = alloc_n(h, &h->lu_part, (size_t)4 * G, "LU partials"))) return st;
      h->lu_part_G = G;
    }
    LuGridParams g{};
    g.n = p.n;
    for (int k = 0; k < 4; ++k) {
      g.sys[k] = h->lu_rows[k];
      g.y[k] = h->lu_y4 + (size_t)k * p.n;
    }
    g.p = p.p;
    g.x = p.x; g.xmin = p.xmin; g.m = p.m; g.v = p.v; g.dx = p.dx; g.w = p.w;
    g.partials = h->lu_part;
    g.bias = p.bias;
    g.L_trace = p.L_trace; g.x_trace = p.x_trace; g.n_trace = p.n_trace;
    g.st = p.st;
    g.iters = p.iters; g.t0 = p.t0;
    g.beta1 = p.beta1; g.beta2 = p.beta2;
    g.timeout_ns = h->opt.barrier_timeout_ns;
    LuClusterParams cp{};
    cp.g = g;
    for (int k = 0; k < 4; ++k) cp.sys[k] = h->lc_sys[k];
    if ((e = cluster ? launch_lu_cluster(cp, h->lc_plan, h->stream, &h->launches)
                     : launch_lu_grid(g, G, h->stream, &h->launches)) ||
        (e = cudaMemcpyAsync(out, h->st, sizeof(RunState), cudaMemcpyDeviceToHost, h->stream)) ||
        (e = cudaStreamSynchronize(h->stream)))
      return cuda_fail(e, cluster ? "running the LU route on a cluster"
                                  : "running the LU route on the grid");
  } else {
    if (!h->lu_params && (st = alloc_n(h, &h->lu_params, 1, "LU run parameters"))) return st;
    if ((e = cudaMemcpyAsync(h->lu_params, &p, sizeof(LuParams), cudaMemcpyHostToDevice, h->stream)) ||
        (e = cudaStreamSynchronize(h->stream)) ||  // p lives on this stack frame
        (e = launch_lu_iter(h->lu_params, 1, smem, p.smem_mode == 1, h->stream, &h->launches)) ||
        (e = cudaMemcpyAsync(out, h->st, sizeof(RunState), cudaMemcpyDeviceToHost, h->stream)) ||
        (e = cudaStreamSynchronize(h->stream)))
      return cuda_fail(e, "running the LU route");
  }
  if ((st = status_error(out))) return st;
  const double sig_inv = out->sigma;  // ||A^{-1} x_min|| / ||x_min||
  out->sigma = 1.0 / sig_inv;
  h->sigma_min = out->sigma;
  h->have_min = true;
  h->have_min_lu = true;
  h->last_kernel = cluster ? 7 : (grid ? 5 : 4);
  h->last_refreshes = 0;
  return (pa_status)out->status;
}

// pa_run for PA_SIGMA_MIN_LU: everything in source order, no permutations.
static pa_status run_lu_traced(pa_ctx* h, int iters, double lr, double b1, double b2, double eps,
                               const double* x_init, int x_kind, double* x_min, double* x_last,
                               double* info, double* L_trace, double* x_trace, int n_trace,
                               double* sigma) {
  const size_t n = (size_t)h->n_cols;
  cudaError_t e = cudaMemcpyAsync(h->Xinit, x_init, sizeof(double) * n,
                                  x_kind == PA_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                  h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "copying x_init");
  pa_status st;
  double *Ld = nullptr, *Xd = nullptr;
  if (L_trace && iters > 0 && (st = alloc_n(h, &Ld, (size_t)iters, "L trace"))) return st;
  if (x_trace && n_trace > 0 && (st = alloc_n(h, &Xd, (size_t)n_trace * n, "x trace"))) {
    if (Ld) dev_free(h, Ld);
    return st;
  }
  RunState rs{};
  pa_status rst = lu_run(h, h->Xinit, iters, lr, b1, b2, eps, Ld, Xd, x_trace ? n_trace : 0, &rs);
  if (rst >= 0) {
    if (x_min) e = cudaMemcpyAsync(x_min, h->xmin_lu, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && x_last)
      e = cudaMemcpyAsync(x_last, h->X0, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && Ld)
      e = cudaMemcpyAsync(L_trace, Ld, sizeof(double) * iters, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && Xd)
      e = cudaMemcpyAsync(x_trace, Xd, sizeof(double) * n_trace * n, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) rst = cuda_fail(e, "reading results");
    if (rst >= 0) {
      if (info) {
        info[0] = rs.L_min;
        info[1] = rs.t_min;
        info[2] = rs.L_last;
        info[3] = rs.iters_run;
      }
      if (sigma) *sigma = rs.sigma;
    }
  }
  if (Ld) dev_free(h, Ld);
  if (Xd) dev_free(h, Xd);
  return rst;
}

extern "C" pa_status pa_run(pa_handle h, pa_mode mode, int iters, double lr, double beta1,
                            double beta2, double eps, const double* x_init, int x_kind,
                            double* x_min, double* x_last, double* info, double* L_trace,
                            double* x_trace, int n_trace, double* sigma) {
  NvtxRange nvtx_range("pa_run");
  g_err.clear();
  if (!h) return fail(PA_ERR_INVALID_ARG, "NULL handle");
  if (mode != PA_SIGMA_MAX && mode != PA_SIGMA_MIN && mode != PA_SIGMA_MIN_LU)
    return fail(PA_ERR_INVALID_ARG, "pa_run takes PA_SIGMA_MAX, PA_SIGMA_MIN or PA_SIGMA_MIN_LU");
  if (!x_init) return fail(PA_ERR_INVALID_ARG, "x_init is NULL");
  if (x_kind != PA_HOST && x_kind != PA_DEVICE) return fail(PA_ERR_INVALID_ARG, "bad x_kind");
  if (n_trace < 0 || n_trace > iters) return fail(PA_ERR_INVALID_ARG, "n_trace must lie in [0, iters]");
  pa_status st;
  if ((st = check_hyper(iters, lr, beta1, beta2, eps)) || (st = ensure_run_buffers(h))) return st;
  const size_t n = (size_t)h->n_cols;
  if (mode == PA_SIGMA_MIN_LU) return run_lu_traced(h, iters, lr, beta1, beta2, eps, x_init, x_kind,
                                                    x_min, x_last, info, L_trace, x_trace, n_trace,
                                                    sigma);
  // x_init arrives in source order; the kernels work in the column order Q
  cudaError_t e = cudaMemcpyAsync(h->dx, x_init, sizeof(double) * n,
                                  x_kind == PA_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                  h->stream);
  if (e == cudaSuccess)
    e = launch_permute(h->n_cols, h->sq.pos, h->dx, h->Xinit, h->stream, &h->launches);
  if (e != cudaSuccess) return cuda_fail(e, "copying x_init");
  double *Ld = nullptr, *Xd = nullptr;
  if (L_trace && iters > 0 && (st = alloc_n(h, &Ld, (size_t)iters, "L trace"))) return st;
  if (x_trace && n_trace > 0 && (st = alloc_n(h, &Xd, (size_t)n_trace * n, "x trace"))) {
    if (Ld) dev_free(h, Ld);
    return st;
  }
  RunState rs{};
  pa_status rst = run_one(h, mode, iters, lr, beta1, beta2, eps, Ld, Xd, x_trace ? n_trace : 0, &rs);
  if (rst >= 0) {
    double* xs[3] = {h->X0, h->X1, h->X2};
    double* keep = mode == PA_SIGMA_MAX ? h->xmin_max : h->xmin_min;  // source order
    if (x_min) e = cudaMemcpyAsync(x_min, keep, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && x_last) {
      e = launch_unpermute(h->n_cols, 1, h->sq.pos, xs[rs.cur], h->dx, h->stream, &h->launches);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(x_last, h->dx, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream);
    }
    if (e == cudaSuccess && Ld)
      e = cudaMemcpyAsync(L_trace, Ld, sizeof(double) * iters, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && Xd) {
      double* Xs = nullptr;
      if (alloc_n(h, &Xs, (size_t)n_trace * n, "x trace") != PA_OK) {
        e = cudaErrorMemoryAllocation;
      } else {
        e = launch_unpermute(h->n_cols, n_trace, h->sq.pos, Xd, Xs, h->stream, &h->launches);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(x_trace, Xs, sizeof(double) * n_trace * n, cudaMemcpyDeviceToHost,
                              h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        dev_free(h, Xs);
      }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) rst = cuda_fail(e, "reading results");
    if (rst >= 0) {
      if (info) {
        info[0] = rs.L_min;
        info[1] = rs.t_min;
        info[2] = rs.L_last;
        info[3] = rs.iters_run;
      }
      if (sigma) *sigma = rs.sigma;
    }
  }
  if (Ld) dev_free(h, Ld);
  if (Xd) dev_free(h, Xd);
  return rst;
}

extern "C" pa_status pa_continue(pa_handle h, int iters, double lr, double beta1, double beta2,
                                 double eps, double* sigma, double* x_last, double* info) {
  NvtxRange nvtx_range("pa_continue");
  g_err.clear();
  if (!h) return fail(PA_ERR_INVALID_ARG, "NULL handle");
  pa_ctx::Cont& c = h->cont;
  if (!c.valid)
    return fail(PA_ERR_INVALID_ARG,
                "nothing to continue: the handle's latest run was not a successful FP64 run "
                "of the three-phase or cluster kernel");
  if (lr != c.lr || beta1 != c.b1 || beta2 != c.b2 || eps != c.eps)
    return fail(PA_ERR_INVALID_ARG, "pa_continue needs the hyperparameters of the run it continues");
  pa_status st;
  if ((st = check_hyper(iters, lr, beta1, beta2, eps))) return st;
  if ((long long)c.t_done + iters > INT_MAX) return fail(PA_ERR_INVALID_ARG, "too many iterations");
  if ((st = ensure_bias(h, c.t_done + iters, lr, beta1, beta2, eps))) return st;
  // x_T to X0, x_min to X1 (through the step buffer, so that no copy
  // overwrites the other's source)
  const size_t n = (size_t)h->n_cols;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(h->dx, pick64h(h, c.cur), sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream)) ||
      (c.minb != 1 &&
       (e = cudaMemcpyAsync(h->X1, pick64h(h, c.minb), sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream))) ||
      (e = cudaMemcpyAsync(h->X0, h->dx, sizeof(double) * n, cudaMemcpyDeviceToDevice, h->stream)))
    return cuda_fail(e, "preparing the continued run");
  const int maxG = c.G;
  RunState rs{};
  const pa_ctx::Cont prev = c;
  c.valid = false;
  if ((st = fp64_run(h, (pa_mode)prev.mode, iters, prev.t_done, false, false, beta1, beta2, eps,
                     prev.G, maxG, nullptr, nullptr, 0, &rs, prev.cluster, 0, &prev)))
    return st;
  double* keep = prev.mode == PA_SIGMA_MAX ? h->xmin_max : h->xmin_min;
  if ((e = launch_unpermute(h->n_cols, 1, h->sq.pos, pick64h(h, rs.minb), keep, h->stream,
                            &h->launches)))
    return cuda_fail(e, "keeping x_min");
  if ((st = status_error(&rs))) return st;
  if (rs.status == PA_OK) {
    c = prev;
    c.valid = true;
    c.t_done = prev.t_done + rs.iters_run;
    c.t_min = rs.t_min;
    c.have_best = rs.have_best;
    c.best_s = rs.best_s;
    c.best_q = rs.best_q;
    c.cur = rs.cur;
    c.minb = rs.minb;
  }
  if (prev.mode == PA_SIGMA_MAX) { h->sigma_max = rs.sigma; h->have_max = true; }
  else { h->sigma_min = rs.sigma; h->have_min = true; h->have_min_direct = true; }
  if (x_last) {
    if ((e = launch_unpermute(h->n_cols, 1, h->sq.pos, pick64h(h, rs.cur), h->dx, h->stream,
                              &h->launches)) ||
        (e = cudaMemcpyAsync(x_last, h->dx, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream)))
      return cuda_fail(e, "reading x_last");
  }
  if ((e = cudaStreamSynchronize(h->stream))) return cuda_fail(e, "reading results");
  if (sigma) *sigma = rs.sigma;
  if (info) {
    info[0] = rs.L_min;
    info[1] = rs.t_min;
    info[2] = rs.L_last;
    info[3] = prev.t_done + rs.iters_run;
  }
  return (pa_status)rs.status;
}

extern "C" pa_status pa_estimate(pa_handle h, pa_mode mode, int iters, double lr, double beta1,
                                 double beta2, double eps, uint64_t seed, double* sigma_max,
                                 double* sigma_min, double* kappa) {
  NvtxRange nvtx_range("pa_estimate");
  g_err.clear();
  if (!h) return fail(PA_ERR_INVALID_ARG, "NULL handle");
  if (mode != PA_SIGMA_MAX && mode != PA_SIGMA_MIN && mode != PA_BOTH &&
      mode != PA_SIGMA_MIN_LU && mode != PA_BOTH_LU)
    return fail(PA_ERR_INVALID_ARG, "unknown mode %d", (int)mode);
  if ((mode & PA_SIGMA_MIN_LU) && !h->have_lu)
    return fail(PA_ERR_INVALID_ARG, "no LU factors attached (pa_attach_lu)");
  pa_status st;
  if ((st = check_hyper(iters, lr, beta1, beta2, eps)) || (st = ensure_run_buffers(h))) return st;
  if ((mode & PA_SIGMA_MIN) && h->n_rows < h->n_cols)
    return fail(PA_ERR_NOT_SQUARE, "sigma_min needs n_rows >= n_cols (%d x %d)", h->n_rows, h->n_cols);
  cudaError_t e = launch_start_vector(h->n_cols, seed, h->sq.pos, h->Xinit, h->blockpart, h->stream,
                                      &h->launches);
  if (e != cudaSuccess) return cuda_fail(e, "building the start vector");
  pa_status worst = PA_OK;
  RunState rs{};
  for (int md : {PA_SIGMA_MAX, PA_SIGMA_MIN, PA_SIGMA_MIN_LU}) {
    if (!(mode & md)) continue;
    if (md == PA_SIGMA_MIN_LU) {  // the same start vector, in source order
      if ((e = launch_unpermute(h->n_cols, 1, h->sq.pos, h->Xinit, h->dx, h->stream, &h->launches)))
        return cuda_fail(e, "building the start vector");
      st = lu_run(h, h->dx, iters, lr, beta1, beta2, eps, nullptr, nullptr, 0, &rs);
    } else {
      st = run_one(h, (pa_mode)md, iters, lr, beta1, beta2, eps, nullptr, nullptr, 0, &rs);
    }
    if (st < 0) return st;
    if (st > worst) worst = st;
  }
  if (sigma_max) *sigma_max = h->have_max ? h->sigma_max : NAN;
  if (sigma_min) *sigma_min = h->have_min ? h->sigma_min : NAN;
  if (kappa) {
    if (h->have_max && h->have_min)
      *kappa = h->sigma_min > 0 ? h->sigma_max / h->sigma_min : INFINITY;
    else
      *kappa = NAN;
  }
  return worst;
}

extern "C" pa_status pa_get_vector(pa_handle h, pa_mode which, double* x_min_host) {
  g_err.clear();
  if (!h || !x_min_host) return fail(PA_ERR_INVALID_ARG, "NULL argument");
  if (which != PA_SIGMA_MAX && which != PA_SIGMA_MIN && which != PA_SIGMA_MIN_LU)
    return fail(PA_ERR_INVALID_ARG, "bad mode");
  if ((which == PA_SIGMA_MAX && !h->have_max) || (which == PA_SIGMA_MIN && !h->have_min_direct) ||
      (which == PA_SIGMA_MIN_LU && !h->have_min_lu))
    return fail(PA_ERR_INVALID_ARG, "no run of that mode yet");
  double* src = which == PA_SIGMA_MAX ? h->xmin_max
                                      : (which == PA_SIGMA_MIN ? h->xmin_min : h->xmin_lu);
  cudaError_t e = cudaMemcpyAsync(x_min_host, src, sizeof(double) * h->n_cols,
                                  cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "reading x_min");
  return PA_OK;
}

// y = A x (or z = A^T y) through the sliced copies: permute the input into
// the kernel order, multiply, map the output back to source order.
static pa_status product(pa_handle h, bool transposed, const double* in, double* out, int kind) {
  g_err.clear();
  if (!h || !in || !out) return fail(PA_ERR_INVALID_ARG, "NULL argument");
  if (kind != PA_HOST && kind != PA_DEVICE) return fail(PA_ERR_INVALID_ARG, "bad ptr_kind");
  const Sell& M = transposed ? h->sq : h->sa;
  const int32_t* pos_in = transposed ? h->sa.pos : h->sq.pos;
  const int32_t n_in = transposed ? h->n_rows : h->n_cols;
  const int32_t n_out = transposed ? h->n_cols : h->n_rows;
  pa_status st;
  double *a = nullptr, *ap = nullptr, *bp = nullptr, *b = nullptr;
  if ((st = alloc_n(h, &a, (size_t)n_in, "product input")) ||
      (st = alloc_n(h, &ap, (size_t)n_in, "product input")) ||
      (st = alloc_n(h, &bp, (size_t)n_out, "product output")) ||
      (st = alloc_n(h, &b, (size_t)n_out, "product output")))
    return st;
  cudaError_t e = cudaMemcpyAsync(a, in, sizeof(double) * n_in,
                                  kind == PA_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                  h->stream);
  if (e == cudaSuccess) e = launch_permute(n_in, pos_in, a, ap, h->stream, &h->launches);
  if (e == cudaSuccess) e = launch_sell_spmv(M, ap, bp, h->stream, &h->launches);
  if (e == cudaSuccess) e = launch_unpermute(n_out, 1, M.pos, bp, b, h->stream, &h->launches);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, b, sizeof(double) * n_out,
                        kind == PA_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  dev_free(h, a);
  dev_free(h, ap);
  dev_free(h, bp);
  dev_free(h, b);
  if (e != cudaSuccess) return cuda_fail(e, "sparse product");
  return PA_OK;
}

extern "C" pa_status pa_spmv(pa_handle h, const double* x, double* y, int ptr_kind) {
  NvtxRange nvtx_range("pa_spmv");
  return product(h, false, x, y, ptr_kind);
}

extern "C" pa_status pa_spmv_t(pa_handle h, const double* y, double* z, int ptr_kind) {
  NvtxRange nvtx_range("pa_spmv_t");
  return product(h, true, y, z, ptr_kind);
}

extern "C" pa_status pa_spmv_ata(pa_handle h, const double* x, double* z, int ptr_kind) {
  NvtxRange nvtx_range("pa_spmv_ata");
  g_err.clear();
  if (!h || !x || !z) return fail(PA_ERR_INVALID_ARG, "NULL argument");
  if (ptr_kind != PA_HOST && ptr_kind != PA_DEVICE) return fail(PA_ERR_INVALID_ARG, "bad ptr_kind");
  pa_status st;
  if ((st = ensure_run_buffers(h))) return st;
  int maxG = 0;
  int G = choose_grid(h, &maxG);
  if (G <= 0) return fail(PA_ERR_LAUNCH, "the persistent kernel does not fit on this GPU");
  const int gs = single_max_blocks(h->opt.loss);
  if (gs > 0) G = std::min(G, gs);
  if ((st = ensure_single(h, G))) return st;
  const int32_t n = h->n_cols;
  double *a = nullptr, *ap = nullptr, *zp = nullptr, *zb = nullptr;
  if ((st = alloc_n(h, &a, (size_t)n, "product input")) ||
      (st = alloc_n(h, &ap, (size_t)n, "product input")) ||
      (st = alloc_n(h, &zp, (size_t)n, "product output")) ||
      (st = alloc_n(h, &zb, (size_t)n, "product output")))
    return st;
  IterParams p{};
  p.n_rows = h->n_rows;
  p.n_cols = h->n_cols;
  p.a_wp = h->sa.wp; p.a_col = h->sa.col; p.a_val = h->sa.val;
  p.y = h->y;
  single_params(h, &p);
  cudaError_t e = cudaMemcpyAsync(a, x, sizeof(double) * n,
                                  ptr_kind == PA_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                  h->stream);
  if (e == cudaSuccess) e = launch_permute(n, h->sq.pos, a, ap, h->stream, &h->launches);
  if (e == cudaSuccess) e = launch_single_product(p, G, ap, zp, h->stream, &h->launches);
  if (e == cudaSuccess) e = launch_unpermute(n, 1, h->sq.pos, zp, zb, h->stream, &h->launches);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(z, zb, sizeof(double) * n,
                        ptr_kind == PA_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  dev_free(h, a);
  dev_free(h, ap);
  dev_free(h, zp);
  dev_free(h, zb);
  if (e != cudaSuccess) return cuda_fail(e, "single-pass product");
  return PA_OK;
}

extern "C" pa_status pa_launch_choice(pa_handle h, int64_t* out, int64_t* cand, double* ms) {
  g_err.clear();
  if (!h || !out) return fail(PA_ERR_INVALID_ARG, "NULL argument");
  out[0] = h->launch_kernel;
  out[1] = h->launch_G;
  out[2] = h->launch_source;
  out[3] = (int64_t)h->launch_cands.size();
  for (size_t i = 0; i < h->launch_cands.size() && i < 4; ++i) {
    if (cand) {
      cand[2 * i] = h->launch_cands[i][0];
      cand[2 * i + 1] = h->launch_cands[i][1];
    }
    if (ms) ms[i] = h->launch_ms[i];
  }
  return PA_OK;
}

extern "C" pa_status pa_single_pass_info(pa_handle h, int64_t* out) {
  g_err.clear();
  if (!h || !out) return fail(PA_ERR_INVALID_ARG, "NULL argument");
  out[0] = h->sp_G;
  out[1] = h->sp_window_cols;
  out[2] = h->sp_plan_entries;
  out[3] = h->sp_plan_slots;
  out[4] = h->sp_groups;
  out[5] = h->a_entries;
  return PA_OK;
}

extern "C" pa_status pa_lu_route_info(pa_handle h, int64_t* out) {
  g_err.clear();
  if (!h || !out) return fail(PA_ERR_INVALID_ARG, "NULL argument");
  if (!h->have_lu) return fail(PA_ERR_INVALID_ARG, "no LU factors attached (pa_attach_lu)");
  const bool cl = h->lu_route == 2;
  out[0] = h->lu_route;
  out[1] = cl ? 1 << h->lc_plan.lgC : 0;
  out[2] = cl ? h->lc_plan.cap : 0;
  out[3] = cl ? h->lc_plan.fin : 0;
  return PA_OK;
}

extern "C" pa_status pa_get_transpose(pa_handle h, int32_t* row_ptr_t, int32_t* col_t, double* val_t) {
  g_err.clear();
  if (!h) return fail(PA_ERR_INVALID_ARG, "NULL handle");
  cudaError_t e = cudaSuccess;
  if (row_ptr_t)
    e = cudaMemcpyAsync(row_ptr_t, h->rpt, sizeof(int32_t) * ((size_t)h->n_cols + 1),
                        cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess && col_t && h->nnz)
    e = cudaMemcpyAsync(col_t, h->cit, sizeof(int32_t) * h->nnz, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess && val_t && h->nnz)
    e = cudaMemcpyAsync(val_t, h->vat, sizeof(double) * h->nnz, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "reading the transpose");
  return PA_OK;
}

extern "C" pa_status pa_last_run_info(pa_handle h, int64_t* out) {
  g_err.clear();
  if (!h || !out) return fail(PA_ERR_INVALID_ARG, "NULL argument");
  out[0] = h->last_kernel;
  out[1] = h->last_refreshes;
  out[2] = h->df_fallbacks;
  out[3] = h->last_G;
  return PA_OK;
}

extern "C" pa_status pa_last_run_profile(pa_handle h, int* grid, double* busy_ns) {
  g_err.clear();
  if (!h || !grid) return fail(PA_ERR_INVALID_ARG, "NULL argument");
  *grid = h->last_G;
  if (!busy_ns || h->last_G == 0) return PA_OK;
  std::vector<unsigned long long> t((size_t)2 * h->last_G);
  cudaError_t e = cudaMemcpyAsync(t.data(), h->cta_ns, sizeof(unsigned long long) * t.size(),
                                  cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "reading the run profile");
  for (size_t i = 0; i < t.size(); ++i) busy_ns[i] = (double)t[i];
  return PA_OK;
}

extern "C" pa_status pa_error_bounds(pa_handle h, const double* x_hat, const double* b,
                                     int ptr_kind, double kappa, double norm_a, double u,
                                     double* out) {
  NvtxRange nvtx_range("pa_error_bounds");
  g_err.clear();
  if (!h || !x_hat || !b || !out) return fail(PA_ERR_INVALID_ARG, "NULL handle or pointer");
  if (ptr_kind != PA_HOST && ptr_kind != PA_DEVICE)
    return fail(PA_ERR_INVALID_ARG, "ptr_kind must be PA_HOST or PA_DEVICE");
  if (!(kappa > 0.0)) {
    if (!h->have_max || !h->have_min)
      return fail(PA_ERR_INVALID_ARG, "kappa not given and the handle has no sigma_max and sigma_min estimates");
    kappa = h->sigma_max / h->sigma_min;
  }
  if (!(norm_a > 0.0)) {
    if (!h->have_max) return fail(PA_ERR_INVALID_ARG, "||A|| not given and the handle has no sigma_max estimate");
    norm_a = h->sigma_max;
  }
  if (!(u > 0.0)) u = 0x1.0p-53;
  pa_status st;
  if ((st = ensure_run_buffers(h))) return st;
  if (!h->eb_part &&
      ((st = alloc_n(h, &h->eb_part, (size_t)3 * kErrorBoundMaxBlocks, "error-bound partials")) ||
       (st = alloc_n(h, &h->eb_out, 10, "error bounds"))))
    return st;
  cudaError_t e = cudaSuccess;
  const double* xd = x_hat;
  const double* bd = b;
  if (ptr_kind == PA_HOST) {  // the run's scratch vectors y (n_rows) and dx (>= n_cols)
    if ((e = cudaMemcpyAsync(h->dx, x_hat, sizeof(double) * h->n_cols, cudaMemcpyHostToDevice, h->stream)) ||
        (e = cudaMemcpyAsync(h->y, b, sizeof(double) * h->n_rows, cudaMemcpyHostToDevice, h->stream)))
      return cuda_fail(e, "copying x_hat and b");
    xd = h->dx;
    bd = h->y;
  }
  if ((e = launch_error_bounds(h->n_rows, h->n_cols, h->rp, h->ci, h->va, xd, bd, kappa, norm_a,
                               u, h->eb_part, h->eb_out, h->stream, &h->launches)) ||
      (e = cudaMemcpyAsync(out, h->eb_out, sizeof(double) * 10, cudaMemcpyDeviceToHost, h->stream)) ||
      (e = cudaStreamSynchronize(h->stream)))
    return cuda_fail(e, "evaluating the error bounds");
  return PA_OK;
}

extern "C" pa_status pa_get_equilibration(pa_handle h, double* d_row, double* d_col) {
  g_err.clear();
  if (!h) return fail(PA_ERR_INVALID_ARG, "NULL handle");
  const double* dr = h->tgt_row ? h->tgt_row : h->d_row;
  const double* dc = h->tgt_row ? h->tgt_col : h->d_col;
  if (!dr) return fail(PA_ERR_INVALID_ARG, "the handle holds no equilibration");
  cudaError_t e = cudaSuccess;
  if (d_row)
    e = cudaMemcpyAsync(d_row, dr, sizeof(double) * h->n_rows, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess && d_col)
    e = cudaMemcpyAsync(d_col, dc, sizeof(double) * h->n_cols, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "reading the equilibration");
  return PA_OK;
}

// ------------------------------------------------------------ batched --

namespace {

// Device memory of one batched call, allocated through the first handle and
// released at the end of the call.
struct BatchScratch {
  pa_ctx* h;
  std::vector<void*> ptrs;
  template <class T>
  pa_status get(T** out, size_t count, const char* what) {
    pa_status st = alloc_n(h, out, count, what);
    if (st == PA_OK) ptrs.push_back((void*)*out);
    return st;
  }
  ~BatchScratch() {
    for (void* p : ptrs) dev_free(h, p);
  }
};

// CTAs per item: at least one each, the rest proportional to the work.
std::vector<int> share_ctas(const std::vector<double>& work, int G) {
  const int n = (int)work.size();
  std::vector<int> c(n, 1);
  double tot = 0;
  for (double w : work) tot += w;
  int left = G - n;
  if (left <= 0 || tot <= 0) return c;
  std::vector<std::pair<double, int>> rem;
  int used = 0;
  for (int i = 0; i < n; ++i) {
    const double want = left * work[i] / tot;
    const int f = (int)floor(want);
    c[i] += f;
    used += f;
    rem.push_back({want - f, i});
  }
  std::sort(rem.begin(), rem.end(), [](auto& a, auto& b) { return a.first > b.first || (a.first == b.first && a.second < b.second); });
  for (int k = 0; k < left - used && k < n; ++k) c[rem[k].second] += 1;
  return c;
}

}  // namespace

// One wave of items [i0, i0 + m), restarts [r0, r0 + k_used) as K columns.
static pa_status batched_wave(const pa_handle* hs, int i0, int m, int r0, int k_used, int K,
                              int k_restarts, pa_mode mode, const int* iters, double lr, double b1,
                              double b2, double eps, uint64_t seed, double* out,
                              pa_status* item_status, bool* captured, bool allow_df = true) {
  pa_ctx* h0 = hs[0];
  cudaStream_t s = h0->stream;  // replaced below by a capturable stream joined to it
  BatchScratch sc{h0, {}};
  // PA_DF64: the double-float kernel when every matrix of the wave fits it
  bool dfb = allow_df && h0->opt.precision == PA_DF64;
  for (int i = 0; dfb && i < m; ++i) {
    pa_status sd;
    if ((sd = build_df_values(hs[i0 + i]))) return sd;
    dfb = hs[i0 + i]->df_ok;
  }
  // MIXED: sigma_max runs an FP32 stage (k_batched32) and an FP64 tail
  const bool mixed = h0->opt.precision == PA_MIXED && (mode & PA_SIGMA_MAX);
  const int tail = !mixed ? 0 : (h0->opt.fp64_tail < 0 ? iters[0] / 10 : std::min(h0->opt.fp64_tail, iters[0]));
  const int t32 = iters[0] - tail;
  // ... and sigma_min with Dot2 products, like the single-vector MIXED run
  const bool dd_min = h0->opt.precision == PA_MIXED && (mode & PA_SIGMA_MIN);
  // the co-resident grid of the kernels this wave launches
  int Gmax = dfb ? batched_df_max_blocks(K) : batched_max_blocks(K);
  if (mixed) Gmax = std::min(Gmax, batched32_max_blocks(K));
  if (dd_min) Gmax = std::min(Gmax, batched_max_blocks(K, true));
  if (Gmax < m) return fail(PA_ERR_LAUNCH, "batched kernel: %d items exceed %d co-resident CTAs", m, Gmax);
  // ---- CTA groups, sized by padded entries plus a per-row weight
  std::vector<double> work(m);
  for (int i = 0; i < m; ++i) {
    const pa_ctx* hi = hs[i0 + i];
    work[i] = (double)hi->a_entries + (double)hi->t_entries + 40.0 * std::max(hi->n_rows, hi->n_cols);
  }
  const std::vector<int> ncta = share_ctas(work, Gmax);
  int G = 0;
  for (int c : ncta) G += c;
  std::vector<BatchItem> items(m);
  std::vector<int32_t> cta_item(G);
  std::vector<int32_t> blk_item, blk_row0, item_blk0(m + 1);
  pa_status st;
  cudaError_t e = cudaSuccess;
  int cta = 0;
  for (int i = 0; i < m; ++i) {
    pa_ctx* hi = hs[i0 + i];
    BatchItem& it = items[i];
    const size_t nx = (size_t)hi->n_cols * K, ny = (size_t)hi->n_rows * K;
    it.n_rows = hi->n_rows;
    it.n_cols = hi->n_cols;
    it.a_wp = hi->sa.wp; it.a_col = hi->sa.col; it.a_val = hi->sa.val;
    it.t_wp = hi->sq.wp; it.t_col = hi->sq.col; it.t_val = hi->sq.val;
    it.pos_c = hi->sq.pos;
    it.n_slices_a = hi->sa.n_slices;
    if (dfb) {
      it.a_val2 = hi->a_val2;
      it.t_val2 = hi->t_val2;
      it.s_scale = ldexp(1.0, 2 * hi->df_k);
    }
    it.cta0 = cta;
    it.ncta = ncta[i];
    for (int c = 0; c < ncta[i]; ++c) cta_item[cta + c] = i;
    cta += ncta[i];
    int32_t *pa_ = nullptr, *pt_ = nullptr;
    if ((st = sc.get(&pa_, (size_t)ncta[i] + 1, "batch partition")) ||
        (st = sc.get(&pt_, (size_t)ncta[i] + 1, "batch partition")) ||
        (st = sc.get(&it.partials, (size_t)ncta[i] * 4 * K, "batch partials")) ||
        (st = sc.get(&it.barrier, 1, "batch barrier")) ||
        (st = sc.get(&it.X0, nx, "batch x")) || (st = sc.get(&it.X1, nx, "batch x")) ||
        (st = sc.get(&it.XMIN, nx, "batch x_min")) || (st = sc.get(&it.M, nx, "batch m")) ||
        (st = sc.get(&it.V, nx, "batch v")) || (st = sc.get(&it.DX, nx, "batch dx")) ||
        (st = sc.get(&it.Y, std::max<size_t>(ny, 1), "batch y")) ||
        (st = sc.get(&it.result, (size_t)4 * K, "batch result")) ||
        (st = sc.get(&it.status, 3, "batch status")))  // [1] the FP32 stage's, [2] sigma_max's
      return st;
    if (dd_min && (st = sc.get(&it.YLO, std::max<size_t>(ny, 1), "batch y (low parts)"))) return st;
    if (mixed) {
      it.a_val32 = hi->a_val32;
      it.t_val32 = hi->t_val32;
      it.dr32 = hi->drp32;
      it.dc32 = hi->dcp32;
      if ((st = sc.get(&it.X0f, nx, "batch x (FP32)")) || (st = sc.get(&it.X1f, nx, "batch x (FP32)")) ||
          (st = sc.get(&it.XMINf, nx, "batch x_min (FP32)")) || (st = sc.get(&it.Mf, nx, "batch m (FP32)")) ||
          (st = sc.get(&it.Vf, nx, "batch v (FP32)")) || (st = sc.get(&it.DXf, nx, "batch dx (FP32)")) ||
          (st = sc.get(&it.Wf, nx, "batch w (FP32)")) ||
          (st = sc.get(&it.Yf, std::max<size_t>(ny, 1), "batch y (FP32)")))
        return st;
    }
    if ((e = launch_partition(hi->sa.wp, hi->sa.n_slices, ncta[i], 2, pa_, s, &h0->launches)) ||
        (e = launch_partition(hi->sq.wp, hi->sq.n_slices, ncta[i], 30, pt_, s, &h0->launches)))
      return cuda_fail(e, "partitioning a batch item");
    it.part_a = pa_;
    it.part_t = pt_;
    // blocks of 256 rows over max(n_rows, n_cols) for the start and sigma kernels
    item_blk0[i] = (int32_t)blk_item.size();
    const int rows = std::max(hi->n_rows, hi->n_cols);
    for (int r = 0; r < rows; r += 256) {
      blk_item.push_back(i);
      blk_row0.push_back(r);
    }
  }
  item_blk0[m] = (int32_t)blk_item.size();
  const int nb = (int)blk_item.size();
  BatchItem* items_d = nullptr;
  int32_t *cta_item_d = nullptr, *blk_item_d = nullptr, *blk_row0_d = nullptr, *item_blk0_d = nullptr;
  double *blockpart = nullptr, *sig = nullptr;
  RunState* rs_d = nullptr;
  if ((st = sc.get(&items_d, (size_t)m, "batch items")) ||
      (st = sc.get(&cta_item_d, (size_t)G, "batch table")) ||
      (st = sc.get(&blk_item_d, (size_t)nb, "batch table")) ||
      (st = sc.get(&blk_row0_d, (size_t)nb, "batch table")) ||
      (st = sc.get(&item_blk0_d, (size_t)m + 1, "batch table")) ||
      (st = sc.get(&blockpart, (size_t)nb * 2 * K + (size_t)m * K + 64, "batch block partials")) ||
      (st = sc.get(&sig, (size_t)3 * m * K, "batch sigma")) ||  // max, min, FP32-stage max
      (st = sc.get(&rs_d, 1, "batch run state")))
    return st;
  const int T = std::max(iters[0], iters[1]);
  std::vector<double2> tab((size_t)std::max(T, 1));
  for (int t = 1; t <= T; ++t) {
    const double r2 = sqrt(1.0 - pow(b2, (double)t));
    tab[t - 1] = make_double2(lr * r2 / (1.0 - pow(b1, (double)t)), eps * r2);
  }
  double2* bias_d = nullptr;
  if ((st = sc.get(&bias_d, tab.size(), "batch bias table"))) return st;
  // the same constants as double-word pairs: hi = float(K), lo = float(K - hi)
  std::vector<float4> tab2(dfb ? tab.size() : 0);
  for (size_t t = 0; t < tab2.size(); ++t) {
    const float k1 = (float)tab[t].x, k2 = (float)tab[t].y;
    tab2[t] = make_float4(k1, (float)(tab[t].x - (double)k1), k2, (float)(tab[t].y - (double)k2));
  }
  float4* bias2_d = nullptr;
  if (dfb && (st = sc.get(&bias2_d, tab2.size(), "batch bias table (double-float)"))) return st;
  if (dfb && (e = cudaMemcpyAsync(bias2_d, tab2.data(), sizeof(float4) * tab2.size(),
                                  cudaMemcpyHostToDevice, s)))
    return cuda_fail(e, "uploading the batch tables");
  // tables to the device (pageable host memory: synchronous copies, before capture)
  if ((e = cudaMemcpyAsync(items_d, items.data(), sizeof(BatchItem) * m, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(cta_item_d, cta_item.data(), sizeof(int32_t) * G, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(blk_item_d, blk_item.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(blk_row0_d, blk_row0.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(item_blk0_d, item_blk0.data(), sizeof(int32_t) * (m + 1), cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(bias_d, tab.data(), sizeof(double2) * tab.size(), cudaMemcpyHostToDevice, s)) ||
      (e = cudaStreamSynchronize(s)))
    return cuda_fail(e, "uploading the batch tables");

  BatchParams bp{};
  bp.items = items_d;
  bp.cta_item = cta_item_d;
  bp.bias = bias_d;
  bp.st = rs_d;
  bp.loss = h0->opt.loss;
  bp.ablation = h0->opt.ablation;
  bp.beta1 = b1;
  bp.w2 = (1.0 - b2) / ((1.0 - b1) * (1.0 - b1));
  bp.beta2 = b2;
  bp.timeout_ns = h0->opt.barrier_timeout_ns;
  bp.bias2 = bias2_d;

  // The whole call as one sequence: start vectors, state reset, the
  // persistent launch, sigma -- for sigma_max, then sigma_min.
  int64_t n_launch = 0;
  auto enqueue = [&]() -> cudaError_t {
    int64_t* L = &n_launch;
    cudaError_t err = cudaSuccess;
    for (int md : {PA_SIGMA_MAX, PA_SIGMA_MIN}) {
      if (!(mode & md)) continue;
      // item i, restart r: SplitMix64 output i * k_restarts + r of `seed`
      err = launch_batch_start(items_d, m, K, k_used, k_restarts, i0, r0, seed, blk_item_d,
                               blk_row0_d, nb, 256, blockpart, item_blk0_d, s, L);
      if (err) return err;
      if ((err = cudaMemsetAsync(rs_d, 0, sizeof(RunState), s))) return err;
      for (int i = 0; i < m; ++i) {
        const size_t nx = (size_t)items[i].n_cols * K;
        // the sigma_max pass clears all three status slots, so no slot that
        // the host combines below is ever read unwritten
        const size_t n_status = md == PA_SIGMA_MAX || !(mode & PA_SIGMA_MAX) ? 3 : 1;
        if ((err = cudaMemsetAsync(items[i].M, 0, sizeof(double) * nx, s)) ||
            (err = cudaMemsetAsync(items[i].V, 0, sizeof(double) * nx, s)) ||
            (err = cudaMemsetAsync(items[i].barrier, 0, sizeof(unsigned), s)) ||
            (err = cudaMemsetAsync(items[i].status, 0, sizeof(int) * n_status, s)))
          return err;
      }
      BatchParams q = bp;
      q.mode = md;
      q.iters = md == PA_SIGMA_MAX ? iters[0] : iters[1];
      if (md == PA_SIGMA_MAX && mixed) {
        // FP32 stage from the same start vectors; its minimisers scored in FP64
        for (int i = 0; i < m; ++i) {
          const size_t nx = (size_t)items[i].n_cols * K;
          if ((err = launch_convert((int64_t)nx, items[i].X0, items[i].X0f, s, L)) ||
              (err = launch_convert((int64_t)nx, items[i].X0, items[i].XMINf, s, L)) ||  // x_min = x_init
              (err = cudaMemsetAsync(items[i].Mf, 0, sizeof(float) * nx, s)) ||
              (err = cudaMemsetAsync(items[i].Vf, 0, sizeof(float) * nx, s)))
            return err;
        }
        q.iters = t32;
        if ((err = launch_batched32(q, K, G, s, L))) return err;
        for (int i = 0; i < m; ++i)
          if ((err = launch_convert((int64_t)items[i].n_cols * K, items[i].XMINf, items[i].XMIN, s, L)))
            return err;
        if ((err = launch_batch_sigma(items_d, m, K, blk_item_d, blk_row0_d, nb, 256, blockpart,
                                      item_blk0_d, sig + (size_t)2 * m * K, false, s, L)))
          return err;
        if (tail == 0) {  // the FP32 stage was all of sigma_max: keep its status
          if (mode & PA_SIGMA_MIN)
            for (int i = 0; i < m; ++i)
              if ((err = cudaMemcpyAsync(items[i].status + 2, items[i].status, sizeof(int),
                                         cudaMemcpyDeviceToDevice, s)))
                return err;
          continue;
        }
        // the FP64 tail continues from the last FP32 iterate and moments
        for (int i = 0; i < m; ++i) {
          const size_t nx = (size_t)items[i].n_cols * K;
          const float* xl = (t32 % 2 == 0) ? items[i].X0f : items[i].X1f;
          if ((err = launch_convert((int64_t)nx, xl, items[i].X0, s, L)) ||
              (err = launch_convert((int64_t)nx, items[i].Mf, items[i].M, s, L)) ||
              (err = launch_convert((int64_t)nx, items[i].Vf, items[i].V, s, L)) ||
              (err = cudaMemcpyAsync(items[i].status + 1, items[i].status, sizeof(int),
                                     cudaMemcpyDeviceToDevice, s)) ||
              (err = cudaMemsetAsync(items[i].barrier, 0, sizeof(unsigned), s)))
            return err;
        }
        q.t0 = t32;
        q.iters = tail;
      }
      const bool dd = md == PA_SIGMA_MIN && dd_min;
      if (dfb) {
        // x_init and x_min as float pairs in place, the double-float run,
        // then x_min back to FP64 for the sigma kernel
        for (int i = 0; i < m; ++i) {
          const int64_t nx = (int64_t)items[i].n_cols * K;
          if ((err = launch_split_df(nx, items[i].X0, 0, reinterpret_cast<float2*>(items[i].X0), s, L)) ||
              (err = launch_split_df(nx, items[i].XMIN, 0, reinterpret_cast<float2*>(items[i].XMIN), s, L)))
            return err;
        }
        if ((err = launch_batched_df(q, K, G, s, L))) return err;
        for (int i = 0; i < m; ++i)
          if ((err = launch_join_df((int64_t)items[i].n_cols * K,
                                    reinterpret_cast<const float2*>(items[i].XMIN), items[i].XMIN, s, L)))
            return err;
      } else if ((err = launch_batched(q, K, G, dd, s, L))) {
        return err;
      }
      if ((err = launch_batch_sigma(items_d, m, K, blk_item_d, blk_row0_d, nb, 256, blockpart,
                                    item_blk0_d, sig + (md == PA_SIGMA_MAX ? 0 : (size_t)m * K), dd,
                                    s, L)))
        return err;
      if (md == PA_SIGMA_MAX && (mode & PA_SIGMA_MIN))  // keep sigma_max's status
        for (int i = 0; i < m; ++i)
          if ((err = cudaMemcpyAsync(items[i].status + 2, items[i].status, sizeof(int),
                                     cudaMemcpyDeviceToDevice, s)))
            return err;
    }
    return cudaSuccess;
  };
  // Capture the sequence into a CUDA graph on a library-owned stream that
  // joins the handle's stream (the legacy default stream cannot be
  // captured); if capture or instantiation is refused, run the same sequence
  // on that stream directly.
  const cudaStream_t user = s;
  cudaStream_t cs = nullptr;
  cudaEvent_t ev = nullptr;
  if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) ||
      (e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) ||
      (e = cudaEventRecord(ev, user)) || (e = cudaStreamWaitEvent(cs, ev, 0))) {
    if (cs) cudaStreamDestroy(cs);
    if (ev) cudaEventDestroy(ev);
    return cuda_fail(e, "preparing the batch stream");
  }
  s = cs;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  *captured = false;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    const cudaError_t ce = enqueue();
    const cudaError_t ee = cudaStreamEndCapture(s, &graph);
    if (ce == cudaSuccess && ee == cudaSuccess && graph &&
        cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess)
      *captured = true;
    cudaGetLastError();  // a refused capture leaves a sticky-free error here
  }
  if (*captured) {
    e = cudaGraphLaunch(exec, s);  // replays the n_launch kernels counted during capture
  } else {
    n_launch = 0;
    e = enqueue();
  }
  h0->launches += n_launch;
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  cudaEventRecord(ev, s);
  cudaStreamWaitEvent(user, ev, 0);
  cudaStreamSynchronize(s);
  cudaEventDestroy(ev);
  cudaStreamDestroy(cs);
  s = user;
  if (e != cudaSuccess) return cuda_fail(e, "running the batched launch");
  // ---- results
  std::vector<double> sg((size_t)3 * m * K);
  RunState rs{};
  if ((e = cudaMemcpyAsync(sg.data(), sig, sizeof(double) * sg.size(), cudaMemcpyDeviceToHost, s)) ||
      (e = cudaMemcpyAsync(&rs, rs_d, sizeof(RunState), cudaMemcpyDeviceToHost, s)) ||
      (e = cudaStreamSynchronize(s)))
    return cuda_fail(e, "reading the batched results");
  std::vector<int> ist(m, PA_OK);
  for (int i = 0; i < m; ++i) {
    int v[3] = {0, 0, 0};
    if ((e = cudaMemcpy(v, items[i].status, sizeof(v), cudaMemcpyDeviceToHost)))
      return cuda_fail(e, "reading the batched status");
    if (dfb && (v[0] == kStatusDfRange || v[1] == kStatusDfRange || v[2] == kStatusDfRange)) {
      // a column left the double-float range: the whole wave again in FP64
      ++h0->df_fallbacks;
      return batched_wave(hs, i0, m, r0, k_used, K, k_restarts, mode, iters, lr, b1, b2, eps,
                          seed, out, item_status, captured, false);
    }
    // the item's status over every launch that ran for it: the first error
    // (< 0), else a warning (> 0), else PA_OK
    int worst = v[0];
    const bool have[3] = {true, mixed && tail > 0, mode == PA_BOTH};
    for (int j = 1; j < 3; ++j) {
      if (!have[j]) continue;
      if (v[j] < 0 && worst >= 0) worst = v[j];
      else if (v[j] > 0 && worst == 0) worst = v[j];
    }
    ist[i] = worst;
  }
  if (rs.abort) return fail(PA_ERR_TIMEOUT, "a batched group barrier wait ran out of time");
  for (int i = 0; i < m; ++i) {
    for (int c = 0; c < k_used; ++c) {
      const int r = r0 + c;
      double* o = out + ((size_t)(i0 + i) * k_restarts + r) * 3;
      double smax = (mode & PA_SIGMA_MAX) ? sg[(size_t)i * K + c] : NAN;
      if (mixed) {  // the stage whose tracked minimiser scores the larger sigma in FP64
        const double s32 = sg[(size_t)2 * m * K + (size_t)i * K + c];
        smax = (tail == 0 || s32 > smax) ? s32 : smax;
      }
      const double smin = (mode & PA_SIGMA_MIN) ? sg[(size_t)m * K + (size_t)i * K + c] : NAN;
      o[0] = smax;
      o[1] = smin;
      o[2] = (mode == PA_BOTH) ? (smin > 0 ? smax / smin : INFINITY) : NAN;
      if (item_status) item_status[(size_t)(i0 + i) * k_restarts + r] = (pa_status)ist[i];
    }
  }
  return PA_OK;
}

static thread_local int g_last_batch_graph = 0;
extern "C" int pa_last_batch_graph(void) { return g_last_batch_graph; }

// sigma_min of every (matrix, restart) item through the matrices' attached LU
// factors (Algorithm 2): one CTA per item runs k_lu_iter on its own vectors,
// from the start vector of the same seed the SpMM engine gives that item (in
// source order).  Fills out[item][1] (and [2] when sigma_max ran).
static pa_status batched_lu(const pa_handle* hs, int n_mat, int k_restarts, int iters, double lr,
                            double b1, double b2, double eps, uint64_t seed, bool have_max,
                            double* out, pa_status* item_status) {
  pa_ctx* h0 = hs[0];
  const cudaStream_t s = h0->stream;
  BatchScratch sc{h0, {}};
  const int n_items = n_mat * k_restarts;
  pa_status st;
  cudaError_t e;
  // bias corrections, shared by the items
  std::vector<double2> tab((size_t)std::max(iters, 1));
  for (int t = 1; t <= iters; ++t) {
    const double r2 = sqrt(1.0 - pow(b2, (double)t));
    tab[t - 1] = make_double2(lr * r2 / (1.0 - pow(b1, (double)t)), eps * r2);
  }
  double2* bias = nullptr;
  RunState* states = nullptr;
  LuParams* items_dev = nullptr;
  int32_t nmax = 0;
  for (int i = 0; i < n_mat; ++i) nmax = std::max(nmax, hs[i]->n_rows);
  double* blockpart = nullptr;
  if ((st = sc.get(&bias, tab.size(), "bias table")) ||
      (st = sc.get(&states, (size_t)n_items, "run states")) ||
      (st = sc.get(&items_dev, (size_t)n_items, "LU items")) ||
      (st = sc.get(&blockpart, (size_t)start_vector_blocks(nmax) + 1, "start vector partials")))
    return st;
  if ((e = cudaMemcpyAsync(bias, tab.data(), sizeof(double2) * tab.size(), cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemsetAsync(states, 0, sizeof(RunState) * n_items, s)))
    return cuda_fail(e, "preparing the LU items");
  std::vector<LuParams> items((size_t)n_items);
  size_t smem = 0;
  bool all_smem = true;
  for (int i = 0; i < n_mat; ++i) {
    pa_ctx* hi = hs[i];
    const size_t n = (size_t)hi->n_rows;
    for (int r = 0; r < k_restarts; ++r) {
      const int it = i * k_restarts + r;
      double* buf = nullptr;
      if ((st = sc.get(&buf, 7 * n, "LU item vectors"))) return st;
      LuParams& p = items[it];
      p.n = hi->n_rows;
      p.L = hi->lu_sys[0];
      p.U = hi->lu_sys[1];
      p.Ut = hi->lu_sys[2];
      p.Lt = hi->lu_sys[3];
      p.p = hi->lu_p;
      p.x = buf;
      p.xmin = buf + n;
      p.m = buf + 2 * n;
      p.v = buf + 3 * n;
      p.dx = buf + 4 * n;
      p.w = buf + 5 * n;
      p.y = buf + 6 * n;
      p.bias = bias;
      p.st = states + it;
      p.iters = iters;
      p.beta1 = b1;
      p.beta2 = b2;
      smem = std::max(smem, lu_layout(&p));
      all_smem = all_smem && p.smem_mode == 1;
      // item (i, r): SplitMix64 output i * k_restarts + r of `seed`, source order
      const uint64_t s_ir = splitmix64_at(seed, (uint64_t)it);
      if ((e = launch_start_vector(hi->n_rows, s_ir, nullptr, p.x, blockpart, s, &h0->launches)) ||
          (e = cudaMemcpyAsync(p.xmin, p.x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s)) ||
          (e = cudaMemsetAsync(p.m, 0, sizeof(double) * 2 * n, s)))
        return cuda_fail(e, "preparing the LU items");
    }
  }
  std::vector<RunState> rs((size_t)n_items);
  // CTAs start in index order: the items with the most solve steps go first,
  // so the last wave holds short items (each item keeps its own run state)
  std::stable_sort(items.begin(), items.end(), [](const LuParams& a, const LuParams& b) {
    const int64_t sa = (int64_t)a.L.nproc + a.U.nproc + a.Ut.nproc + a.Lt.nproc;
    const int64_t sb = (int64_t)b.L.nproc + b.U.nproc + b.Ut.nproc + b.Lt.nproc;
    return sa > sb;
  });
  if ((e = cudaMemcpyAsync(items_dev, items.data(), sizeof(LuParams) * n_items, cudaMemcpyHostToDevice, s)) ||
      (e = launch_lu_iter(items_dev, n_items, smem, all_smem, s, &h0->launches)) ||
      (e = cudaMemcpyAsync(rs.data(), states, sizeof(RunState) * n_items, cudaMemcpyDeviceToHost, s)) ||
      (e = cudaStreamSynchronize(s)))
    return cuda_fail(e, "running the batched LU route");
  for (int it = 0; it < n_items; ++it) {
    double* o = out + (size_t)it * 3;
    o[1] = rs[it].status == PA_OK ? 1.0 / rs[it].sigma : NAN;
    o[2] = have_max ? o[0] / o[1] : NAN;
    if (item_status && rs[it].status != PA_OK) item_status[it] = (pa_status)rs[it].status;
  }
  return PA_OK;
}

// The SpMM engine over all items, restarts in blocks of at most kb columns
// (each block rounded up to a kernel width K in {1, 2, 4, 8}), matrices in
// waves that leave every matrix at least two CTAs.
static pa_status spmm_batches(const pa_handle* handles, int n_mat, int k_restarts, int kb,
                              pa_mode spmm_mode, const int* iters, double lr, double b1, double b2,
                              double eps, uint64_t seed, double* out, pa_status* item_status) {
  bool captured = false;
  pa_status st;
  for (int r0 = 0; r0 < k_restarts; r0 += kb) {
    const int k_used = std::min(kb, k_restarts - r0);
    const int K = k_used <= 1 ? 1 : (k_used <= 2 ? 2 : (k_used <= 4 ? 4 : 8));
    const int Gmax = batched_max_blocks(K);
    if (Gmax <= 0) return fail(PA_ERR_LAUNCH, "the batched kernel does not fit on this GPU");
    const int wave = std::max(1, Gmax / 2);
    for (int i0 = 0; i0 < n_mat; i0 += wave) {
      const int m = std::min(wave, n_mat - i0);
      if ((st = batched_wave(handles, i0, m, r0, k_used, K, k_restarts, spmm_mode, iters, lr, b1,
                             b2, eps, seed, out, item_status, &captured)))
        return st;
      g_last_batch_graph = captured ? 1 : 0;
    }
  }
  return PA_OK;
}

extern "C" pa_status pa_estimate_batched(int n_mat, const pa_handle* handles, pa_mode mode,
                                         int k_restarts, const int* iters, double lr, double beta1,
                                         double beta2, double eps, uint64_t seed, double* out,
                                         pa_status* item_status) {
  NvtxRange nvtx_range("pa_estimate_batched");
  g_err.clear();
  if (n_mat <= 0 || !handles || !iters || !out || k_restarts <= 0)
    return fail(PA_ERR_INVALID_ARG, "invalid batched arguments");
  if (mode != PA_SIGMA_MAX && mode != PA_SIGMA_MIN && mode != PA_BOTH &&
      mode != PA_SIGMA_MIN_LU && mode != PA_BOTH_LU)
    return fail(PA_ERR_INVALID_ARG, "unknown mode %d", (int)mode);
  pa_status st;
  if ((st = check_hyper(std::min(iters[0], iters[1]), lr, beta1, beta2, eps))) return st;
  const bool lu = (mode & PA_SIGMA_MIN_LU) != 0;
  for (int i = 0; lu && i < n_mat; ++i)
    if (!handles[i] || !handles[i]->have_lu)
      return fail(PA_ERR_INVALID_ARG, "handle %d has no LU factors attached", i);
  const pa_mode spmm_mode = (pa_mode)(mode & PA_BOTH);
  for (int i = 0; i < n_mat; ++i) {
    const pa_ctx* hi = handles[i];
    if (!hi) return fail(PA_ERR_INVALID_ARG, "handle %d is NULL", i);
    if (hi->stream != handles[0]->stream)
      return fail(PA_ERR_INVALID_ARG, "all handles of a batch must share one stream");
    if (hi->opt.precision != handles[0]->opt.precision)
      return fail(PA_ERR_INVALID_ARG, "all handles of a batch must share one precision mode (handle %d)", i);
    if ((mode & PA_SIGMA_MIN) && hi->n_rows < hi->n_cols)
      return fail(PA_ERR_NOT_SQUARE, "sigma_min needs n_rows >= n_cols (handle %d)", i);
  }
  if (item_status)
    for (int it = 0; it < n_mat * k_restarts; ++it) item_status[it] = PA_OK;
  if (spmm_mode == 0) {  // PA_SIGMA_MIN_LU alone
    for (int it = 0; it < n_mat * k_restarts; ++it) out[(size_t)it * 3] = NAN;
    return batched_lu(handles, n_mat, k_restarts, iters[1], lr, beta1, beta2, eps, seed, false, out,
                      item_status);
  }
  // restart-block width: K = 8 by default (4 for PA_DF64, whose narrower
  // blocks run three CTAs per SM); with autotune on the first handle, the
  // fastest of 8, 4 and 2 on a short trial of this batch (cached per k)
  pa_ctx* h0 = handles[0];
  int kb = h0->opt.precision == PA_DF64 ? 4 : 8;
  if (h0->opt.autotune > 0 && k_restarts >= 2) {
    auto hit = h0->batch_kb.find(k_restarts);
    if (hit != h0->batch_kb.end()) {
      kb = hit->second;
    } else {
      const int trial[2] = {std::min(iters[0], 30), std::min(iters[1], 30)};
      std::vector<double> scratch((size_t)n_mat * k_restarts * 3);
      double best = INFINITY;
      for (int cand : {8, 4, 2}) {
        if (cand > 2 * k_restarts - 1 && cand != 2) continue;  // wider than the restarts need
        const auto t0 = std::chrono::steady_clock::now();
        if ((st = spmm_batches(handles, n_mat, k_restarts, cand, spmm_mode, trial, lr, beta1,
                               beta2, eps, seed, scratch.data(), nullptr)))
          return st;
        const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (dt < best) { best = dt; kb = cand; }
      }
      h0->batch_kb[k_restarts] = kb;
    }
  }
  if ((st = spmm_batches(handles, n_mat, k_restarts, kb, spmm_mode, iters, lr, beta1, beta2, eps,
                         seed, out, item_status)))
    return st;
  if (lu)
    return batched_lu(handles, n_mat, k_restarts, iters[1], lr, beta1, beta2, eps, seed, true, out,
                      item_status);
  return PA_OK;
}
