// pa_lu.cu -- sigma_min through ||A^{-1}||_2 with a given LU factorisation:
// the paper's Algorithm 2 ("Compute Gradient for A^{-1}") inside Algorithm 1.
//
// With P A Q = L U, A^{-1} = Q U^{-1} L^{-1} P and A^{-T} = P^T L^{-T} U^{-T} Q^T.
// Per iteration, for B = A^{-1}:
//   r = B x        : w = P x, L t = w, U u = t (r = Q u, so ||r|| = ||u||)
//   score          : L(x_{t-1}) = log||x|| - log||r|| against L_min
//   s = B^T r      : U^T a = u, L^T c = a, s = P^T c
//   grad           : x / ||x||^2 - s / ||r||^2   (Algorithm 2)
//   Adam, tangent projection, update, normalisation as in Algorithm 1.
// sigma_min(A) = 1 / sigma_max(B) = ||x_min|| / ||B x_min||.
//
// The four triangular solves are level-scheduled: the host sorts the rows of
// each factor by level (a row's level is one more than the highest level of
// the rows it depends on), and the solve walks the levels in order, the rows
// of one level in parallel.  Sparse LU factors of 2D operators in fill-reducing
// orders have long, thin level sets (hundreds of levels of a few rows for a
// few thousand unknowns), so one CTA runs the whole iteration: a level then
// costs one __syncthreads instead of a grid-wide barrier.  The factors are
// stored in level order, so a level's entries are contiguous and are
// prefetched into L1 two levels ahead; for small n the solve vectors live in
// shared memory.  The kernel waits on nothing outside its CTA.
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "pa_device.cuh"
#include "pa_internal.h"

namespace pa {

std::string tri_analyse(int32_t n, const int32_t* rp, const int32_t* ci, const double* va,
                        bool lower, TriHost* out) {
  out->rp.assign((size_t)n + 1, 0);
  out->ci.clear();
  out->va.clear();
  out->diag.assign((size_t)n, 0.0);
  std::vector<int32_t> level((size_t)n, 0);
  for (int32_t i = 0; i < n; ++i) {
    bool have_diag = false;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
      const int32_t j = ci[k];
      if (j < 0 || j >= n) return "column index out of range in row " + std::to_string(i);
      if (j == i) {
        if (have_diag) return "two diagonal entries in row " + std::to_string(i);
        have_diag = true;
        out->diag[i] = va[k];
      } else if ((lower && j > i) || (!lower && j < i)) {
        return std::string(lower ? "entry above the diagonal" : "entry below the diagonal") +
               " in row " + std::to_string(i);
      }
    }
    if (!have_diag || out->diag[i] == 0.0 || !std::isfinite(out->diag[i]))
      return "zero or missing diagonal in row " + std::to_string(i);
  }
  // levels: a forward solve visits rows upwards, a backward solve downwards
  int32_t nlev = 0;
  for (int32_t s = 0; s < n; ++s) {
    const int32_t i = lower ? s : n - 1 - s;
    int32_t lv = 0;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
      if (ci[k] != i) lv = std::max(lv, level[ci[k]] + 1);
    level[i] = lv;
    nlev = std::max(nlev, lv + 1);
  }
  out->lvl.assign((size_t)nlev + 1, 0);
  for (int32_t i = 0; i < n; ++i) ++out->lvl[level[i] + 1];
  for (int32_t k = 0; k < nlev; ++k) out->lvl[k + 1] += out->lvl[k];
  out->order.assign((size_t)n, 0);
  std::vector<int32_t> cur(out->lvl.begin(), out->lvl.end() - 1);
  for (int32_t i = 0; i < n; ++i) out->order[cur[level[i]]++] = i;
  // rows in level order, each with its off-diagonal entries in stored order
  std::vector<double> diag_row(out->diag);
  for (int32_t k = 0; k < n; ++k) {
    const int32_t i = out->order[k];
    for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
      if (ci[e] == i) continue;
      out->ci.push_back(ci[e]);
      out->va.push_back(va[e]);
    }
    out->rp[k + 1] = (int32_t)out->ci.size();
    out->diag[k] = 1.0 / diag_row[i];  // the solve multiplies by the reciprocal
  }
  // packed per-level and per-position records: one load each in the solve
  out->lvinfo.resize((size_t)nlev);
  for (int32_t l = 0; l < nlev; ++l)
    out->lvinfo[l] = make_int4(out->lvl[l], out->lvl[l + 1], out->rp[out->lvl[l]],
                               out->rp[out->lvl[l + 1]]);
  out->pos.resize((size_t)n);
  for (int32_t k = 0; k < n; ++k) out->pos[k] = make_int4(out->rp[k], out->rp[k + 1], out->order[k], 0);
  return std::string();
}

void csr_transpose_host(int32_t n, const int32_t* rp, const int32_t* ci, const double* va,
                        bool reverse, std::vector<int32_t>* trp, std::vector<int32_t>* tci,
                        std::vector<double>* tva) {
  trp->assign((size_t)n + 1, 0);
  for (int32_t k = 0; k < rp[n]; ++k) ++(*trp)[ci[k] + 1];
  for (int32_t j = 0; j < n; ++j) (*trp)[j + 1] += (*trp)[j];
  tci->assign((size_t)rp[n], 0);
  tva->assign((size_t)rp[n], 0.0);
  std::vector<int32_t> cur(trp->begin(), trp->end() - 1);
  for (int32_t s = 0; s < n; ++s) {
    const int32_t i = reverse ? n - 1 - s : s;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
      const int32_t j = ci[k];
      (*tci)[cur[j]] = i;
      (*tva)[cur[j]] = va[k];
      ++cur[j];
    }
  }
}

namespace {

constexpr int kLuWarps = kLuThreads / 32;

struct LuShared {
  double scratch[2 * kLuThreads];
  double ca, cb;      // g' = (1 - beta1) grad = ca x + cb s
  double c, inv;      // projection coefficient and 1 / ||x'||
  double q_keep;      // ||x||^2 of the current iterate
  double L_min, L_last;
  int brk, improved;
  int t_min, iters_run, status;
};

// The solve vectors: in dynamic shared memory for small n, else global.
struct LuVec {
  double *w, *t, *u, *a, *c;
};

// Ask L1 for what level `lev` reads (its positions and entries are
// contiguous: position records, diagonals, columns, values).  Called by the
// warps that have no row in the current level, `first` being the first of
// them; every prefetched address lies inside its array.
__device__ __forceinline__ void prefetch_level(const TriSys& T, int lev, int first) {
  if (lev >= T.nlev) return;
  const int4 L = T.lvinfo[lev];
  const int nr = L.y - L.x, ne = L.w - L.z;
  const char* base[4] = {reinterpret_cast<const char*>(T.pos + L.x),
                         reinterpret_cast<const char*>(T.diag + L.x),
                         reinterpret_cast<const char*>(T.ci + L.z),
                         reinterpret_cast<const char*>(T.va + L.z)};
  const int bytes[4] = {16 * nr, 8 * nr, 4 * ne, 8 * ne};
  int l = (int)threadIdx.x - 32 * first;
  for (int r = 0; r < 4; ++r) {
    const int nl = (bytes[r] + 127) / 128;
    for (; l < nl; l += kLuThreads - 32 * first)
      asm volatile("prefetch.global.L1 [%0];" ::"l"(base[r] + 128 * l));
    l -= nl;
  }
}

// x = T^{-1} b for one level-scheduled triangular system (all threads): a
// warp per row, its lanes striding the row's entries, then a fixed-order
// butterfly sum and one multiply by the stored reciprocal of the diagonal.
// A level's time is the latency of that chain of FP64 instructions (each
// occupies GB300's narrow FP64 pipe for many cycles), so the division is
// replaced by the reciprocal, and the warps without a row in the level
// prefetch the next two levels meanwhile.  The rounding differs from plain
// substitution; the route's iterates are insensitive to it at the 1e-15 level.
__device__ __forceinline__ void tri_solve(const TriSys& T, const double* b, double* x) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int lev = 0; lev < T.nlev; ++lev) {
    const int4 L = T.lvinfo[lev];
    const int rows = L.y - L.x;
    if (warp >= rows) {  // idle this level: fetch the next two
      prefetch_level(T, lev + 1, rows);
      prefetch_level(T, lev + 2, rows);
    }
    for (int k = L.x + warp; k < L.y; k += kLuWarps) {
      const int4 P = T.pos[k];
      double acc = 0.0;
      for (int e = P.x + lane; e < P.y; e += 32) acc = fma(T.va[e], x[T.ci[e]], acc);
      // butterfly over the lanes that hold entries (a row of 9 entries needs
      // 4 levels, not 5); the level count is the same for the whole warp
      const int len = P.y - P.x;
#pragma unroll
      for (int d = 16; d > 0; d >>= 1)
        if (d < len) acc += __shfl_xor_sync(0xffffffffu, acc, d);
      if (lane == 0) x[P.z] = (b[P.z] - acc) * T.diag[k];
    }
    __syncthreads();
  }
}

// u = Q^T A^{-1} x: w = P x, L t = w, U u = t.
__device__ __forceinline__ void apply_inv(const LuParams& p, const LuVec& V, const double* x) {
  for (int i = threadIdx.x; i < p.n; i += kLuThreads) V.w[i] = x[p.p ? p.p[i] : i];
  __syncthreads();
  tri_solve(p.L, V.w, V.t);
  tri_solve(p.U, V.t, V.u);
}

// One CTA per item: item b runs Algorithm 1 on the inverse of its own matrix
// from its own start vector, independently of the other CTAs.
__global__ void __launch_bounds__(kLuThreads, 1) k_lu_iter(const LuParams* __restrict__ items) {
  const LuParams& p = items[blockIdx.x];
  __shared__ LuShared sh;
  extern __shared__ double dyn[];
  const int n = p.n, tid = threadIdx.x;
  LuVec V;
  if (p.smem_mode >= 1) {
    V = LuVec{dyn, dyn + n, dyn + 2 * n, dyn + 3 * n, dyn + 4 * n};
  } else {
    V = LuVec{p.w, p.t, p.u, p.a, p.c};
  }
  if (tid == 0) {
    sh.L_min = INFINITY;
    sh.L_last = NAN;
    sh.t_min = 0;
    sh.iters_run = 0;
    sh.status = PA_OK;
  }
  __syncthreads();
  double* x = p.x;
  for (int t = 1;; ++t) {
    // ---- r = A^{-1} x (Algorithm 2: solve L U r = x), ||r||^2, ||x||^2
    apply_inv(p, V, x);
    {
      double v[2] = {0.0, 0.0};
      for (int i = tid; i < n; i += kLuThreads) {
        v[0] = fma(V.u[i], V.u[i], v[0]);
        v[1] = fma(x[i], x[i], v[1]);
      }
      block_sum_to0<2>(v, sh.scratch);
      if (tid == 0) {
        const double rr = v[0], q2 = v[1];
        int brk = 0, improved = 0;
        if (!isfinite(rr) || !isfinite(q2) || rr == 0.0) {
          sh.status = PA_ERR_NONFINITE;
          brk = 1;
        } else {
          if (t > 1) {  // score x_{t-1}: L = log||x|| - log||A^{-1} x||
            const double L = log(sqrt(q2)) - log(sqrt(rr));
            sh.L_last = L;
            if (p.L_trace) p.L_trace[t - 2] = L;
            if (L < sh.L_min) {
              sh.L_min = L;
              sh.t_min = t - 1;
              improved = 1;
            }
          }
          if (t == p.iters + 1) brk = 1;
        }
        const double omb1 = 1.0 - p.beta1;
        sh.ca = omb1 / q2;
        sh.cb = -omb1 / rr;
        sh.q_keep = q2;
        sh.brk = brk;
        sh.improved = improved;
      }
      __syncthreads();
    }
    if (sh.improved) {
      for (int i = tid; i < n; i += kLuThreads) p.xmin[i] = x[i];
      __syncthreads();  // the final sigma reads x_min across threads
    }
    if (sh.brk) break;

    // ---- s = A^{-T} r (Algorithm 2: solve U^T L^T s = r), into w
    tri_solve(p.Ut, V.u, V.a);
    tri_solve(p.Lt, V.a, V.c);
    for (int i = tid; i < n; i += kLuThreads) V.w[p.p ? p.p[i] : i] = V.c[i];
    __syncthreads();

    // ---- gradient x/||x||^2 - s/||r||^2, Adam, partials x.dx and dx.dx
    {
      const double ca = sh.ca, cb = sh.cb;
      const double2 bc = p.bias[p.t0 + t - 1];
      const double b1 = p.beta1, b2 = p.beta2;
      const double w2 = (1.0 - b2) / ((1.0 - b1) * (1.0 - b1));
      double v[2] = {0.0, 0.0};
      for (int j = tid; j < n; j += kLuThreads) {
        const double xj = x[j];
        const double g = fma(ca, xj, cb * V.w[j]);
        const double mj = fma(b1, p.m[j], g);
        const double vj = fma(b2, p.v[j], w2 * (g * g));
        p.m[j] = mj;
        p.v[j] = vj;
        const double d = adam_quotient(bc.x * mj, vj, bc.y);
        p.dx[j] = d;
        v[0] = fma(xj, d, v[0]);
        v[1] = fma(d, d, v[1]);
      }
      block_sum_to0<2>(v, sh.scratch);
      if (tid == 0) {
        const double p1 = v[0], p2 = v[1];
        if (!isfinite(p1) || !isfinite(p2)) {
          sh.status = PA_ERR_NONFINITE;
          sh.brk = 1;
        }
        const double a1c = 1.0 + p1;
        // ||(1+c) x - dx||^2 = (1+c)^2 q - 2 (1+c) p1 + p2, c = x.dx
        const double nrm2 = fma(a1c * a1c, sh.q_keep, fma(-2.0 * a1c, p1, p2));
        sh.c = p1;
        sh.inv = 1.0 / sqrt(nrm2);
      }
      __syncthreads();
    }
    if (sh.brk) break;

    // ---- x_t = ((1 + c) x - dx) / ||.||: projection, update, normalisation
    {
      const double a1c = 1.0 + sh.c, inv = sh.inv;
      double* tr = (p.x_trace && t <= p.n_trace) ? p.x_trace + (size_t)(t - 1) * n : nullptr;
      for (int j = tid; j < n; j += kLuThreads) {
        const double xn = fma(a1c, x[j], -p.dx[j]) * inv;
        x[j] = xn;
        if (tr) tr[j] = xn;
      }
      if (tid == 0) sh.iters_run = t;
      __syncthreads();
    }
  }

  // ---- sigma_max(A^{-1}) = ||A^{-1} x_min|| / ||x_min||
  apply_inv(p, V, p.xmin);
  double v[2] = {0.0, 0.0};
  for (int i = tid; i < n; i += kLuThreads) {
    v[0] = fma(V.u[i], V.u[i], v[0]);
    v[1] = fma(p.xmin[i], p.xmin[i], v[1]);
  }
  block_sum_to0<2>(v, sh.scratch);
  if (tid == 0) {
    RunState* st = p.st;
    st->status = sh.status;
    st->t_min = sh.t_min;
    st->L_min = sh.L_min;
    st->L_last = sh.L_last;
    st->iters_run = sh.iters_run;
    st->sigma = sqrt(v[0]) / sqrt(v[1]);
  }
}

}  // namespace

size_t lu_smem_bytes(const LuParams& p, int mode) {
  if (mode == 0) return 0;
  const size_t b = sizeof(double) * 5 * (size_t)p.n;
  return b <= kLuSmemBudget ? b : 0;
}

cudaError_t launch_lu_iter(const LuParams* items_dev, int n_items, size_t smem, cudaStream_t s,
                           int64_t* launches) {
  if (smem > 0) {
    cudaError_t e = cudaFuncSetAttribute(k_lu_iter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_lu_iter<<<n_items, kLuThreads, smem, s>>>(items_dev);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace pa
