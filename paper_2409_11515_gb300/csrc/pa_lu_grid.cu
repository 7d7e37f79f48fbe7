// pa_lu_grid.cu -- the paper's Algorithm 2 (sigma_min through ||A^{-1}||_2
// with given LU factors) inside Algorithm 1, for factors too large for one
// CTA: the four triangular solves of each iteration run on the whole GPU
// without level barriers.
//
// The single-CTA kernel (pa_lu.cu) steps through the levels of each
// triangular system with a CTA barrier per level.  Fill-reducing orders of
// 2D operators give thousands of levels (about 5,400 per system at 100k
// rows), and at that size the solve vector no longer fits in shared memory,
// so each level costs an L2 round trip and the single CTA falls behind one
// CPU core.  Here every warp of a cooperative grid owns rows in a fixed
// cyclic order over the system's rows sorted by level (the r-th row of that
// order -> warp r mod W) and solves each row on its own as soon as the
// entries it depends on are written --
// the synchronisation-free scheme of Liu, Li, Hou and Vinter ("A
// synchronization-free algorithm for parallel sparse triangular solves",
// Euro-Par 2016), with no per-row flags: each solve vector is reset to a
// reserved NaN bit pattern before use and a value other than that pattern
// is itself the sign that it is final, so a dependency costs one L2 round
// trip.  A row only waits on rows of lower levels, which come earlier in
// every warp's sequence, and the grid is co-resident (cooperative launch), so
// every wait ends; each wait is bounded anyway (time limit and the shared
// abort flag).  Visiting the rows in plain index order instead made a warp's
// shallow rows wait behind its deep ones (2.9x slower at 100k rows).
//
// Per row the arithmetic is the single-CTA kernel's: x_i = b_i (1/T_ii) +
// sum_j (-T_ij/T_ii) x_j, the off-diagonal values stored pre-divided by the
// diagonal, lanes summing the row's entries in stored order with a stride of
// 32 and a butterfly at the end (fixed order: runs are reproducible).
// Between the solves: grid barriers for ||A^{-1} x||^2 and ||x||^2 (the
// score and the gradient coefficients), for the Adam step's partials, and
// before the next iteration reads x.
#include <math.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "pa_device.cuh"
#include "pa_internal.h"

namespace pa {

namespace {

constexpr int kLgThreads = 256;
constexpr int kLgWarps = kLgThreads / 32;
// "not written yet": a signalling-NaN payload that no arithmetic produces
constexpr unsigned long long kUnset = 0x7FF4DEADBEEFCAFEull;

struct LgShared {
  double scratch[2 * kLgThreads];
  double ca, cb, c, inv, q_keep, L_min, L_last;
  int brk, improved, t_min, iters_run, status, ok;
};

__device__ __forceinline__ void st_relaxed(double* a, double v) {
  asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(a), "d"(v) : "memory");
}

// The value of a[0] once it is no longer kUnset; ok becomes 0 when the wait
// gives up (time limit or another CTA's abort), after which it returns 0.
__device__ __forceinline__ double wait_value(const double* a, RunState* st, long long timeout_ns,
                                             int& ok) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(a) : "memory");
  if (v != kUnset || !ok) return __longlong_as_double(v);
  const long long t0 = globaltimer_ns();
  for (int spins = 1;; ++spins) {
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(a) : "memory");
    if (v != kUnset) return __longlong_as_double(v);
    if ((spins & 31) == 0) {
      if (ld_relaxed_u32(&st->abort) != 0u) break;
      if (globaltimer_ns() - t0 > timeout_ns) {
        atomicExch(&st->abort, 1u);
        break;
      }
    }
  }
  ok = 0;
  return 0.0;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const double* a) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(a) : "memory");
  return v;
}

// One triangular system, every row owned by this warp, in level order
// (T.order: rows sorted by the level of the system, so a warp's rows never
// wait behind a deeper row of its own).  Row i's right-hand side is
// bsrc[bperm[i]] of a finished vector (b_wait false) or bsrc[i] of the
// previous solve's vector, which may still be unset (b_wait true); it is
// loaded when the row starts.  out receives the solution; on_row(i, b_i,
// y_i) runs in lane 0 after row i is written.  Each lane takes the row's
// entries k0 + lane, k0 + lane + 32, ... four at a time: their loads are
// issued together, then only values still unset are waited for.
template <int UL, typename F>
__device__ __forceinline__ bool solve_rows(const TriRows& T, int n, int gw, int W, double* out,
                                           const double* bsrc, const int32_t* bperm, bool b_wait,
                                           F on_row, RunState* st, long long timeout_ns) {
  const int lane = threadIdx.x & 31;
  int ok = ld_relaxed_u32(&st->abort) == 0u;
  for (int r = gw; r < n && ok; r += W) {
    const int i = __ldg(T.order + r);
    unsigned long long bv;
    if (b_wait) bv = ld_relaxed_u64(bsrc + i);
    else bv = __double_as_longlong(bsrc[bperm ? __ldg(bperm + i) : i]);
    const int k0 = __ldg(T.rp + i), k1 = __ldg(T.rp + i + 1);
    double acc = 0.0;
    for (int kb = k0 + lane; kb < k1; kb += 32 * UL) {
      int c[UL];
      double a[UL];
      unsigned long long v[UL];
#pragma unroll
      for (int u = 0; u < UL; ++u) {
        const int k = kb + 32 * u;
        c[u] = k < k1 ? __ldg(T.ci + k) : -1;
        a[u] = k < k1 ? __ldg(T.va + k) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < UL; ++u) v[u] = c[u] >= 0 ? ld_relaxed_u64(out + c[u]) : 0ull;
#pragma unroll
      for (int u = 0; u < UL; ++u) {
        if (c[u] < 0) continue;
        const double xv = v[u] != kUnset ? __longlong_as_double(v[u])
                                         : wait_value(out + c[u], st, timeout_ns, ok);
        acc = fma(a[u], xv, acc);
      }
    }
    ok = __all_sync(0xffffffffu, ok);
    acc = warp_sum(acc);
    const double bi = (b_wait && bv == kUnset) ? wait_value(bsrc + i, st, timeout_ns, ok)
                                               : __longlong_as_double(bv);
    ok = __all_sync(0xffffffffu, ok);
    if (!ok) break;
    const double yi = fma(bi, __ldg(T.dinv + i), acc);
    if (lane == 0) {
      st_relaxed(out + i, yi);
      on_row(i, bi, yi);
    }
  }
  return ok;
}

__device__ __forceinline__ void fill_unset(double* a, int n) {
  const double u = __longlong_as_double(kUnset);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = u;
}

template <int UL, int MINB>
__global__ void __launch_bounds__(kLgThreads, MINB) k_lu_grid(const LuGridParams p) {
  __shared__ LgShared sh;
  const int n = p.n, tid = threadIdx.x, lane = tid & 31;
  const unsigned G = gridDim.x;
  const int W = G * kLgWarps, gw = blockIdx.x * kLgWarps + (tid >> 5);
  const int b = blockIdx.x;
  RunState* st = p.st;
  double* part = p.partials;
  unsigned target = 0;
  int site = 0;
  if (tid == 0) {
    sh.L_min = INFINITY;
    sh.L_last = NAN;
    sh.t_min = 0;
    sh.iters_run = 0;
    sh.status = PA_OK;
  }
  for (int s = 0; s < 4; ++s) fill_unset(p.y[s], n);
  bool alive = grid_barrier(st, target, G, p.timeout_ns, false, site++, sh.ok);
  const int32_t* perm = p.p;
  // r = A^{-1} v: L t = P v, U u = t; lane 0 sums ||v||^2 and ||u||^2
  auto apply_inv = [&](const double* vsrc, double& q2, double& rr) -> bool {
    if (!solve_rows<UL>(p.sys[0], n, gw, W, p.y[0], vsrc, perm, false,
                    [&](int, double bi, double) { q2 = fma(bi, bi, q2); }, st, p.timeout_ns))
      return false;
    return solve_rows<UL>(p.sys[1], n, gw, W, p.y[1], p.y[0], nullptr, true,
                      [&](int, double, double yi) { rr = fma(yi, yi, rr); }, st, p.timeout_ns);
  };
  double* x = p.x;
  for (int t = 1; alive; ++t) {
    // ---- r = A^{-1} x, ||r||^2, ||x||^2 (Algorithm 2's first solves)
    {
      double v[2] = {0.0, 0.0};  // ||r||^2, ||x||^2
      apply_inv(x, v[1], v[0]);
      block_sum_to0<2>(v, sh.scratch);
      if (tid == 0) {
        part[b * 4 + 0] = v[0];
        part[b * 4 + 1] = v[1];
      }
    }
    if (!(alive = grid_barrier(st, target, G, p.timeout_ns, false, site++, sh.ok))) break;
    if (tid < 32) {
      const double rr = ordered_sum(part, G, 4, 0), q2 = ordered_sum(part, G, 4, 1);
      if (tid == 0) {
        int brk = 0, improved = 0;
        if (!isfinite(rr) || !isfinite(q2) || rr == 0.0) {
          sh.status = PA_ERR_NONFINITE;
          brk = 1;
        } else {
          if (t > 1) {  // score x_{t-1}: L = log||x|| - log||A^{-1} x||
            const double L = log(sqrt(q2)) - log(sqrt(rr));
            sh.L_last = L;
            if (p.L_trace && b == 0) p.L_trace[t - 2] = L;
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
    }
    __syncthreads();
    if (sh.improved)
      for (int i = b * kLgThreads + tid; i < n; i += G * kLgThreads) p.xmin[i] = x[i];
    if (sh.brk) break;

    // ---- s = A^{-T} r: U^T a = u, L^T c = a, s = P^T c (into w)
    if (!solve_rows<UL>(p.sys[2], n, gw, W, p.y[2], p.y[1], nullptr, true,
                    [](int, double, double) {}, st, p.timeout_ns) ||
        !solve_rows<UL>(p.sys[3], n, gw, W, p.y[3], p.y[2], nullptr, true,
                    [&](int i, double, double yi) { p.w[perm ? perm[i] : i] = yi; }, st,
                    p.timeout_ns))
      ;  // a wait gave up: the barrier below sees the abort flag
    if (!(alive = grid_barrier(st, target, G, p.timeout_ns, false, site++, sh.ok))) break;

    // ---- gradient x/||x||^2 - s/||r||^2, Adam, partials x.dx and dx.dx;
    // the solve vectors are reset for the next iteration on the way
    {
      const double ca = sh.ca, cb = sh.cb;
      const double2 bc = p.bias[p.t0 + t - 1];
      const double b1 = p.beta1, b2 = p.beta2;
      const double w2 = (1.0 - b2) / ((1.0 - b1) * (1.0 - b1));
      const double u = __longlong_as_double(kUnset);
      double v[2] = {0.0, 0.0};
      for (int j = b * kLgThreads + tid; j < n; j += G * kLgThreads) {
        const double xj = x[j];
        const double g = fma(ca, xj, cb * p.w[j]);
        const double mj = fma(b1, p.m[j], g);
        const double vj = fma(b2, p.v[j], w2 * (g * g));
        p.m[j] = mj;
        p.v[j] = vj;
        const double d = adam_quotient(bc.x * mj, vj, bc.y);
        p.dx[j] = d;
        v[0] = fma(xj, d, v[0]);
        v[1] = fma(d, d, v[1]);
        p.y[0][j] = u;
        p.y[1][j] = u;
        p.y[2][j] = u;
        p.y[3][j] = u;
      }
      block_sum_to0<2>(v, sh.scratch);
      if (tid == 0) {
        part[b * 4 + 2] = v[0];
        part[b * 4 + 3] = v[1];
      }
    }
    if (!(alive = grid_barrier(st, target, G, p.timeout_ns, false, site++, sh.ok))) break;
    if (tid < 32) {
      const double p1 = ordered_sum(part, G, 4, 2), p2 = ordered_sum(part, G, 4, 3);
      if (tid == 0) {
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
    }
    __syncthreads();
    if (sh.brk) break;

    // ---- x_t = ((1 + c) x - dx) / ||.||: projection, update, normalisation
    {
      const double a1c = 1.0 + sh.c, inv = sh.inv;
      double* tr = (p.x_trace && t <= p.n_trace) ? p.x_trace + (size_t)(t - 1) * n : nullptr;
      for (int j = b * kLgThreads + tid; j < n; j += G * kLgThreads) {
        const double xn = fma(a1c, x[j], -p.dx[j]) * inv;
        x[j] = xn;
        if (tr) tr[j] = xn;
      }
      if (tid == 0) sh.iters_run = t;
    }
    if (!(alive = grid_barrier(st, target, G, p.timeout_ns, false, site++, sh.ok))) break;
  }

  // ---- sigma_max(A^{-1}) = ||A^{-1} x_min|| / ||x_min||
  double sig = NAN;
  if (alive) {
    fill_unset(p.y[0], n);
    fill_unset(p.y[1], n);
    alive = grid_barrier(st, target, G, p.timeout_ns, false, site++, sh.ok);
  }
  if (alive) {
    double v[2] = {0.0, 0.0};
    apply_inv(p.xmin, v[1], v[0]);
    block_sum_to0<2>(v, sh.scratch);
    if (tid == 0) {
      part[b * 4 + 0] = v[0];
      part[b * 4 + 1] = v[1];
    }
    alive = grid_barrier(st, target, G, p.timeout_ns, false, site++, sh.ok);
    if (alive && b == 0 && tid < 32) {
      const double rr = ordered_sum(part, G, 4, 0), q2 = ordered_sum(part, G, 4, 1);
      sig = sqrt(rr) / sqrt(q2);
    }
  }
  if (b == 0 && tid == 0) {
    if (!alive || ld_relaxed_u32(&st->abort) != 0u) sh.status = PA_ERR_TIMEOUT;
    st->status = sh.status;
    st->t_min = sh.t_min;
    st->L_min = sh.L_min;
    st->L_last = sh.L_last;
    st->iters_run = sh.iters_run;
    st->sigma = sig;
  }
  (void)lane;
}

}  // namespace

void tri_rows_host(int32_t n, const int32_t* rp, const int32_t* ci, const double* va, bool lower,
                   TriRowsHost* out) {
  out->rp.assign((size_t)n + 1, 0);
  out->ci.clear();
  out->va.clear();
  out->dinv.assign((size_t)n, 0.0);
  // levels (a row's level is one more than the highest level it depends on)
  // and the rows sorted by level, stably
  std::vector<int32_t> level((size_t)n, 0);
  int32_t nlev = 0;
  for (int32_t s = 0; s < n; ++s) {
    const int32_t i = lower ? s : n - 1 - s;
    int32_t lv = 0;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
      if (ci[k] != i) lv = std::max(lv, level[ci[k]] + 1);
    level[i] = lv;
    nlev = std::max(nlev, lv + 1);
  }
  std::vector<int32_t> start((size_t)nlev + 1, 0);
  for (int32_t i = 0; i < n; ++i) ++start[level[i] + 1];
  for (int32_t l = 0; l < nlev; ++l) start[l + 1] += start[l];
  out->order.assign((size_t)n, 0);
  for (int32_t s = 0; s < n; ++s) {
    const int32_t i = lower ? s : n - 1 - s;
    out->order[start[level[i]]++] = i;
  }
  for (int32_t i = 0; i < n; ++i) {
    double d = 0.0;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
      if (ci[k] == i) d = va[k];
    out->dinv[i] = 1.0 / d;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
      if (ci[k] != i) {
        out->ci.push_back(ci[k]);
        out->va.push_back(-va[k] / d);
      }
    out->rp[i + 1] = (int32_t)out->ci.size();
  }
}

// Eight loads in flight per lane, two CTAs of 256 threads per SM (96
// registers).  Measured at 100k rows: 4 per lane (four CTAs per SM) 67 ms per
// iteration, 8 per lane 64 ms, 16 per lane 68 ms; a smaller grid, backing off
// between polls, or re-polling all of a lane's pending values together did
// not help either -- the time is the chain of dependent levels.
static void* lu_grid_fn() { return (void*)k_lu_grid<8, 2>; }

int lu_grid_max_blocks() {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, lu_grid_fn(), kLgThreads, 0) != cudaSuccess)
    return -1;
  return per * sms;
}

cudaError_t launch_lu_grid(const LuGridParams& p, int G, cudaStream_t s, int64_t* launches) {
  void* args[] = {(void*)&p};
  ++*launches;
  return cudaLaunchCooperativeKernel(lu_grid_fn(), dim3(G), dim3(kLgThreads), args, 0, s);
}

}  // namespace pa
