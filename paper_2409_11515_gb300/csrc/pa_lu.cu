// pa_lu.cu -- sigma_min through ||A^{-1}||_2 with a given LU factorisation:
// the paper's Algorithm 2 ("Compute Gradient for A^{-1}") inside Algorithm 1.
//
// With P A Q = L U, A^{-1} = Q U^{-1} L^{-1} P and A^{-T} = P^T L^{-T} U^{-T} Q^T.
// Per iteration, for B = A^{-1}:
//   r = B x        : L t = P x, U u = t (r = Q u, so ||r|| = ||u||)
//   score          : L(x_{t-1}) = log||x|| - log||r|| against L_min
//   s = B^T r      : U^T a = u, L^T c = a, s = P^T c
//   grad           : x / ||x||^2 - s / ||r||^2   (Algorithm 2)
//   Adam, tangent projection, update, normalisation as in Algorithm 1.
// sigma_min(A) = 1 / sigma_max(B) = ||x_min|| / ||B x_min||.
//
// The triangular solves are level-scheduled.  Sparse LU factors of 2D
// operators in fill-reducing orders have long, thin level sets: hundreds of
// levels of a few rows, most of them rows of the dense triangles that such
// orders leave at the separators, each depending on the previous row.
// A row-per-warp solve pays a dot product, a butterfly sum and a division per
// level; on GB300, where every dependent FP64 instruction costs tens of
// cycles, that chain is the whole cost.  Here each row's entries are split
// by the level of their column and applied, as x_i += sum va_ij x_j, in the
// step right after that column level is final: a step is mostly one FMA per
// thread (the column-oriented update of a dense triangle falls out of this),
// followed by one __syncthreads.  The values are stored pre-divided by the
// diagonal and x starts as b / diag, so a row is final after its last
// segment.  One CTA runs the whole iteration; the solve vector lives in
// shared memory, and one thread copies each step's records there with bulk
// (TMA) copies several steps ahead, each slot of the staging ring completing
// on its own mbarrier.  The kernel waits on nothing outside its CTA.
#include <math.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <string>
#include <vector>

#include "pa_device.cuh"
#include "pa_internal.h"

namespace pa {

namespace {

constexpr int kAhead = 6;          // steps staged ahead of the one being applied
constexpr int kRing = kAhead + 1;  // staging slots
constexpr int kMinCap = 64;        // smallest slot worth having
constexpr int kApplyThreads = kLuThreads - 32;  // all warps but the last apply steps

// One slot: the step's own record, the record kAhead steps later, then the
// step's items and the values and columns of its longer segments (16-byte
// windows around them).
__host__ __device__ constexpr size_t slot_bytes(int n_items, int n_ent) {
  return 32 + 16 * (size_t)n_items + 12 * (size_t)n_ent;
}

// Lanes per item for a step of n_items items whose longest segment has
// max_len entries: the fewest dependent FP64 operations (FMAs along a lane,
// then the butterfly), counting the rounds when the items outnumber the lanes.
int pick_lanes_log2(int64_t n_items, int max_len) {
  int best = 0;
  int64_t best_cost = LLONG_MAX;
  for (int lg = 0; lg <= 5; ++lg) {
    const int64_t G = 1 << lg;
    const int64_t rounds = (n_items * G + kApplyThreads - 1) / kApplyThreads;
    const int64_t cost = rounds * ((max_len + G - 1) / G + lg);
    if (cost < best_cost) {
      best_cost = cost;
      best = lg;
    }
  }
  return best;
}

}  // namespace

std::string tri_analyse(int32_t n, const int32_t* rp, const int32_t* ci, const double* va,
                        bool lower, TriHost* out) {
  *out = TriHost();
  std::vector<double> diag((size_t)n, 0.0);
  std::vector<int32_t> level((size_t)n, 0);
  for (int32_t i = 0; i < n; ++i) {
    bool have_diag = false;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
      const int32_t j = ci[k];
      if (j < 0 || j >= n) return "column index out of range in row " + std::to_string(i);
      if (j == i) {
        if (have_diag) return "two diagonal entries in row " + std::to_string(i);
        have_diag = true;
        diag[i] = va[k];
      } else if ((lower && j > i) || (!lower && j < i)) {
        return std::string(lower ? "entry above the diagonal" : "entry below the diagonal") +
               " in row " + std::to_string(i);
      }
    }
    if (!have_diag || diag[i] == 0.0 || !std::isfinite(diag[i]))
      return "zero or missing diagonal in row " + std::to_string(i);
  }
  // levels: a forward solve visits rows upwards, a backward solve downwards
  int32_t nlev = n > 0 ? 1 : 0;
  for (int32_t s = 0; s < n; ++s) {
    const int32_t i = lower ? s : n - 1 - s;
    int32_t lv = 0;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
      if (ci[k] != i) lv = std::max(lv, level[ci[k]] + 1);
    level[i] = lv;
    nlev = std::max(nlev, lv + 1);
  }
  out->nproc = std::max(nlev - 1, 0);
  out->dinv.resize((size_t)n);
  for (int32_t i = 0; i < n; ++i) out->dinv[i] = 1.0 / diag[i];
  // every off-diagonal entry, keyed by (step = level of its column, level of
  // its row, row, stored position): a step's items are then contiguous, rows
  // that become final in the step first, each segment in stored order
  struct Key {
    int32_t step, rlev, row, k;
  };
  std::vector<Key> keys;
  keys.reserve((size_t)rp[n]);
  for (int32_t i = 0; i < n; ++i)
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
      if (ci[k] != i) keys.push_back(Key{level[ci[k]], level[i], i, k});
  std::sort(keys.begin(), keys.end(), [](const Key& a, const Key& b) {
    if (a.step != b.step) return a.step < b.step;
    if (a.rlev != b.rlev) return a.rlev > b.rlev;
    if (a.row != b.row) return a.row < b.row;
    return a.k < b.k;
  });
  if (keys.size() > (size_t)INT_MAX - 8) return "factor too large for the LU route";
  out->linfo.assign((size_t)out->nproc, make_int4(0, 0, 0, 0));
  size_t q = 0;
  for (int32_t l = 0; l < out->nproc; ++l) {
    const int32_t i0 = (int32_t)out->items.size(), e0 = (int32_t)out->ci.size();
    int max_len = 0;
    while (q < keys.size() && keys[q].step == l) {
      const int32_t row = keys[q].row;
      size_t r = q;
      while (r < keys.size() && keys[r].step == l && keys[r].row == row) ++r;
      const int len = (int)(r - q);
      if (len == 1) {  // {row, column, value}
        const double v = -va[keys[q].k] / diag[row];
        int2 w;
        memcpy(&w, &v, sizeof(double));
        out->items.push_back(make_int4(row, ci[keys[q].k], w.x, w.y));
      } else {  // {~row, first entry, end entry, 0}
        const int32_t b0 = (int32_t)out->ci.size();
        for (size_t k = q; k < r; ++k) {
          out->ci.push_back(ci[keys[k].k]);
          out->va.push_back(-va[keys[k].k] / diag[row]);
        }
        out->items.push_back(make_int4(~row, b0, (int32_t)out->ci.size(), 0));
      }
      max_len = std::max(max_len, len);
      q = r;
    }
    const int32_t i1 = (int32_t)out->items.size(), e1 = (int32_t)out->ci.size();
    if (i1 > kItemMask) return "factor too large for the LU route";
    const int lg = pick_lanes_log2(i1 - i0, max_len);
    out->linfo[l] = make_int4(i0, i1 | (lg << 27), e0, e1);
    const int win_v = ((e1 + 1) & ~1) - (e0 & ~1);
    const int win_c = ((e1 + 3) & ~3) - (e0 & ~3);
    out->max_items = std::max(out->max_items, i1 - i0);
    out->max_ent = std::max({out->max_ent, win_v, win_c});
  }
  // padding for the 16-byte windows
  const size_t E = out->ci.size();
  out->ci.resize((E + 7) & ~(size_t)3, 0);
  out->va.resize((E + 3) & ~(size_t)1, 0.0);
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

struct LuShared {
  double scratch[2 * kLuThreads];
  double ca, cb;      // g' = (1 - beta1) grad = ca x + cb s
  double c, inv;      // projection coefficient and 1 / ||x'||
  double q_keep;      // ||x||^2 of the current iterate
  double L_min, L_last;
  int brk, improved;
  int t_min, iters_run, status;
  unsigned long long bar[kRing];  // one mbarrier per staging slot
  unsigned phase_bits;            // parity of each slot's next completion
  int stall;                      // a staging wait gave up: skip the rest
};

struct Slot {
  int4* own;
  int4* next;
  int4* items;
  double* va;
  int32_t* ci;
};

__device__ __forceinline__ Slot slot_at(char* ring, int idx, int ni, int ne) {
  char* b = ring + (size_t)idx * slot_bytes(ni, ne);
  return Slot{reinterpret_cast<int4*>(b), reinterpret_cast<int4*>(b + 16),
              reinterpret_cast<int4*>(b + 32), reinterpret_cast<double*>(b + 32 + 16 * (size_t)ni),
              reinterpret_cast<int32_t*>(b + 32 + 16 * (size_t)ni + 8 * (size_t)ne)};
}

// First index of the 16-byte windows of a step's values and columns, and
// whether the step fits a slot.
struct Win {
  int va, ca;
  bool fits;
};

__device__ __forceinline__ Win window(const int4& I, int ni, int ne) {
  Win w;
  w.va = I.z & ~1;
  w.ca = I.z & ~3;
  w.fits = (I.y & kItemMask) - I.x <= ni && ((I.w + 1) & ~1) - w.va <= ne &&
           ((I.w + 3) & ~3) - w.ca <= ne;
  return w;
}

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}
// Arrive once, announcing `bytes` of bulk copies that complete the phase.
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bulk copy (TMA engine) of `bytes` (a multiple of 16, both addresses 16-byte
// aligned) from global to this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

constexpr long long kStageTimeoutNs = 1000000000LL;  // 1 s

// Wait for a slot's copies.  Gives up after kStageTimeoutNs (or at once once
// another thread gave up), sets the CTA's stall flag and returns false.
__device__ __noinline__ bool wait_slot_slow(unsigned long long* bar, unsigned parity, volatile int* stall) {
  const long long t0 = globaltimer_ns();
  for (int spins = 1;; ++spins) {
    if (mbar_test(bar, parity)) return true;
    if ((spins & 7) == 0 && (*stall || globaltimer_ns() - t0 > kStageTimeoutNs)) {
      *stall = 1;
      return false;
    }
  }
}
__device__ __forceinline__ bool wait_slot(unsigned long long* bar, unsigned parity, volatile int* stall) {
  return mbar_test(bar, parity) || wait_slot_slow(bar, parity, stall);
}

// Stage step l (record I) into slot S with barrier bar: the own record by a
// plain store, then the step's items, values and columns and the record of
// step l + kAhead by bulk copies (one thread).
__device__ __forceinline__ void stage(const TriSys& T, int l, const int4& I, const Slot& S, int ni,
                                      int ne, unsigned long long* bar) {
  const Win w = window(I, ni, ne);
  *S.own = make_int4(I.x, I.y | (w.fits ? 1 << 30 : 0), I.z, I.w);
  const bool nx = l + kAhead < T.nproc;
  const unsigned bi = w.fits ? 16u * (unsigned)((I.y & kItemMask) - I.x) : 0u;
  const unsigned bv = w.fits ? 8u * (unsigned)(((I.w + 1) & ~1) - w.va) : 0u;
  const unsigned bc = w.fits ? 4u * (unsigned)(((I.w + 3) & ~3) - w.ca) : 0u;
  mbar_arrive_tx(bar, bi + bv + bc + (nx ? 16u : 0u));
  if (nx) bulk_g2s(S.next, T.linfo + l + kAhead, 16, bar);
  if (bi) bulk_g2s(S.items, T.items + I.x, bi, bar);
  if (bv) bulk_g2s(S.va, T.va + w.va, bv, bar);
  if (bc) bulk_g2s(S.ci, T.ci + w.ca, bc, bar);
}

// One item: add its segment's sum to x[row] (a thread, or lane gl of a
// group of G for a longer segment, whose partial the caller sums).
__device__ __forceinline__ double item_sum(const int4& r, const double* VA, const int32_t* CI, int ov,
                                           int oc, const double* x, int gl, int G, int* row) {
  if (r.x >= 0) {
    *row = r.x;
    return gl == 0 ? fma(__hiloint2double(r.w, r.z), x[r.y], x[r.x]) : 0.0;
  }
  *row = ~r.x;
  double acc = gl == 0 ? x[~r.x] : 0.0;
  for (int e = r.y + gl; e < r.z; e += G) acc = fma(VA[e - ov], x[CI[e - oc]], acc);
  return acc;
}

// Apply one step (apply threads, each with an item or in a group).  ST: the
// step's records are in slot S (else read from global memory).
template <bool ST>
__device__ __forceinline__ void apply_step(const TriSys& T, const int4& I, const Slot& S, double* x) {
  const int4* IT = ST ? S.items : T.items + I.x;
  const double* VA = ST ? S.va : T.va;
  const int32_t* CI = ST ? S.ci : T.ci;
  const int ov = ST ? I.z & ~1 : 0, oc = ST ? I.z & ~3 : 0;
  const int nit = (I.y & kItemMask) - I.x, lg = (I.y >> 27) & 7;
  const int tid = threadIdx.x;
  if (lg == 0) {  // a thread per item
    for (int k = tid; k < nit; k += kApplyThreads) {
      int row;
      const double v = item_sum(IT[k], VA, CI, ov, oc, x, 0, 1, &row);
      x[row] = v;
    }
  } else {  // 2^lg lanes per item, then a butterfly inside the group
    const int G = 1 << lg, gid = tid >> lg, gl = tid & (G - 1), ng = kApplyThreads >> lg;
    for (int k0 = 0; k0 < nit; k0 += ng) {  // the same trip count for all apply warps
      const int k = k0 + gid;
      double acc = 0.0;
      int row = 0;
      if (k < nit) acc = item_sum(IT[k], VA, CI, ov, oc, x, gl, G, &row);
      for (int d = G >> 1; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
      if (k < nit && gl == 0) x[row] = acc;
    }
  }
}

extern __shared__ __align__(16) double lu_dyn[];

// The solve vector and the staging ring: with XS, the vector in dynamic
// shared memory followed by the ring (addresses the compiler can see are
// shared); else the vector in global memory and the ring at the start.
template <bool XS>
__device__ __forceinline__ double* solve_vector(int n, double* y_global) {
  return XS ? lu_dyn : y_global;
}
template <bool XS>
__device__ __forceinline__ char* staging_ring(int n) {
  return XS ? reinterpret_cast<char*>(lu_dyn + n + (n & 1)) : reinterpret_cast<char*>(lu_dyn);
}

// T x = b for x holding b / diag on entry.  One thread of the last warp
// stages steps into the ring kAhead steps ahead (bulk copies completing on
// the slot's mbarrier); the other warps apply the current step, each thread
// that has an item waiting for its slot first.  A thread with no item in a
// step costs a record load and the barrier.
template <bool XS>
__device__ __noinline__ void tri_solve(const TriSys& Tg, int n, double* y_global, int ni, int ne,
                                       LuShared& sh) {
  const TriSys T = Tg;  // in registers
  double* const x = solve_vector<XS>(n, y_global);
  char* const ring = staging_ring<XS>(n);
  const int np = T.nproc, tid = threadIdx.x;
  const bool stager = tid == kApplyThreads;
  unsigned phases = sh.phase_bits;
  if (stager) {
    for (int j = 0; j < kAhead && j < np; ++j)
      stage(T, j, T.linfo[j], slot_at(ring, j, ni, ne), ni, ne, &sh.bar[j]);
  }
  __syncthreads();
  for (int l = 0, cur = 0; l < np; ++l) {
    const Slot S = slot_at(ring, cur, ni, ne);
    const unsigned par = (phases >> cur) & 1u;
    if (tid < kApplyThreads) {
      const int4 I = *S.own;  // stored at least one barrier ago
      const int nit = (I.y & kItemMask) - I.x, lg = (I.y >> 27) & 7;
      const bool fits = (I.y >> 30) & 1;
      if (lg != 0 || tid < nit) {  // a group step needs every apply thread
        const bool ok = !fits || wait_slot(&sh.bar[cur], par, &sh.stall);
        if (ok) {
          if (fits) apply_step<true>(T, I, S, x);
          else apply_step<false>(T, I, S, x);
        }
      }
    } else if (stager && l + kAhead < np) {
      // the slot of step l + kAhead held step l - 1, finished before the last barrier
      const int nxt = cur == 0 ? kRing - 1 : cur - 1;  // (l + kAhead) % kRing
      if (wait_slot(&sh.bar[cur], par, &sh.stall))      // step l's copies carry step l + kAhead's record
        stage(T, l + kAhead, *S.next, slot_at(ring, nxt, ni, ne), ni, ne, &sh.bar[nxt]);
    }
    phases ^= 1u << cur;
    cur = cur == kRing - 1 ? 0 : cur + 1;
    __syncthreads();  // x of step l is final
  }
  if (tid == 0) sh.phase_bits = phases;
  __syncthreads();
}

// y = U^{-1} L^{-1} P x (= Q^T A^{-1} x)
template <bool XS>
__device__ __forceinline__ void apply_inv(const LuParams& p, const double* x, double* y, LuShared& sh) {
  for (int i = threadIdx.x; i < p.n; i += kLuThreads) y[i] = x[p.p ? p.p[i] : i] * p.L.dinv[i];
  tri_solve<XS>(p.L, p.n, p.y, p.slot_items, p.slot_ent, sh);
  for (int i = threadIdx.x; i < p.n; i += kLuThreads) y[i] *= p.U.dinv[i];
  tri_solve<XS>(p.U, p.n, p.y, p.slot_items, p.slot_ent, sh);
}

// One CTA per item: item b runs Algorithm 1 on the inverse of its own matrix
// from its own start vector, independently of the other CTAs.
// XS: every item keeps its solve vector in shared memory (smem_mode 1), so
// the compiler sees shared-memory addresses throughout the solve.
template <bool XS>
__global__ void __launch_bounds__(kLuThreads, 1) k_lu_iter(const LuParams* __restrict__ items) {
  const LuParams& p = items[blockIdx.x];
  __shared__ LuShared sh;
  const int n = p.n, tid = threadIdx.x;
  double* const y = solve_vector<XS>(n, p.y);
  if (tid == 0) {
    sh.L_min = INFINITY;
    sh.L_last = NAN;
    sh.t_min = 0;
    sh.iters_run = 0;
    sh.status = PA_OK;
    sh.phase_bits = 0;
    sh.stall = 0;
    for (int s = 0; s < kRing; ++s) mbar_init(&sh.bar[s]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  double* x = p.x;
  for (int t = 1;; ++t) {
    // ---- r = A^{-1} x (Algorithm 2: solve L U r = x), ||r||^2, ||x||^2
    apply_inv<XS>(p, x, y, sh);
    {
      double v[2] = {0.0, 0.0};
      for (int i = tid; i < n; i += kLuThreads) {
        v[0] = fma(y[i], y[i], v[0]);
        v[1] = fma(x[i], x[i], v[1]);
      }
      block_sum_to0<2>(v, sh.scratch);
      if (tid == 0) {
        const double rr = v[0], q2 = v[1];
        int brk = 0, improved = 0;
        if (sh.stall) {
          sh.status = PA_ERR_TIMEOUT;
          brk = 1;
        } else if (!isfinite(rr) || !isfinite(q2) || rr == 0.0) {
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
    for (int i = tid; i < n; i += kLuThreads) y[i] *= p.Ut.dinv[i];
    tri_solve<XS>(p.Ut, n, p.y, p.slot_items, p.slot_ent, sh);
    for (int i = tid; i < n; i += kLuThreads) y[i] *= p.Lt.dinv[i];
    tri_solve<XS>(p.Lt, n, p.y, p.slot_items, p.slot_ent, sh);
    for (int i = tid; i < n; i += kLuThreads) p.w[p.p ? p.p[i] : i] = y[i];
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
        const double g = fma(ca, xj, cb * p.w[j]);
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
  apply_inv<XS>(p, p.xmin, y, sh);
  double v[2] = {0.0, 0.0};
  for (int i = tid; i < n; i += kLuThreads) {
    v[0] = fma(y[i], y[i], v[0]);
    v[1] = fma(p.xmin[i], p.xmin[i], v[1]);
  }
  block_sum_to0<2>(v, sh.scratch);
  if (tid == 0) {
    RunState* st = p.st;
    if (sh.stall) {  // a wait gave up: let copies still in flight land before the CTA exits
      sh.status = PA_ERR_TIMEOUT;
      const long long t0 = globaltimer_ns();
      while (globaltimer_ns() - t0 < kStageTimeoutNs) __nanosleep(1000000);
    }
    st->status = sh.status;
    st->t_min = sh.t_min;
    st->L_min = sh.L_min;
    st->L_last = sh.L_last;
    st->iters_run = sh.iters_run;
    st->sigma = sqrt(v[0]) / sqrt(v[1]);
  }
}

}  // namespace

size_t lu_layout(LuParams* p) {
  const TriSys* ts[4] = {&p->L, &p->U, &p->Ut, &p->Lt};
  int need_i = kMinCap, need_e = kMinCap;
  for (const TriSys* t : ts) {
    need_i = std::max(need_i, t->max_items);
    need_e = std::max(need_e, t->max_ent);
  }
  need_e = (need_e + 3) & ~3;
  const size_t vec = sizeof(double) * ((size_t)p->n + (p->n & 1));
  size_t avail;
  if (vec + kRing * slot_bytes(kMinCap, kMinCap) <= kLuSmemBudget) {
    p->smem_mode = 1;
    avail = kLuSmemBudget - vec;
  } else {
    p->smem_mode = 0;
    avail = kLuSmemBudget;
  }
  int ni = need_i, ne = need_e;
  const size_t per_slot = avail / kRing;
  if (slot_bytes(ni, ne) > per_slot) {  // shrink both in proportion
    const double f = (double)(per_slot - 32) / (double)(slot_bytes(ni, ne) - 32);
    ni = std::max(kMinCap / 2, (int)(ni * f));
    ne = std::max(kMinCap / 2, (int)(ne * f) & ~3);
    while (slot_bytes(ni, ne) > per_slot) ni -= 1;
  }
  p->slot_items = ni;
  p->slot_ent = ne;
  return (p->smem_mode == 1 ? vec : 0) + kRing * slot_bytes(ni, ne);
}

cudaError_t launch_lu_iter(const LuParams* items_dev, int n_items, size_t smem, bool all_smem,
                           cudaStream_t s, int64_t* launches) {
  auto* k = all_smem ? k_lu_iter<true> : k_lu_iter<false>;
  if (smem > 0) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k<<<n_items, kLuThreads, smem, s>>>(items_dev);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace pa
