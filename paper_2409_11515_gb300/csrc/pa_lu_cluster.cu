// pa_lu_cluster.cu -- the paper's Algorithm 2 (sigma_min through
// ||A^{-1}||_2 with given LU factors) inside Algorithm 1 on one thread-block
// cluster, the solve vector in distributed shared memory.
//
// The single-CTA kernel (pa_lu.cu) walks each triangular system in steps: in
// step l every row adds the products of its entries whose columns sit at
// dependency level l (one item per row and step, values pre-divided by the
// diagonal, x starting as b / diag), and one CTA barrier ends the step.  It
// is fast while the solve vector fits that CTA's shared memory (about
// 20,000 rows).  Past that, the grid kernel (pa_lu_grid.cu) solves rows as
// their dependencies are written, which costs about 3 us per dependent
// level through L2 -- measured the same when the dependencies travel
// through distributed shared memory instead, so the per-row chain, not the
// memory hop, sets that pace.
//
// Here the steps run on a cluster of up to 16 CTAs.  The solve vector is
// spread over their shared memories (element i in CTA i mod C, slot i / C),
// and each CTA applies the items of its own rows: a row's partial sum is
// read and written in the CTA's own shared memory, only column values come
// from the other CTAs (distributed shared memory loads).  Where shared
// memory allows (FIN), each CTA also keeps its rows' final values in a
// second array, reset to a marker before every solve and written once, by a
// row's last item.  A column read waits for the marker to go, so no step
// needs a cluster barrier: each CTA runs its steps, ordered by a barrier of
// its own item warps, as the column values it reads arrive, and one cluster
// barrier closes each solve.  Measured on GB300, a release arrive at a
// per-step cluster barrier cost 0.3 to 0.6 us a step (it waits for the
// staging copies in flight) against 80 ns without memory ordering.  Without
// room for the second array every step ends with a release/acquire cluster
// barrier instead.  Each CTA's records are one stream of per-step blocks
// cut into batches; warp 0 copies the next batches into a ring of
// shared-memory slots with the bulk-copy (TMA) engine and fetches the one
// after into L2, so no load from global memory is left on a step's path.
// Every solve of the chain L t = P x, U u = t, U^T a = u, L^T c = a starts
// from the previous solve's result at the same index (b_i / T_ii), so one
// vector serves the whole chain, transformed in place.  Nothing waits on
// anything but the cluster and CTA barriers, the ring's mbarriers, the
// item warps' step count and the marked values (each wait bounded in time);
// every CTA passes each cluster barrier the same number of times.  The
// reductions are the grid kernel's (fixed orders: runs are reproducible),
// and every row adds its entries in the single-CTA kernel's order (a
// segment's lanes may differ).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <climits>

#include <cooperative_groups.h>

#include "pa_device.cuh"
#include "pa_internal.h"
#include "pa_lu_cluster.h"

namespace pa {

namespace {

constexpr int kLcThreads = 512;
constexpr int kLcWork = kLcThreads - 32;  // item threads (warps 1..)
constexpr int kLcSlots = 4;              // staging slots (batches in flight)
constexpr long long kLcTimeoutNs = 1000000000LL;  // 1 s per staging wait

struct LcShared {
  double scratch[2 * kLcThreads];
  double ca, cb, c, inv, q_keep, L_min, L_last;
  int brk, improved, t_min, iters_run, status;
  int stall;                               // a staging wait gave up
  unsigned done;                           // FIN: steps the item warps have finished (running)
  unsigned long long bar[kLcSlots];        // one mbarrier per staging slot
  int4 meta[kLcSlots];                     // the batch record of each slot
};

// dynamic shared memory: [kLcSlots][cap] staged records, then this CTA's
// vector slots
extern __shared__ int4 lc_dyn[];

__device__ __forceinline__ uint32_t lc_saddr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint32_t lc_map(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}

__device__ __forceinline__ double lc_load(uint32_t ra) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(ra) : "memory");
  return v;
}

// A final value not yet written: a NaN payload that arithmetic on finite
// values (or on its default NaN) never produces.
constexpr long long kLcUnset = 0x7FF4C0DEC0DEC0DELL;

__device__ __forceinline__ double lc_load_relaxed(uint32_t ra) {
  double v;
  asm volatile("ld.relaxed.cluster.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(ra) : "memory");
  return v;
}
__device__ __forceinline__ void lc_store_final(double* p, double v) {
  asm volatile("st.relaxed.cluster.shared::cta.f64 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(p)),
               "d"(v)
               : "memory");
}
constexpr long long kLcPollTimeoutNs = 1000000000LL;  // 1 s
// Wait for a final value (time-bounded: gives up, sets the stall flag and
// returns what it read).
__device__ __noinline__ double lc_poll_slow(uint32_t ra, volatile int* stall) {
  const long long t0 = globaltimer_ns();
  for (int spins = 1;; ++spins) {
    __nanosleep(16);  // a short pause keeps the polls from crowding the writers' stores
    const double v = lc_load_relaxed(ra);
    if (__double_as_longlong(v) != kLcUnset) return v;
    if ((spins & 15) == 0 && (*stall || globaltimer_ns() - t0 > kLcPollTimeoutNs)) {
      *stall = 1;
      return v;
    }
  }
}
// Column value at cluster address ra, in two parts so that several loads can
// be in flight before the first is checked: the load (FIN: from the
// final-value array; else a plain load, ordered by the step barrier), then
// (FIN) the wait for a value not yet written.
template <bool FIN>
__device__ __forceinline__ double lc_col(uint32_t ra) {
  if constexpr (FIN) return lc_load_relaxed(ra);
  else return lc_load(ra);
}
template <bool FIN>
__device__ __forceinline__ double lc_col_ready(double v, uint32_t ra, volatile int* stall) {
  if constexpr (FIN)
    return __double_as_longlong(v) != kLcUnset ? v : lc_poll_slow(ra, stall);
  else
    return v;
}

// Element i of the solve vector (slots start at shared address `base`, the
// same offset in every CTA of the cluster).
__device__ __forceinline__ uint32_t lc_elem(uint32_t base, int i, int lgC) {
  return lc_map(base + 8u * (uint32_t)(i >> lgC), (uint32_t)i & ((1u << lgC) - 1u));
}

__device__ __forceinline__ void lc_sync() { cooperative_groups::this_cluster().sync(); }

__device__ __forceinline__ void lc_mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(lc_saddr(bar)) : "memory");
}
// Arrive once, announcing `bytes` of bulk copies that complete the phase.
__device__ __forceinline__ void lc_arrive_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(lc_saddr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool lc_test(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(lc_saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
// from global memory to this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void lc_copy(void* dst, const void* src, unsigned bytes,
                                        unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          lc_saddr(dst)),
      "l"(src), "r"(bytes), "r"(lc_saddr(bar))
      : "memory");
}

// Wait for the phase of `bar` with the given parity.  Gives up after
// kLcTimeoutNs (at once when another thread of the CTA gave up), sets the
// CTA's stall flag and returns false.
__device__ __noinline__ bool lc_wait_slow(unsigned long long* bar, unsigned parity,
                                          volatile int* stall) {
  const long long t0 = globaltimer_ns();
  for (int spins = 1;; ++spins) {
    if (lc_test(bar, parity)) return true;
    if ((spins & 7) == 0 && (*stall || globaltimer_ns() - t0 > kLcTimeoutNs)) {
      *stall = 1;
      return false;
    }
  }
}
__device__ __forceinline__ bool lc_wait(unsigned long long* bar, unsigned parity, volatile int* stall) {
  return lc_test(bar, parity) || lc_wait_slow(bar, parity, stall);
}

// The staging slots of one CTA and the count of batches staged so far,
// modulo 2 kLcSlots (every thread keeps the same count).
struct LcRing {
  int4* rec;  // [kLcSlots][cap]
  int cap;
  unsigned u;
  unsigned steps;  // steps of the earlier solves (running, wraps)
};

// Thread 0 (FIN): wait until the item warps have finished `target` steps
// (running count).  Gives up after kLcTimeoutNs, sets the stall flag and
// returns false.
__device__ __noinline__ bool lc_wait_done(const unsigned* done, unsigned target,
                                          volatile int* stall) {
  long long t0 = -1;
  for (int spins = 0;; ++spins) {
    unsigned d;
    asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(d) : "r"(lc_saddr(done)) : "memory");
    if ((int)(d - target) >= 0) return true;
    if (*stall) return false;
    if ((spins & 15) == 15) {
      const long long now = globaltimer_ns();
      if (t0 < 0) t0 = now;
      else if (now - t0 > kLcTimeoutNs) {
        *stall = 1;
        return false;
      }
    }
    __nanosleep(32);
  }
}

// Thread 0: batch record bt (the batch's k-th use of the ring, counted
// modulo 2 kLcSlots) into slot k mod kLcSlots: its record first, then its
// first cap records by one bulk copy.  The slot's previous batch is done
// with (its last step ended) and its copy complete (its steps awaited it).
__device__ __forceinline__ void lc_issue(const LcSys& T, const int4& bt, unsigned k, LcRing& rg,
                                         LcShared& sh) {
  const unsigned s = k % kLcSlots;
  const unsigned bytes = 16u * (unsigned)min(bt.w, rg.cap);
  sh.meta[s] = bt;
  lc_arrive_tx(&sh.bar[s], bytes);
  lc_copy(rg.rec + (size_t)s * rg.cap, T.stream + bt.z, bytes, &sh.bar[s]);
}

// Thread 0: the records of batch record bt into L2, ahead of its copy.
__device__ __forceinline__ void lc_prefetch(const LcSys& T, const int4& bt) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(T.stream + bt.z),
               "r"(16u * (unsigned)bt.w)
               : "memory");
}

// A batch as the item threads see it: record p of the batch (a position
// past the staged cap comes from global memory).
struct LcBatch {
  const int4* smem;
  const int4* gmem;
  int staged;
  __device__ __forceinline__ int4 at(int p) const { return p < staged ? smem[p] : __ldg(gmem + p); }
};

// One item of a step for lane gl of G (lane 0 starts from the row's
// partial): the row's new partial (lane 0) or this lane's share of it, the
// row's slot in this CTA, and whether the item is the row's last.  Entries
// sit at block positions [r.y, r.z), the block starting at batch position
// pos; column values come from the array at cluster address base.
template <bool FIN>
__device__ __forceinline__ double lc_item(const int4& r, const LcBatch& B, int pos,
                                          const double* vec, uint32_t base, int lgC, int gl, int G,
                                          int* slot, bool* last, volatile int* stall) {
  if (r.x >= 0) {
    const int row = r.x & kItemMask;
    *slot = row >> lgC;
    *last = (r.x & kLcLast) != 0;
    if (gl != 0) return 0.0;
    const double xr = vec[row >> lgC];
    const uint32_t ra = lc_elem(base, r.y, lgC);
    const double xc = lc_col_ready<FIN>(lc_col<FIN>(ra), ra, stall);
    return fma(__hiloint2double(r.w, r.z), xc, xr);
  }
  *slot = (~r.x) >> lgC;
  *last = r.w != 0;
  double acc = gl == 0 ? vec[(~r.x) >> lgC] : 0.0;
  int e = r.y + gl;
  // four entries at a time: their loads in flight together, the sum in
  // entry order
  for (; e + 3 * G < r.z; e += 4 * G) {
    int4 q[4];
    uint32_t ra[4];
    double c[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k] = B.at(pos + e + k * G);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      ra[k] = lc_elem(base, q[k].x, lgC);
      c[k] = lc_col<FIN>(ra[k]);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
      acc = fma(__hiloint2double(q[k].w, q[k].z), lc_col_ready<FIN>(c[k], ra[k], stall), acc);
  }
  for (; e < r.z; e += G) {
    const int4 q = B.at(pos + e);
    const uint32_t ra = lc_elem(base, q.x, lgC);
    acc = fma(__hiloint2double(q.w, q.z), lc_col_ready<FIN>(lc_col<FIN>(ra), ra, stall), acc);
  }
  return acc;
}

// T x = b for x holding b / diag on entry (vec: this CTA's partial sums,
// fin its final values (FIN), base the shared address column values are read
// from): the steps, each CTA applying its own rows' items.  Warp 0 stages:
// thread 0 refills the slot of a batch whose steps are done.  Warps 1..
// apply the items.  FIN: the item warps end each step with their own CTA
// barrier and publish the count of finished steps, which thread 0 waits on.
// Otherwise every step ends with the cluster barrier: warp 0 arrives without
// memory ordering (it writes nothing the other CTAs read) and refills while
// the barrier completes; the item warps arrive with release semantics (their
// stores of the step's rows); every thread's wait acquires.
template <bool FIN>
__device__ void lc_steps(const LcSys& T, double* vec, double* fin, uint32_t base, int lgC,
                         LcRing& rg, LcShared& sh) {
  const int np = T.nproc;
  if (np == 0) return;
  const int tid = threadIdx.x;
  const int b0 = __ldg(T.bbase + blockIdx.x), nb = __ldg(T.bbase + blockIdx.x + 1) - b0;
  const int4* BT = T.batch + b0;
  bool ok = true;  // every staging wait of this thread succeeded
  if (tid < 32) {  // warp 0: staging
    // thread 0: batches issued, and the records of the next two batches
    // (loaded a refill ahead of their use, so no refill waits for a load)
    int issued = 0;
    int4 next = make_int4(0, 0, 0, 0), next2 = next;
    if (tid == 0) {
      for (; issued < min(kLcSlots, nb); ++issued) lc_issue(T, __ldg(BT + issued), rg.u + issued, rg, sh);
      if (issued < nb) {
        next = __ldg(BT + issued);
        lc_prefetch(T, next);
      }
      if (issued + 1 < nb) next2 = __ldg(BT + issued + 1);
    }
    // refill the slot of the oldest batch once its steps are done
    auto refill = [&](unsigned k) {
      lc_issue(T, next, k, rg, sh);
      ++issued;
      next = next2;
      if (issued < nb) lc_prefetch(T, next);  // into L2 while the slots are busy
      if (issued + 1 < nb) next2 = __ldg(BT + issued + 1);
    };
    if constexpr (FIN) {
      // the item warps report their finished steps in sh.done
      if (tid == 0)
        while (ok && issued < nb) {
          const unsigned k = rg.u + (unsigned)issued, s = k % kLcSlots;
          ok = lc_wait_done(&sh.done, rg.steps + (unsigned)sh.meta[s].y, &sh.stall) &&
               lc_wait(&sh.bar[s], (k / kLcSlots - 1) & 1, &sh.stall);
          if (ok) refill(k);
        }
    } else {
      for (int l = 0; l < np; ++l) {
        asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
        // steps before l are done: refill the slots whose batches ended
        if (tid == 0)
          while (ok && issued < nb) {
            const unsigned k = rg.u + (unsigned)issued, s = k % kLcSlots;
            if (sh.meta[s].y > l) break;
            if (!(ok = lc_wait(&sh.bar[s], (k / kLcSlots - 1) & 1, &sh.stall))) break;
            refill(k);
          }
        asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
      }
    }
    // thread 0: the last batches' copies have landed before the slots are
    // reused or the kernel ends
    if (tid == 0)
      for (int i = max(0, nb - kLcSlots); i < nb; ++i) {
        const unsigned k = rg.u + (unsigned)i;
        if (!lc_wait(&sh.bar[k % kLcSlots], (k / kLcSlots) & 1, &sh.stall)) break;
      }
  } else {  // warps 1..: the items
    const int wt = tid - 32;
    int bi = -1, end = 0, pos = 0;  // current batch, its end step, this step's block in it
    LcBatch B{nullptr, nullptr, 0};
    for (int l = 0; l < np; ++l) {
      if (l == end) {  // the next batch: wait for its copy
        ++bi;
        const unsigned k = rg.u + (unsigned)bi, s = k % kLcSlots;
        ok = ok && bi < nb && lc_wait(&sh.bar[s], (k / kLcSlots) & 1, &sh.stall);
        if (ok) {
          const int4 bt = sh.meta[s];
          end = bt.y;
          B = LcBatch{rg.rec + (size_t)s * rg.cap, T.stream + bt.z, min(bt.w, rg.cap)};
          pos = 0;
        }
      }
      if (ok) {
        const int4 h = B.at(pos);
        const int cnt = h.x & kItemMask, lg = (h.x >> 27) & 7;
        if (lg == 0) {  // a thread per item
          for (int j = wt; j < cnt; j += kLcWork) {
            int slot;
            bool last;
            const double v = lc_item<FIN>(B.at(pos + 1 + j), B, pos, vec, base, lgC, 0, 1, &slot,
                                          &last, &sh.stall);
            vec[slot] = v;
            if (FIN && last) lc_store_final(fin + slot, v);
          }
        } else {  // 2^lg lanes per item, then a butterfly inside the group
          const int G = 1 << lg, gid = wt >> lg, gl = wt & (G - 1), ng = kLcWork >> lg;
          for (int j0 = 0; j0 < cnt; j0 += ng) {  // the same trip count for every thread
            const int j = j0 + gid;
            double acc = 0.0;
            int slot = -1;
            bool last = false;
            if (j < cnt)
              acc = lc_item<FIN>(B.at(pos + 1 + j), B, pos, vec, base, lgC, gl, G, &slot, &last,
                                 &sh.stall);
            for (int d = G >> 1; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
            if (slot >= 0 && gl == 0) {
              vec[slot] = acc;
              if (FIN && last) lc_store_final(fin + slot, acc);
            }
          }
        }
        pos += 1 + cnt + h.y;
      }
      if constexpr (FIN) {
        // partial sums stay in this CTA, ordered by the item warps' own
        // barrier; readers of final values wait for them, so the CTAs need
        // no common barrier per step and each runs as its inputs arrive
        asm volatile("bar.sync 1, %0;" ::"r"(kLcWork) : "memory");
        if (tid == 32)  // the step's reads of its slot are done (release)
          asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(lc_saddr(&sh.done)),
                       "r"(rg.steps + (unsigned)l + 1u)
                       : "memory");
      } else {
        // the step's rows are written before the next step reads them
        asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
        asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
      }
    }
  }
  // FIN: every CTA has finished reading this solve's final values before any
  // CTA resets them for the next one (the non-aligned form: thread 0 may
  // come from its refill loop after the rest of its warp)
  if constexpr (FIN) {
    asm volatile("barrier.cluster.arrive;" ::: "memory");
    asm volatile("barrier.cluster.wait;" ::: "memory");
  }
  rg.u = (rg.u + (unsigned)nb) % (2 * kLcSlots);
  rg.steps += (unsigned)np;
}

// Bytes of dynamic shared memory below the vector slots.
__host__ __device__ constexpr size_t lc_ring_bytes(int cap) {
  return 16 * (size_t)kLcSlots * (size_t)cap;
}

template <bool FIN>
__global__ void __launch_bounds__(kLcThreads, 1) k_lu_cluster(const LuClusterParams P, int R,
                                                              int lgC, int cap) {
  __shared__ LcShared sh;
  const LuGridParams& p = P.g;
  const int n = p.n, tid = threadIdx.x;
  const unsigned C = gridDim.x;
  const int b = blockIdx.x;
  RunState* st = p.st;
  double* part = p.partials;
  LcRing rg;
  rg.rec = lc_dyn;
  rg.cap = cap;
  rg.u = 0;
  rg.steps = 0;
  // this CTA's partial sums, and (FIN) its rows' final values; a solve's
  // result is in res
  double* const lc_vec = reinterpret_cast<double*>(rg.rec + (size_t)kLcSlots * cap);
  double* const fin = FIN ? lc_vec + R : lc_vec;
  double* const res = fin;
  const uint32_t V = lc_saddr(fin);  // where the steps read column values
  const int32_t* perm = p.p;
  if (tid == 0) {
    sh.L_min = INFINITY;
    sh.L_last = NAN;
    sh.t_min = 0;
    sh.iters_run = 0;
    sh.status = PA_OK;
    sh.stall = 0;
    sh.done = 0;
    for (int k = 0; k < kLcSlots; ++k) lc_mbar_init(&sh.bar[k]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  // every CTA has started (its shared memory exists) before any remote access
  lc_sync();
  // this CTA's slots: slot s holds element i = s C + b of the vector
  auto own = [&](int s) { return s * (int)C + b; };
  // r = A^{-1} v: L t = P v, U u = t in place; ||v||^2 and ||u||^2 per thread
  // slot s of a solve's start: b_i / T_ii, and (FIN) its final value when
  // row i has no items, else the mark of a value not yet written
  auto start = [&](const LcSys& T, int s, int i, double bi) {
    const double y = bi * __ldg(T.dinv + i);
    lc_vec[s] = y;
    if (FIN) fin[s] = __ldg(T.fin0 + i) ? y : __longlong_as_double(kLcUnset);
  };
  auto apply_inv = [&](const double* vsrc, double& q2, double& rr) {
    for (int s = tid; s < R; s += kLcThreads) {
      const int i = own(s);
      if (i < n) {
        const double bi = vsrc[perm ? __ldg(perm + i) : i];
        q2 = fma(bi, bi, q2);
        start(P.sys[0], s, i, bi);
      }
    }
    lc_sync();
    lc_steps<FIN>(P.sys[0], lc_vec, fin, V, lgC, rg, sh);
    for (int s = tid; s < R; s += kLcThreads) {
      const int i = own(s);
      if (i < n) start(P.sys[1], s, i, res[s]);
    }
    lc_sync();
    lc_steps<FIN>(P.sys[1], lc_vec, fin, V, lgC, rg, sh);
    for (int s = tid; s < R; s += kLcThreads) {
      const int i = own(s);
      if (i < n) rr = fma(res[s], res[s], rr);
    }
  };
  double* x = p.x;
  for (int t = 1;; ++t) {
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
    lc_sync();
    if (tid < 32) {
      const double rr = ordered_sum(part, C, 4, 0), q2 = ordered_sum(part, C, 4, 1);
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
      for (int i = b * kLcThreads + tid; i < n; i += (int)C * kLcThreads) p.xmin[i] = x[i];
    if (sh.brk) break;  // the same decision in every CTA (the same sums)

    // ---- s = A^{-T} r: U^T a = u, L^T c = a in place, s = P^T c (into w)
    for (int s = tid; s < R; s += kLcThreads) {
      const int i = own(s);
      if (i < n) start(P.sys[2], s, i, res[s]);
    }
    lc_sync();
    lc_steps<FIN>(P.sys[2], lc_vec, fin, V, lgC, rg, sh);
    for (int s = tid; s < R; s += kLcThreads) {
      const int i = own(s);
      if (i < n) start(P.sys[3], s, i, res[s]);
    }
    lc_sync();
    lc_steps<FIN>(P.sys[3], lc_vec, fin, V, lgC, rg, sh);
    for (int s = tid; s < R; s += kLcThreads) {
      const int i = own(s);
      if (i < n) p.w[perm ? __ldg(perm + i) : i] = res[s];
    }
    lc_sync();  // w is complete

    // ---- gradient x/||x||^2 - s/||r||^2, Adam, partials x.dx and dx.dx
    {
      const double ca = sh.ca, cb = sh.cb;
      const double2 bc = p.bias[p.t0 + t - 1];
      const double b1 = p.beta1, b2 = p.beta2;
      const double w2 = (1.0 - b2) / ((1.0 - b1) * (1.0 - b1));
      double v[2] = {0.0, 0.0};
      for (int j = b * kLcThreads + tid; j < n; j += (int)C * kLcThreads) {
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
        part[b * 4 + 2] = v[0];
        part[b * 4 + 3] = v[1];
      }
    }
    lc_sync();
    if (tid < 32) {
      const double p1 = ordered_sum(part, C, 4, 2), p2 = ordered_sum(part, C, 4, 3);
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
      for (int j = b * kLcThreads + tid; j < n; j += (int)C * kLcThreads) {
        const double xn = fma(a1c, x[j], -p.dx[j]) * inv;
        x[j] = xn;
        if (tr) tr[j] = xn;
      }
      if (tid == 0) sh.iters_run = t;
    }
    lc_sync();  // x is complete before the next iteration's first solve reads it
  }

  // ---- sigma_max(A^{-1}) = ||A^{-1} x_min|| / ||x_min||; every CTA leaves
  // the loop at the same point
  double sig = NAN;
  lc_sync();  // x_min is complete
  {
    double v[2] = {0.0, 0.0};
    apply_inv(p.xmin, v[1], v[0]);
    block_sum_to0<2>(v, sh.scratch);
    if (tid == 0) {
      part[b * 4 + 0] = v[0];
      part[b * 4 + 1] = v[1];
    }
  }
  lc_sync();
  if (b == 0 && tid < 32) {
    const double rr = ordered_sum(part, C, 4, 0), q2 = ordered_sum(part, C, 4, 1);
    sig = sqrt(rr) / sqrt(q2);
  }
  if (b == 0 && tid == 0) {
    st->status = sh.status;
    st->t_min = sh.t_min;
    st->L_min = sh.L_min;
    st->L_last = sh.L_last;
    st->iters_run = sh.iters_run;
    st->sigma = sig;
  }
  // no CTA leaves while another may still read its shared memory
  lc_sync();
  if (tid == 0 && sh.stall) st->status = PA_ERR_TIMEOUT;  // after CTA 0's write above
}

size_t lc_smem(int R, int cap, int fin) {
  return lc_ring_bytes(cap) + sizeof(double) * (size_t)R * (fin ? 2 : 1);
}

void* lc_kernel(int fin) { return fin ? (void*)k_lu_cluster<true> : (void*)k_lu_cluster<false>; }

// Lanes per item (log2) for cnt items of one CTA whose longest segment has
// max_len entries: the fewest rounds of (entries per lane + butterfly).
int lc_lanes_log2(int64_t cnt, int max_len) {
  int best = 0;
  int64_t best_cost = INT64_MAX;
  for (int lg = 0; lg <= 5; ++lg) {
    const int64_t G = 1 << lg;
    const int64_t rounds = (cnt * G + kLcWork - 1) / kLcWork;
    const int64_t cost = rounds * ((max_len + G - 1) / G + lg);
    if (cost < best_cost) {
      best_cost = cost;
      best = lg;
    }
  }
  return best;
}

}  // namespace

void lc_build(const TriHost& t, int lgC, int cap, LcHost* out) {
  const int C = 1 << lgC, np = t.nproc;
  out->nproc = np;
  out->stream.clear();
  out->stream.reserve(t.items.size() + (size_t)C * (size_t)np);
  out->batch.clear();
  out->bbase.assign((size_t)C + 1, 0);
  // each CTA's items of each step, in the step form's order, and each row's
  // last step
  const int32_t n = (int32_t)t.dinv.size();
  std::vector<std::vector<int32_t>> own((size_t)C * (size_t)np);
  std::vector<int32_t> last((size_t)n, -1);
  for (int l = 0; l < np; ++l) {
    const int4 I = t.linfo[l];
    for (int32_t i = I.x; i < (I.y & kItemMask); ++i) {
      const int4 r = t.items[i];
      const int32_t row = r.x >= 0 ? r.x : ~r.x;
      own[(size_t)(row & (C - 1)) * np + l].push_back(i);
      last[(size_t)row] = l;
    }
  }
  out->fin0.assign((size_t)n, 0);
  for (int32_t i = 0; i < n; ++i) out->fin0[(size_t)i] = last[(size_t)i] < 0 ? 1 : 0;
  for (int b = 0; b < C; ++b) {
    out->bbase[(size_t)b] = (int32_t)out->batch.size();
    int4 bt = make_int4(0, 0, (int32_t)out->stream.size(), 0);  // the open batch
    for (int l = 0; l < np; ++l) {
      const std::vector<int32_t>& its = own[(size_t)b * np + l];
      int ne = 0, max_len = 0;
      for (int32_t i : its) {
        const int4 r = t.items[i];
        const int len = r.x >= 0 ? 1 : r.z - r.y;
        if (r.x < 0) ne += len;
        max_len = std::max(max_len, len);
      }
      const int cnt = (int)its.size(), len = 1 + cnt + ne;
      if (bt.y > bt.x && bt.w + len > cap) {  // close the batch before this block
        out->batch.push_back(bt);
        bt = make_int4(l, l, (int32_t)out->stream.size(), 0);
      }
      // the block: header, items, entries (positions relative to the header)
      out->stream.push_back(make_int4(cnt | (lc_lanes_log2(cnt, max_len) << 27), ne, 0, 0));
      int e_pos = 1 + cnt;
      for (int32_t i : its) {
        const int4 r = t.items[i];
        const bool fin = last[(size_t)(r.x >= 0 ? r.x : ~r.x)] == l;  // the row's last item
        if (r.x >= 0) {
          out->stream.push_back(make_int4(r.x | (fin ? kLcLast : 0), r.y, r.z, r.w));
        } else {
          out->stream.push_back(make_int4(r.x, e_pos, e_pos + (r.z - r.y), fin ? 1 : 0));
          e_pos += r.z - r.y;
        }
      }
      for (int32_t i : its) {
        const int4 r = t.items[i];
        if (r.x >= 0) continue;
        for (int32_t e = r.y; e < r.z; ++e) {
          const double v = t.va[e];
          int2 w;
          memcpy(&w, &v, sizeof(double));
          out->stream.push_back(make_int4(t.ci[e], 0, w.x, w.y));
        }
      }
      bt.y = l + 1;
      bt.w += len;
    }
    if (bt.y > bt.x) out->batch.push_back(bt);
  }
  out->bbase[(size_t)C] = (int32_t)out->batch.size();
}

bool lu_cluster_plan(int n, LcPlan* plan) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  for (int fin = 1; fin >= 0; --fin) {  // final values where they fit
    void* fn = lc_kernel(fin);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    for (int lgC = 4; lgC >= 3; --lgC) {  // clusters of 16, else 8
      const int C = 1 << lgC;
      const int R = (n + C - 1) / C;
      for (int cap = 1280; cap >= 160; cap /= 2) {  // the largest staging slots that fit
        const size_t dyn = lc_smem(R, cap, fin);
        if (dyn + sizeof(LcShared) > (size_t)optin) continue;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) !=
            cudaSuccess) {
          cudaGetLastError();
          continue;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(C);
        cfg.blockDim = dim3(kLcThreads);
        cfg.dynamicSmemBytes = dyn;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg) == cudaSuccess && clusters >= 1) {
          plan->lgC = lgC;
          plan->R = R;
          plan->cap = cap;
          plan->fin = fin;
          return true;
        }
        cudaGetLastError();
      }
    }
  }
  return false;
}

cudaError_t launch_lu_cluster(const LuClusterParams& p, const LcPlan& plan, cudaStream_t s,
                              int64_t* launches) {
  void* fn = lc_kernel(plan.fin);
  const int C = 1 << plan.lgC;
  const size_t dyn = lc_smem(plan.R, plan.cap, plan.fin);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(kLcThreads);
  cfg.dynamicSmemBytes = dyn;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int R = plan.R, lgC = plan.lgC, cap = plan.cap;
  void* args[] = {(void*)&p, (void*)&R, (void*)&lgC, (void*)&cap};
  ++*launches;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace pa
