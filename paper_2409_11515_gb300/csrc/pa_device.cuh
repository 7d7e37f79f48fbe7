// pa_device.cuh -- device helpers shared by the kernel translation units:
// SplitMix64, deterministic block reductions, CSR row products, timers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pa_internal.h"

namespace pa {

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): output i of the generator
// whose state starts at `seed` and advances by the golden gamma.
__host__ __device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ long long globaltimer_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Butterfly sum over a warp: every lane ends with the same bits (each level
// adds the same two values, and + is commutative), in a fixed order.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  return v;
}

// Deterministic block sum of NV values per thread.  `scratch` holds
// NV * (blockDim.x / 32) doubles.  Result valid in every thread.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
  __syncthreads();  // scratch may still be read from a previous call
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) scratch[i * nw + warp] = v[i];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double a = 0.0;
    for (int w = lane; w < nw; w += 32) a += scratch[i * nw + w];
    v[i] = warp_sum(a);
  }
}

// Fixed-order sum of part[k * stride + slot], k < count, done by every warp
// that calls it; all lanes and all callers get identical bits.  Each lane
// issues the loads of up to 16 values before adding any (a loop that adds as
// it loads waits one L2 latency per value: 6 us for 304 values on GB300),
// then adds them pairwise, then a butterfly across the lanes.
__device__ __forceinline__ double ordered_sum(const double* part, int count, int stride, int slot) {
  const int lane = threadIdx.x & 31;
  double acc = 0.0;
  for (int base = 0; base < count; base += 512) {
    double v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int k = base + lane + 32 * i;
      v[i] = k < count ? part[(size_t)k * stride + slot] : 0.0;
    }
#pragma unroll
    for (int w = 1; w < 16; w *= 2)
#pragma unroll
      for (int i = 0; i + w < 16; i += 2 * w) v[i] += v[i + w];
    acc += v[0];
  }
  return warp_sum(acc);
}

// Dot product of one CSR row with a dense vector, entries in storage order,
// one fused multiply-add each.
__device__ __forceinline__ double row_dot(const int32_t* __restrict__ ci,
                                          const double* __restrict__ va, int k0, int k1,
                                          const double* x) {
  double acc = 0.0;
  int k = k0;
  for (; k + 4 <= k1; k += 4) {
    const int c0 = __ldg(ci + k), c1 = __ldg(ci + k + 1), c2 = __ldg(ci + k + 2),
              c3 = __ldg(ci + k + 3);
    const double v0 = __ldg(va + k), v1 = __ldg(va + k + 1), v2 = __ldg(va + k + 2),
                 v3 = __ldg(va + k + 3);
    const double x0 = x[c0], x1 = x[c1], x2 = x[c2], x3 = x[c3];
    acc = fma(v0, x0, acc);
    acc = fma(v1, x1, acc);
    acc = fma(v2, x2, acc);
    acc = fma(v3, x3, acc);
  }
  for (; k < k1; ++k) acc = fma(__ldg(va + k), x[__ldg(ci + k)], acc);
  return acc;
}

// Dot product of lane `lane`'s row of slice s of a sliced-ELL matrix with x:
// entry k sits at 32 * (wp[s] + k) + lane; padding entries hold 0.0.
__device__ __forceinline__ double slice_dot(const int32_t* __restrict__ wp,
                                            const int32_t* __restrict__ col,
                                            const double* __restrict__ val, int s, int lane,
                                            const double* x) {
  const int w0 = __ldg(wp + s), w = __ldg(wp + s + 1) - w0;
  const int64_t base = 32ll * w0 + lane;
  const int32_t* __restrict__ c = col + base;
  const double* __restrict__ v = val + base;
  double acc = 0.0;
  int k = 0;
  for (; k + 4 <= w; k += 4) {
    const int c0 = __ldg(c + 32 * k), c1 = __ldg(c + 32 * (k + 1)), c2 = __ldg(c + 32 * (k + 2)),
              c3 = __ldg(c + 32 * (k + 3));
    const double v0 = __ldg(v + 32 * k), v1 = __ldg(v + 32 * (k + 1)),
                 v2 = __ldg(v + 32 * (k + 2)), v3 = __ldg(v + 32 * (k + 3));
    const double x0 = x[c0], x1 = x[c1], x2 = x[c2], x3 = x[c3];
    acc = fma(v0, x0, acc);
    acc = fma(v1, x1, acc);
    acc = fma(v2, x2, acc);
    acc = fma(v3, x3, acc);
  }
  for (; k < w; ++k) acc = fma(__ldg(v + 32 * k), x[__ldg(c + 32 * k)], acc);
  return acc;
}

// Ask L2 for slice s's columns and values (one warp; s must be a valid
// slice): issued one slice ahead of its use, it turns the warp's dependent
// HBM latency into overlapped traffic.  Every address lies inside the slice.
template <typename V>
__device__ __forceinline__ void prefetch_slice_l2(const int32_t* __restrict__ wp,
                                                  const int32_t* col, const V* val, int s,
                                                  int lane) {
  const int w0 = __ldg(wp + s), w1 = __ldg(wp + s + 1);
  // 32 lanes x 4 bytes of column and 32 x sizeof(V) bytes of value per entry
  const int nbc = 128 * (w1 - w0), nbv = 32 * (int)sizeof(V) * (w1 - w0);
  const char* cb = reinterpret_cast<const char*>(col + 32ll * w0);
  const char* vb = reinterpret_cast<const char*>(val + 32ll * w0);
  for (int l = lane; 128 * l < nbc + nbv; l += 32) {
    const char* a = 128 * l < nbc ? cb + 128 * l : vb + (128 * l - nbc);
    asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
  }
}

// Adam's step K1 m / (sqrt(v) + K2) through one reciprocal square root.  With
// r = 1 / sqrt(v): K1 m / (sqrt(v) (1 + K2 r)) = K1 m r (1 - K2 r + ...), and
// the dropped terms stay below 2^-54 relative while K2 r < 2^-27; otherwise
// (v at or below about (2^27 K2)^2, or v = 0) the quotient itself.  GB300's
// FP64 pipe is narrow, and rsqrt costs far fewer FP64 instructions than a
// square root followed by a division; the result differs from the correctly
// rounded quotient by a few ulp.
__device__ __forceinline__ double adam_quotient(double num, double v, double K2) {
  const double r = rsqrt(v);
  const double kr = K2 * r;
  return kr < 0x1.0p-27 ? num * fma(-kr, r, r) : num / (sqrt(v) + K2);
}

// ---- compensated (double-double) products --------------------------------
// Error-free transformations: TwoProduct with one FMA (p + e = a b exactly)
// and TwoSum (Knuth; s + e = a + b exactly).  The additions are written with
// __dadd_rn / __dsub_rn so the compiler cannot contract them into FMAs.
__device__ __forceinline__ void two_prod(double a, double b, double& p, double& e) {
  p = __dmul_rn(a, b);
  e = fma(a, b, -p);
}
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  const double x = __dadd_rn(a, b);
  const double z = __dsub_rn(x, a);
  e = __dadd_rn(__dsub_rn(a, __dsub_rn(x, z)), __dsub_rn(b, z));
  s = x;
}
// One step of the Dot2 scheme (Ogita, Rump & Oishi 2005): add a*b to the
// running sum s with its error collected in c.
__device__ __forceinline__ void dot2_step(double a, double b, double& s, double& c) {
  double p, pe, t, te;
  two_prod(a, b, p, pe);
  two_sum(s, p, t, te);
  s = t;
  c = __dadd_rn(c, __dadd_rn(te, pe));
}

// Compensated row product of lane `lane` of slice s: returns hi, lo with
// hi = fl(hi + lo) (the unevaluated double-double sum), entries in storage order.
__device__ __forceinline__ void slice_dot_dd(const int32_t* __restrict__ wp,
                                             const int32_t* __restrict__ col,
                                             const double* __restrict__ val, int s, int lane,
                                             const double* x, double& hi, double& lo) {
  const int w0 = __ldg(wp + s), w = __ldg(wp + s + 1) - w0;
  const int64_t base = 32ll * w0 + lane;
  double sum = 0.0, c = 0.0;
  int k = 0;
  for (; k + 4 <= w; k += 4) {  // loads of four entries issued before the chain
    const int64_t e = base + 32ll * k;
    const int j0 = __ldg(col + e), j1 = __ldg(col + e + 32), j2 = __ldg(col + e + 64),
              j3 = __ldg(col + e + 96);
    const double a0 = __ldg(val + e), a1 = __ldg(val + e + 32), a2 = __ldg(val + e + 64),
                 a3 = __ldg(val + e + 96);
    const double x0 = x[j0], x1 = x[j1], x2 = x[j2], x3 = x[j3];
    dot2_step(a0, x0, sum, c);
    dot2_step(a1, x1, sum, c);
    dot2_step(a2, x2, sum, c);
    dot2_step(a3, x3, sum, c);
  }
  for (; k < w; ++k) {
    const int64_t e = base + 32ll * k;
    dot2_step(__ldg(val + e), x[__ldg(col + e)], sum, c);
  }
  two_sum(sum, c, hi, lo);
}

// Compensated row product with a double-double vector (xh + xl): for each
// entry the hi term, then the lo term; rounded to one double.
__device__ __forceinline__ double slice_dot_dd2(const int32_t* __restrict__ wp,
                                                const int32_t* __restrict__ col,
                                                const double* __restrict__ val, int s,
                                                int lane, const double* xh, const double* xl) {
  // sum a (xh + xl): Dot2 over the a xh terms; the a xl terms are O(u) of
  // them, so adding them by FMA to the compensation sum costs only O(u^2)
  // relative error
  const int w0 = __ldg(wp + s), w = __ldg(wp + s + 1) - w0;
  const int64_t base = 32ll * w0 + lane;
  double sum = 0.0, c = 0.0;
  int k = 0;
  for (; k + 2 <= w; k += 2) {  // loads of two entries issued before the chain
    const int64_t e = base + 32ll * k;
    const int32_t j0 = __ldg(col + e), j1 = __ldg(col + e + 32);
    const double a0 = __ldg(val + e), a1 = __ldg(val + e + 32);
    const double h0 = xh[j0], l0 = xl[j0], h1 = xh[j1], l1 = xl[j1];
    dot2_step(a0, h0, sum, c);
    c = fma(a0, l0, c);
    dot2_step(a1, h1, sum, c);
    c = fma(a1, l1, c);
  }
  for (; k < w; ++k) {
    const int64_t e = base + 32ll * k;
    const double a = __ldg(val + e);
    const int32_t j = __ldg(col + e);
    dot2_step(a, xh[j], sum, c);
    c = fma(a, xl[j], c);
  }
  return __dadd_rn(sum, c);
}

// Block sum of NV per-thread values, result in warp 0 (thread 0 uses it).
// Every thread stores its values in `scratch` (NV * blockDim.x doubles); warp
// 0 adds them in a fixed order (lane l: threads l, l+32, ... in a fixed
// pairwise tree, then a butterfly), so the result does not depend on timing.
template <int NV>
__device__ __forceinline__ void block_sum_to0(double (&v)[NV], double* scratch) {
  const int nt = blockDim.x;
  __syncthreads();  // scratch may still be read from a previous call
#pragma unroll
  for (int i = 0; i < NV; ++i) scratch[i * nt + threadIdx.x] = v[i];
  __syncthreads();
  if (threadIdx.x < 32) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      // eight shared-memory values per chunk loaded before they are added
      // pairwise (a running sum would chain one FP64 latency per value)
      double a = 0.0;
      for (int base = 0; base < nt; base += 256) {
        double u[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int t = base + (int)threadIdx.x + 32 * j;
          u[j] = t < nt ? scratch[i * nt + t] : 0.0;
        }
        u[0] += u[1]; u[2] += u[3]; u[4] += u[5]; u[6] += u[7];
        u[0] += u[2]; u[4] += u[6];
        a += u[0] + u[4];
      }
      v[i] = warp_sum(a);
    }
  }
}

// ----------------------------------------------------------- grid sync --
// (used by the persistent kernels; RunState comes from pa_internal.h)

// Grid-wide barrier with a time limit.  Returns false when the wait gave up
// (this CTA's or another's), after which the caller must leave the kernel.
__device__ __forceinline__ bool grid_barrier(RunState* st, unsigned& target, unsigned G,
                                             long long timeout_ns, bool skip_arrival,
                                             int site, int& ok_slot) {
  __syncthreads();
  if (threadIdx.x == 0) {
    target += G;
    int ok = 1;
    if (!skip_arrival) {
      __threadfence();
      atomicAdd(&st->barrier, 1u);
    }
    const long long t0 = globaltimer_ns();
    int spins = 0;
    while (true) {
      const unsigned c = ld_acquire_u32(&st->barrier);
      if ((int)(c - target) >= 0) break;
      // the abort flag and the clock every 8th poll: one L2 round trip per
      // poll, not two, while the barrier is about to complete
      if ((++spins & 7) == 0) {
        if (ld_relaxed_u32(&st->abort) != 0u) { ok = 0; break; }
        if (spins > 64) {
          if (globaltimer_ns() - t0 > timeout_ns) {
            if (atomicExch(&st->abort, 1u) == 0u) st->timeout_site = site;
            ok = 0;
            break;
          }
          __nanosleep(64);
        }
      }
    }
    __threadfence();
    ok_slot = ok;
  }
  __syncthreads();
  return ok_slot != 0;
}

// Wait until every CTA in [lo, hi] has published iterate t (its ready flag
// reaches t), with the same time limit and abort flag as grid_barrier.  Only
// the CTAs whose x rows this CTA's products read take part, so this replaces
// a grid-wide barrier between the update of x and the next product.
// The lanes of warp 0 poll the flags in parallel (lane l takes CTAs lo + l,
// lo + l + 32, ...), so flags that are already set cost one L2 round trip,
// not one per neighbour.
__device__ __forceinline__ bool wait_ready(RunState* st, const unsigned* ready, int lo, int hi,
                                           unsigned t, long long timeout_ns, int site,
                                           int& ok_slot) {
  if (threadIdx.x < 32) {
    int ok = 1;
    const long long t0 = globaltimer_ns();
    int spins = 0;
    for (int j = lo + (int)threadIdx.x; j <= hi && ok; j += 32) {
      while (true) {
        const unsigned c = ld_acquire_u32(ready + j);
        if ((int)(c - t) >= 0) break;
        if ((++spins & 7) == 0) {  // abort flag and clock every 8th poll
          if (ld_relaxed_u32(&st->abort) != 0u) { ok = 0; break; }
          if (spins > 64) {
            if (globaltimer_ns() - t0 > timeout_ns) {
              if (atomicExch(&st->abort, 1u) == 0u) st->timeout_site = site;
              ok = 0;
              break;
            }
            __nanosleep(32);
          }
        }
      }
    }
    ok = __all_sync(0xffffffffu, ok);  // every lane's wait is bounded, so all arrive
    if (threadIdx.x == 0) {
      __threadfence();
      ok_slot = ok;
    }
  }
  __syncthreads();
  return ok_slot != 0;
}

__device__ __forceinline__ void publish_ready(unsigned* flag, unsigned t) {
  __threadfence();
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(flag), "r"(t) : "memory");
}

// ---- shared by the batched (SpMM) kernels ----

// Barrier of one CTA group (the CTAs of one batch item) on its own arrival
// counter, with the same time limit and abort flag as grid_barrier.
__device__ __forceinline__ bool group_barrier(unsigned* counter, unsigned& target, unsigned G,
                                              RunState* st, long long timeout_ns, int& ok_slot) {
  __syncthreads();
  if (threadIdx.x == 0) {
    target += G;
    int ok = 1;
    __threadfence();
    atomicAdd(counter, 1u);
    const long long t0 = globaltimer_ns();
    int spins = 0;
    while (true) {
      const unsigned c = ld_acquire_u32(counter);
      if ((int)(c - target) >= 0) break;
      if ((++spins & 7) == 0) {  // abort flag and clock every 8th poll
        if (ld_relaxed_u32(&st->abort) != 0u) { ok = 0; break; }
        if (spins > 64) {
          if (globaltimer_ns() - t0 > timeout_ns) {
            atomicExch(&st->abort, 1u);
            ok = 0;
            break;
          }
          __nanosleep(64);
        }
      }
    }
    __threadfence();
    ok_slot = ok;
  }
  __syncthreads();
  return ok_slot != 0;
}

// Fixed-order sum of part[q][c][0..nt) by warp w (c = w's column); result in
// lane 0.
__device__ __forceinline__ double slot_sum(const double* slots, int nt) {
  const int lane = threadIdx.x & 31;
  double a = 0.0;
  for (int base = 0; base < nt; base += 256) {  // loads before adds, pairwise
    double u[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int t = base + lane + 32 * j;
      u[j] = t < nt ? slots[t] : 0.0;
    }
    u[0] += u[1]; u[2] += u[3]; u[4] += u[5]; u[6] += u[7];
    u[0] += u[2]; u[4] += u[6];
    a += u[0] + u[4];
  }
  return warp_sum(a);
}

// Compensated (Kahan) FP32 accumulation of bounded per-row terms; the pair
// is handed to the FP64 block reduction as (double)sum - (double)comp.
struct Kahan32 {
  float sum = 0.f, comp = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float y = __fsub_rn(v, comp);
    const float t = __fadd_rn(sum, y);
    comp = __fsub_rn(__fsub_rn(t, sum), y);
    sum = t;
  }
  __device__ __forceinline__ double value() const { return (double)sum - (double)comp; }
};

}  // namespace pa
