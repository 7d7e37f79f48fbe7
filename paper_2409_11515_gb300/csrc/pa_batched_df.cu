// pa_batched_df.cu -- the double-float (PA_DF64) form of the batched engine:
// for every (matrix, restart) item, Algorithm 1 of the paper (gradient
// Eq. nabla_loss, log-ratio loss) with the K restarts of a matrix advancing
// together as an n x K block (SpMM).
//
// The arithmetic per column is that of the single-vector double-float
// kernel (pa_iter2.cu): the sliced values of 2^-k A and every vector as
// (hi, lo) float pairs, the products and Adam's per-row arithmetic on the
// FP32 pipe (pa_df.cuh), each thread's partial sums converted to FP64 and
// every block and group reduction and per-column scalar step in FP64.  The
// CTA groups, partitions, group barriers, fixed-order reductions and
// per-column tracking are those of the FP64 batched kernel (pa_batched.cu),
// so every column is bit-reproducible.  The vector blocks are the FP64
// kernel's buffers read as float pairs (the same 8 bytes per value).  A
// column whose ||y||^2 leaves [2^-100, 2^100] ends the item with
// kStatusDfRange, and the host reruns the wave in FP64.
#include <math.h>

#include "pa_device.cuh"
#include "pa_df.cuh"
#include "pa_internal.h"

namespace pa {

namespace {

constexpr int kBTD = 256;  // threads per CTA (the FP64 batched kernel's)

template <int K>
struct SharedBD {
  double part[2][K][kBTD];  // per-thread partials, two quantities per phase
  df ca[K], cb[K];          // g' = ca x + cb z per column
  df a1c[K], inv[K];        // 1 + c and 1 / ||x'|| per column
  double q[K];              // ||x_{t-1}||^2 per column
  double best_s[K], best_q[K], last_s[K], last_q[K];  // (||2^-k A x||^2, ||x||^2)
  int have_best[K], have_last[K];
  int t_min[K], improved[K];
  int brk, ok, status;
  int iters_run;
};

// A row of a block (its K columns, contiguous) as float pairs: 16-byte loads
// and stores when K is even (a row then starts on a 16-byte boundary).
template <int K>
__device__ __forceinline__ void load_row(const float2* p, df (&v)[K]) {
  if constexpr (K % 2 == 0) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int c = 0; c < K / 2; ++c) {
      const float4 t = q[c];
      v[2 * c] = df{t.x, t.y};
      v[2 * c + 1] = df{t.z, t.w};
    }
  } else {
#pragma unroll
    for (int c = 0; c < K; ++c) v[c] = df_load(p + c);
  }
}

template <int K>
__device__ __forceinline__ void store_row(float2* p, const df (&v)[K]) {
  if constexpr (K % 2 == 0) {
    float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
    for (int c = 0; c < K / 2; ++c)
      q[c] = make_float4(v[2 * c].hi, v[2 * c].lo, v[2 * c + 1].hi, v[2 * c + 1].lo);
  } else {
#pragma unroll
    for (int c = 0; c < K; ++c) df_store(p + c, v[c]);
  }
}

// Each column's two CTA partials (slots 2 q and 2 q + 1 of the group's
// partials, q = phase) from the per-thread values in shared memory.
template <int K>
__device__ __forceinline__ void group_partials(SharedBD<K>& sh, double* part, int lb, int q) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = warp; c < K; c += kBTD / 32) {
    const double a0 = slot_sum(sh.part[0][c], kBTD);
    const double a1 = slot_sum(sh.part[1][c], kBTD);
    if (lane == 0) {
      part[((size_t)lb * 4 + 2 * q) * K + c] = a0;
      part[((size_t)lb * 4 + 2 * q + 1) * K + c] = a1;
    }
  }
}

// Two CTAs per SM at K = 8 (128 registers), three at K <= 4 (80 registers):
// the gathers are latency-bound, so the narrower blocks gain from the third CTA.
template <int K>
__global__ void __launch_bounds__(kBTD, (K <= 4 ? 3 : 2)) k_batched_df(const BatchParams bp) {
  __shared__ SharedBD<K> sh;
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = kBTD / 32;
  const int item = bp.cta_item[b];
  const BatchItem& it = bp.items[item];
  const int lb = b - it.cta0;  // CTA index inside the group
  const unsigned G = (unsigned)it.ncta;
  const int sa0 = it.part_a[lb], sa1 = it.part_a[lb + 1];
  const int st0 = it.part_t[lb], st1 = it.part_t[lb + 1];
  const int n = it.n_cols;
  const int r0 = 32 * st0, r1 = min(32 * st1, n);
  RunState* st = bp.st;
  unsigned* counter = it.barrier;
  double* part = it.partials;  // [G][4][K]
  float2* const X0 = reinterpret_cast<float2*>(it.X0);
  float2* const X1 = reinterpret_cast<float2*>(it.X1);
  float2* const XMIN = reinterpret_cast<float2*>(it.XMIN);
  float2* const M = reinterpret_cast<float2*>(it.M);
  float2* const V = reinterpret_cast<float2*>(it.V);
  float2* const DX = reinterpret_cast<float2*>(it.DX);
  float2* const Y = reinterpret_cast<float2*>(it.Y);
  const df b1d = df_from_double(bp.beta1), b2d = df_from_double(bp.beta2),
           w2d = df_from_double(bp.w2);
  unsigned target = 0;
  int status = PA_OK;

  if (tid < K) {
    sh.have_best[tid] = 0;
    sh.have_last[tid] = 0;
    sh.t_min[tid] = 0;
    sh.improved[tid] = 0;
  }
  int cur = 0;  // every thread flips it in step: X0/X1 hold x_{t-1} / x_t
  if (tid == 0) {
    sh.brk = 0;
    sh.status = PA_OK;
    sh.iters_run = 0;
  }
  // ||x_init||^2 per column over the own rows
  {
    DfAcc qa[K];
    for (int j = r0 + tid; j < r1; j += kBTD)
#pragma unroll
      for (int c = 0; c < K; ++c) {
        const df xv = df_load(X0 + (size_t)j * K + c);
        qa[c].add_prod(xv, xv);
      }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < K; ++c) sh.part[1][c][tid] = df_to_double(qa[c].value());
  }

  for (int t = 1;; ++t) {
    const float2* x = cur == 0 ? X0 : X1;
    // ---- phase A: Y = 2^-k A X, partials ||y_c||^2 (q partials are in slot 1)
    {
      DfAcc sv[K];
      for (int s = sa0 + warp; s < sa1; s += NW) {
        if (s + NW < sa1) prefetch_slice_l2(it.a_wp, it.a_col, it.a_val2, s + NW, lane);
        const int w0 = __ldg(it.a_wp + s), w = __ldg(it.a_wp + s + 1) - w0;
        const int64_t base = 32ll * w0 + lane;
        DfAcc acc[K];
        for (int k = 0; k < w; ++k) {
          const float2 av = __ldg(it.a_val2 + base + 32ll * k);
          const df a{av.x, av.y};
          df xv[K];
          load_row<K>(x + (size_t)__ldg(it.a_col + base + 32ll * k) * K, xv);
#pragma unroll
          for (int c = 0; c < K; ++c) acc[c].add_prod(a, xv[c]);
        }
        const int r = 32 * s + lane;
        if (r < it.n_rows) {
          df y[K];
#pragma unroll
          for (int c = 0; c < K; ++c) {
            y[c] = acc[c].value();
            sv[c].add_prod(y[c], y[c]);
          }
          store_row<K>(Y + (size_t)r * K, y);
        }
      }
#pragma unroll
      for (int c = 0; c < K; ++c) sh.part[0][c][tid] = df_to_double(sv[c].value());
      __syncthreads();
      group_partials<K>(sh, part, lb, 0);
    }
    if (!group_barrier(counter, target, G, st, bp.timeout_ns, sh.ok)) { status = PA_ERR_TIMEOUT; break; }
    // ---- per-column scalars (FP64): score x_{t-1}, gradient coefficients
    for (int c = warp; c < K; c += NW) {
      const double s_ = ordered_sum(part, G, 4 * K, c);
      const double q = ordered_sum(part, G, 4 * K, K + c);
      if (lane == 0) {
        int imp = 0;
        if (!isfinite(q) || !(s_ >= 0x1.0p-100 && s_ <= 0x1.0p100)) {
          atomicExch(&sh.status, kStatusDfRange);  // outside the variant's range
        } else if (t > 1) {
          // L < L_min through the monotone map of the log-ratio loss:
          // sigma_max: q s_b < q_b s; sigma_min: s q_b < s_b q (the 4^k of
          // the scaled products cancels)
          bool better;
          if (!sh.have_best[c]) better = true;
          else better = bp.mode == PA_SIGMA_MAX ? q * sh.best_s[c] < sh.best_q[c] * s_
                                                : s_ * sh.best_q[c] < sh.best_s[c] * q;
          if (better) {
            sh.best_s[c] = s_;
            sh.best_q[c] = q;
            sh.have_best[c] = 1;
            sh.t_min[c] = t - 1;
            imp = 1;
          }
          sh.last_s[c] = s_;
          sh.last_q[c] = q;
          sh.have_last[c] = 1;
        }
        sh.improved[c] = imp;
        double ca = 1.0 / q, cb = -1.0 / s_;
        if (bp.mode == PA_SIGMA_MIN) { ca = -ca; cb = -cb; }
        const double omb1 = 1.0 - bp.beta1;
        sh.ca[c] = df_from_double(omb1 * ca);
        sh.cb[c] = df_from_double(omb1 * cb);
        sh.q[c] = q;
      }
    }
    __syncthreads();
    if (tid == 0) sh.brk = (sh.status != PA_OK) || (t == bp.iters + 1);
    __syncthreads();
    if (sh.brk) {  // the last pass has no phase B: x_min of improved columns here
      if (sh.status == PA_OK) {
        for (int j = r0 + tid; j < r1; j += kBTD)
#pragma unroll
          for (int c = 0; c < K; ++c)
            if (sh.improved[c]) XMIN[(size_t)j * K + c] = x[(size_t)j * K + c];
      }
      break;
    }

    // ---- phase B: Z = 2^-k A^T Y, Adam per column, partials x.dx, dx.dx
    {
      const float4 bq = bp.bias2[bp.t0 + t - 1];
      const df K1{bq.x, bq.y}, K2{bq.z, bq.w};
      DfAcc pxd[K], pdd[K];
      for (int s = st0 + warp; s < st1; s += NW) {
        if (s + NW < st1) prefetch_slice_l2(it.t_wp, it.t_col, it.t_val2, s + NW, lane);
        const int w0 = __ldg(it.t_wp + s), w = __ldg(it.t_wp + s + 1) - w0;
        const int64_t base = 32ll * w0 + lane;
        DfAcc z[K];
        for (int k = 0; k < w; ++k) {
          const float2 av = __ldg(it.t_val2 + base + 32ll * k);
          const df a{av.x, av.y};
          df yv[K];
          load_row<K>(Y + (size_t)__ldg(it.t_col + base + 32ll * k) * K, yv);
#pragma unroll
          for (int c = 0; c < K; ++c) z[c].add_prod(a, yv[c]);
        }
        const int j = 32 * s + lane;
        if (j < n) {
          const size_t o = (size_t)j * K;
          df xr[K], mr[K], vr[K];
          load_row<K>(x + o, xr);
          load_row<K>(M + o, mr);
          load_row<K>(V + o, vr);
#pragma unroll
          for (int c = 0; c < K; ++c) {
            const df xj = xr[c];
            if (sh.improved[c]) df_store(XMIN + o + c, xj);
            const df g = df_add(df_mul(sh.ca[c], xj), df_mul(sh.cb[c], z[c].value()));
            mr[c] = df_add(df_mul(b1d, mr[c]), g);
            vr[c] = df_add(df_mul(b2d, vr[c]), df_mul(w2d, df_mul(g, g)));
            const df d = df_div(df_mul(K1, mr[c]), df_add(df_sqrt(vr[c]), K2));
            xr[c] = d;  // the row of dx
            pxd[c].add_prod(xj, d);
            pdd[c].add_prod(d, d);
          }
          store_row<K>(M + o, mr);
          store_row<K>(V + o, vr);
          store_row<K>(DX + o, xr);
        }
      }
#pragma unroll
      for (int c = 0; c < K; ++c) {
        sh.part[0][c][tid] = df_to_double(pxd[c].value());
        sh.part[1][c][tid] = df_to_double(pdd[c].value());
      }
      __syncthreads();
      group_partials<K>(sh, part, lb, 1);
    }
    if (!group_barrier(counter, target, G, st, bp.timeout_ns, sh.ok)) { status = PA_ERR_TIMEOUT; break; }
    for (int c = warp; c < K; c += NW) {
      const double p1 = ordered_sum(part, G, 4 * K, 2 * K + c);
      const double p2 = ordered_sum(part, G, 4 * K, 3 * K + c);
      if (lane == 0) {
        if (!isfinite(p1) || !isfinite(p2)) atomicExch(&sh.status, kStatusDfRange);
        const double cc = (bp.ablation & PA_ABLATE_NO_TANGENT) ? 0.0 : p1;
        double inv = 1.0;
        if (!(bp.ablation & PA_ABLATE_NO_NORMALISE)) {
          const double a1c = 1.0 + cc;
          inv = rsqrt(fma(a1c * a1c, sh.q[c], fma(-2.0 * a1c, p1, p2)));
        }
        sh.a1c[c] = df_from_double(1.0 + cc);
        sh.inv[c] = df_from_double(inv);
      }
    }
    __syncthreads();
    if (sh.status != PA_OK) break;

    // ---- phase C: x_t per column, ||x_t||^2 partials (slot 1 of phase A)
    {
      float2* xo = cur == 0 ? X1 : X0;
      DfAcc qv[K];
      for (int j = r0 + tid; j < r1; j += kBTD) {
        const size_t o = (size_t)j * K;
        df xr[K], dr[K];
        load_row<K>(x + o, xr);
        load_row<K>(DX + o, dr);
#pragma unroll
        for (int c = 0; c < K; ++c) {
          xr[c] = df_mul(df_sub(df_mul(sh.a1c[c], xr[c]), dr[c]), sh.inv[c]);
          qv[c].add_prod(xr[c], xr[c]);
        }
        store_row<K>(xo + o, xr);
      }
#pragma unroll
      for (int c = 0; c < K; ++c) sh.part[1][c][tid] = df_to_double(qv[c].value());
      cur ^= 1;
      if (tid == 0) sh.iters_run = t;
    }
    if (!group_barrier(counter, target, G, st, bp.timeout_ns, sh.ok)) { status = PA_ERR_TIMEOUT; break; }
  }

  // results of the group, written by its first CTA (L with ||A x||^2 = 4^k s)
  if (lb == 0 && tid < K) {
    double* out = it.result + (size_t)tid * 4;
    auto Lof = [&](double s_, double q) {
      const double lx = log(sqrt(q)), lax = log(sqrt(s_ * it.s_scale));
      return bp.mode == PA_SIGMA_MAX ? lx - lax : lax - lx;
    };
    out[0] = sh.have_best[tid] ? Lof(sh.best_s[tid], sh.best_q[tid]) : INFINITY;
    out[1] = sh.t_min[tid];
    out[2] = sh.have_last[tid] ? Lof(sh.last_s[tid], sh.last_q[tid]) : NAN;
    out[3] = sh.iters_run;
  }
  if (lb == 0 && tid == 0) {
    int s = sh.status;
    if (status == PA_ERR_TIMEOUT || ld_relaxed_u32(&st->abort) != 0u) s = PA_ERR_TIMEOUT;
    it.status[0] = s;
  }
}

static void* batched_df_fn(int k) {
  switch (k) {
    case 1: return (void*)k_batched_df<1>;
    case 2: return (void*)k_batched_df<2>;
    case 4: return (void*)k_batched_df<4>;
    case 8: return (void*)k_batched_df<8>;
    default: return nullptr;
  }
}

}  // namespace

int batched_df_max_blocks(int k) {
  void* fn = batched_df_fn(k);
  if (!fn) return -1;
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kBTD, 0) != cudaSuccess) return -1;
  return per * sms;
}

cudaError_t launch_batched_df(const BatchParams& p, int k, int G, cudaStream_t s,
                              int64_t* launches) {
  void* fn = batched_df_fn(k);
  if (!fn) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(kBTD);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[] = {(void*)&p};
  ++*launches;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace pa
