// pa_batched.cu -- many Projected Adam runs in one persistent launch: n_mat
// matrices of different sizes, K restart vectors each (Algorithm 1 of the
// paper for every (matrix, restart) pair, gradient Eq. nabla_loss).
//
// The K vectors of a matrix advance together as an n x K block stored row
// major (x[j*K + c]), so each matrix entry is read once per iteration and
// multiplies K gathered values that sit in one contiguous K*8-byte segment
// (sparse matrix times dense block, SpMM).  The grid is cut into groups of
// CTAs, one group per matrix, sized by the matrix's share of the work; a
// group synchronises only among itself (its own barrier counter), so small
// and large matrices proceed independently inside the same launch.
//
// Per column c the CTA keeps its partial sums in fixed shared-memory slots
// (thread t, column c), reduced in a fixed order: the K runs of a matrix are
// each bit-reproducible and independent of the others.  Algorithm 1's
// tracking is per column; when column c improves, phase B copies its x (the
// iterate just scored) into the column's x_min storage, so two iterate
// buffers suffice.
#include <math.h>

#include "pa_device.cuh"
#include "pa_internal.h"

namespace pa {

namespace {

constexpr int kBT = 256;  // threads per CTA of the batched kernel

template <int K>
struct SharedB {
  double part[2][K][kBT];  // per-thread partials, two quantities per phase
  double ca[K], cb[K];     // gradient coefficients per column
  double c[K], inv[K];     // projection coefficient, 1/||x'||
  double q[K];             // ||x_{t-1}||^2 per column
  double best_s[K], best_q[K], last_s[K], last_q[K];  // best / latest scored (||y||^2, ||x||^2)
  int have_best[K], have_last[K];
  int t_min[K], improved[K];
  int brk, ok, status;
  int iters_run;
};

// DD: the products of phase A with Dot2 (TwoProd + TwoSum) kept as y_hi +
// y_lo, and phase B's A^T (y_hi + y_lo) likewise (the MIXED sigma_min).
template <int K, bool DD>
__global__ void __launch_bounds__(kBT, 2) k_batched(const BatchParams bp) {
  __shared__ SharedB<K> sh;
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = kBT / 32;
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
    double qv[K];
#pragma unroll
    for (int c = 0; c < K; ++c) qv[c] = 0.0;
    for (int j = r0 + tid; j < r1; j += kBT)
#pragma unroll
      for (int c = 0; c < K; ++c) qv[c] = fma(it.X0[(size_t)j * K + c], it.X0[(size_t)j * K + c], qv[c]);
    __syncthreads();
#pragma unroll
    for (int c = 0; c < K; ++c) sh.part[1][c][tid] = qv[c];
  }

  for (int t = 1;; ++t) {
    const double* x = cur == 0 ? it.X0 : it.X1;
    // ---- phase A: Y = A X, partials ||y_c||^2 (q partials are in slot 1)
    {
      double sv[K];
#pragma unroll
      for (int c = 0; c < K; ++c) sv[c] = 0.0;
      for (int s = sa0 + warp; s < sa1; s += NW) {
        if (s + NW < sa1) prefetch_slice_l2(it.a_wp, it.a_col, it.a_val, s + NW, lane);
        const int w0 = __ldg(it.a_wp + s), w = __ldg(it.a_wp + s + 1) - w0;
        const int64_t base = 32ll * w0 + lane;
        double acc[K], cmp[K];
#pragma unroll
        for (int c = 0; c < K; ++c) acc[c] = cmp[c] = 0.0;
        for (int k = 0; k < w; ++k) {
          const double a = __ldg(it.a_val + base + 32ll * k);
          const double* xr = x + (size_t)__ldg(it.a_col + base + 32ll * k) * K;
#pragma unroll
          for (int c = 0; c < K; ++c) {
            if (DD) dot2_step(a, xr[c], acc[c], cmp[c]);
            else acc[c] = fma(a, xr[c], acc[c]);
          }
        }
        const int r = 32 * s + lane;
        if (r < it.n_rows) {
#pragma unroll
          for (int c = 0; c < K; ++c) {
            if (DD) {
              double hi, lo;
              two_sum(acc[c], cmp[c], hi, lo);
              acc[c] = hi;
              it.YLO[(size_t)r * K + c] = lo;
            }
            it.Y[(size_t)r * K + c] = acc[c];
            sv[c] = fma(acc[c], acc[c], sv[c]);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < K; ++c) sh.part[0][c][tid] = sv[c];
      __syncthreads();
      // warp w sums column w (and w + NW, ...) of both slots
      for (int c = warp; c < K; c += NW) {
        const double a0 = slot_sum(sh.part[0][c], kBT);
        const double a1 = slot_sum(sh.part[1][c], kBT);
        if (lane == 0) {
          part[((size_t)lb * 4 + 0) * K + c] = a0;
          part[((size_t)lb * 4 + 1) * K + c] = a1;
        }
      }
    }
    if (!group_barrier(counter, target, G, st, bp.timeout_ns, sh.ok)) { status = PA_ERR_TIMEOUT; break; }
    // ---- per-column scalars: score x_{t-1}, gradient coefficients
    for (int c = warp; c < K; c += NW) {
      const double s_ = ordered_sum(part, G, 4 * K, c);
      const double q = ordered_sum(part, G, 4 * K, K + c);
      if (lane == 0) {
        int imp = 0;
        if (!isfinite(s_) || !isfinite(q)) {
          atomicExch(&sh.status, PA_ERR_NONFINITE);
        } else if (t > 1) {
          // L < L_min through the monotone map of the loss (no logarithm in
          // the loop): log-ratio sigma_max: q s_b < q_b s; sigma_min: s q_b < s_b q
          bool better;
          if (!sh.have_best[c]) {
            better = bp.loss == PA_LOSS_QUADRATIC || bp.mode == PA_SIGMA_MIN || s_ > 0.0;
          } else if (bp.loss == PA_LOSS_QUADRATIC) {
            better = bp.mode == PA_SIGMA_MAX ? s_ > sh.best_s[c] : s_ < sh.best_s[c];
          } else {
            better = bp.mode == PA_SIGMA_MAX ? q * sh.best_s[c] < sh.best_q[c] * s_
                                             : s_ * sh.best_q[c] < sh.best_s[c] * q;
          }
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
        if (s_ == 0.0 && isfinite(q)) atomicCAS(&sh.status, PA_OK, PA_WARN_SINGULAR);
        sh.improved[c] = imp;
        double ca, cb;
        if (bp.loss == PA_LOSS_QUADRATIC) { ca = 0.0; cb = -2.0; }
        else { ca = 1.0 / q; cb = -1.0 / s_; }
        if (bp.mode == PA_SIGMA_MIN) { ca = -ca; cb = -cb; }
        const double omb1 = 1.0 - bp.beta1;
        sh.ca[c] = omb1 * ca;
        sh.cb[c] = omb1 * cb;
        sh.q[c] = q;
      }
    }
    __syncthreads();
    if (tid == 0) sh.brk = (sh.status != PA_OK) || (t == bp.iters + 1);
    __syncthreads();
    // x_min of improved columns (phase B would copy them; on the last pass
    // there is no phase B, so the copy happens here)
    if (sh.brk) {
      if (sh.status == PA_OK || sh.status == PA_WARN_SINGULAR) {
        for (int j = r0 + tid; j < r1; j += kBT)
#pragma unroll
          for (int c = 0; c < K; ++c)
            if (sh.improved[c]) it.XMIN[(size_t)j * K + c] = x[(size_t)j * K + c];
      }
      break;
    }

    // ---- phase B: Z = A^T Y, Adam per column, partials x.dx, dx.dx
    {
      const double2 bc = bp.bias[bp.t0 + t - 1];
      const double b1 = bp.beta1, b2 = bp.beta2;
      const double w2 = bp.w2;
      double pxd[K], pdd[K];
#pragma unroll
      for (int c = 0; c < K; ++c) pxd[c] = pdd[c] = 0.0;
      for (int s = st0 + warp; s < st1; s += NW) {
        if (s + NW < st1) prefetch_slice_l2(it.t_wp, it.t_col, it.t_val, s + NW, lane);
        const int w0 = __ldg(it.t_wp + s), w = __ldg(it.t_wp + s + 1) - w0;
        const int64_t base = 32ll * w0 + lane;
        // DD: Dot2 over the a y_hi terms; the a y_lo terms, O(u) of them, are
        // added by FMA to the compensation sum (O(u^2) relative error), as in
        // slice_dot_dd2
        double z[K], zc[K];
#pragma unroll
        for (int c = 0; c < K; ++c) z[c] = zc[c] = 0.0;
        for (int k = 0; k < w; ++k) {
          const double a = __ldg(it.t_val + base + 32ll * k);
          const size_t i = (size_t)__ldg(it.t_col + base + 32ll * k) * K;
          const double* yr = it.Y + i;
#pragma unroll
          for (int c = 0; c < K; ++c) {
            if (DD) {
              dot2_step(a, yr[c], z[c], zc[c]);
              zc[c] = fma(a, it.YLO[i + c], zc[c]);
            } else {
              z[c] = fma(a, yr[c], z[c]);
            }
          }
        }
        if (DD) {
#pragma unroll
          for (int c = 0; c < K; ++c) z[c] = __dadd_rn(z[c], zc[c]);
        }
        const int j = 32 * s + lane;
        if (j < n) {
#pragma unroll
          for (int c = 0; c < K; ++c) {
            const size_t o = (size_t)j * K + c;
            const double xj = x[o];
            if (sh.improved[c]) it.XMIN[o] = xj;
            const double g = (bp.loss == PA_LOSS_QUADRATIC) ? sh.cb[c] * z[c]
                                                            : fma(sh.ca[c], xj, sh.cb[c] * z[c]);
            const double mj = fma(b1, it.M[o], g);
            const double vj = fma(b2, it.V[o], w2 * (g * g));
            it.M[o] = mj;
            it.V[o] = vj;
            const double d = adam_quotient(bc.x * mj, vj, bc.y);
            it.DX[o] = d;
            pxd[c] = fma(xj, d, pxd[c]);
            pdd[c] = fma(d, d, pdd[c]);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < K; ++c) {
        sh.part[0][c][tid] = pxd[c];
        sh.part[1][c][tid] = pdd[c];
      }
      __syncthreads();
      for (int c = warp; c < K; c += NW) {
        const double a0 = slot_sum(sh.part[0][c], kBT);
        const double a1 = slot_sum(sh.part[1][c], kBT);
        if (lane == 0) {
          part[((size_t)lb * 4 + 2) * K + c] = a0;
          part[((size_t)lb * 4 + 3) * K + c] = a1;
        }
      }
    }
    if (!group_barrier(counter, target, G, st, bp.timeout_ns, sh.ok)) { status = PA_ERR_TIMEOUT; break; }
    for (int c = warp; c < K; c += NW) {
      const double p1 = ordered_sum(part, G, 4 * K, 2 * K + c);
      const double p2 = ordered_sum(part, G, 4 * K, 3 * K + c);
      if (lane == 0) {
        if (!isfinite(p1) || !isfinite(p2)) atomicExch(&sh.status, PA_ERR_NONFINITE);
        const double cc = (bp.ablation & PA_ABLATE_NO_TANGENT) ? 0.0 : p1;
        double inv = 1.0;
        if (!(bp.ablation & PA_ABLATE_NO_NORMALISE)) {
          const double a1c = 1.0 + cc;
          inv = rsqrt(fma(a1c * a1c, sh.q[c], fma(-2.0 * a1c, p1, p2)));
        }
        sh.c[c] = cc;
        sh.inv[c] = inv;
      }
    }
    __syncthreads();
    if (sh.status != PA_OK && sh.status != PA_WARN_SINGULAR) break;

    // ---- phase C: x_t per column, ||x_t||^2 partials (slot 1 of phase A)
    {
      double* xo = cur == 0 ? it.X1 : it.X0;
      double qv[K];
#pragma unroll
      for (int c = 0; c < K; ++c) qv[c] = 0.0;
      for (int j = r0 + tid; j < r1; j += kBT) {
#pragma unroll
        for (int c = 0; c < K; ++c) {
          const size_t o = (size_t)j * K + c;
          const double xn = fma(1.0 + sh.c[c], x[o], -it.DX[o]) * sh.inv[c];
          xo[o] = xn;
          qv[c] = fma(xn, xn, qv[c]);
        }
      }
#pragma unroll
      for (int c = 0; c < K; ++c) sh.part[1][c][tid] = qv[c];
      cur ^= 1;
      if (tid == 0) sh.iters_run = t;
    }
    if (!group_barrier(counter, target, G, st, bp.timeout_ns, sh.ok)) { status = PA_ERR_TIMEOUT; break; }
  }

  // results of the group, written by its first CTA
  if (lb == 0 && tid < K) {
    double* out = it.result + (size_t)tid * 4;
    auto Lof = [&](double s_, double q) {
      if (bp.loss == PA_LOSS_QUADRATIC) return bp.mode == PA_SIGMA_MAX ? -s_ : s_;
      const double lx = log(sqrt(q)), lax = log(sqrt(s_));
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

// ---- start vectors and sigma for a batch (blocks of 256 rows per item) ----
constexpr int kRowsPerBlock = 256;

// Raw start vectors: column c of item i from SplitMix64 seeded with output
// (i0 + i) * k_stride + c of `seed` (columns >= k_used repeat column 0).
template <int K>
__global__ void __launch_bounds__(kRowsPerBlock) k_bstart_raw(
    const BatchItem* items, int k_used, int k_stride, int i0, int r0, uint64_t seed,
    const int32_t* blk_item, const int32_t* blk_row0, double* blockpart) {
  __shared__ double sh[K][kRowsPerBlock];
  const int b = blockIdx.x, i = blk_item[b];
  const BatchItem& it = items[i];
  const int64_t j = (int64_t)blk_row0[b] + threadIdx.x;
  double q[K];
#pragma unroll
  for (int c = 0; c < K; ++c) q[c] = 0.0;
  if (j < it.n_cols) {
    const int32_t p = it.pos_c[j];
#pragma unroll
    for (int c = 0; c < K; ++c) {
      const int cc = c < k_used ? c : 0;
      const uint64_t s =
          splitmix64_at(seed, (uint64_t)(i0 + i) * (uint64_t)k_stride + (uint64_t)(r0 + cc));
      const double u = (double)(splitmix64_at(s, (uint64_t)j) >> 11) * 0x1.0p-53;
      const double xv = 2.0 * u - 1.0;
      it.X0[(size_t)p * K + c] = xv;
      q[c] = xv * xv;
    }
  }
#pragma unroll
  for (int c = 0; c < K; ++c) sh[c][threadIdx.x] = q[c];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = warp; c < K; c += kRowsPerBlock / 32) {
    double a = 0.0;
    for (int t = lane; t < kRowsPerBlock; t += 32) a += sh[c][t];
    a = warp_sum(a);
    if (lane == 0) blockpart[(size_t)b * K + c] = a;
  }
}

// One warp per (item, column): 1 / ||x0_c|| from the item's block partials
// in block order.
template <int K>
__global__ void k_bstart_norm(int n_items, const int32_t* item_blk0, const double* blockpart,
                              double* inv) {
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (gw >= n_items * K) return;
  const int i = gw / K, c = gw % K;
  const int b0 = item_blk0[i], nb = item_blk0[i + 1] - b0;
  const double q = ordered_sum(blockpart + (size_t)b0 * K, nb, K, c);
  if ((threadIdx.x & 31) == 0) inv[gw] = 1.0 / sqrt(q);
}

// x0 /= ||x0|| per column; x_min starts as x0 (Algorithm 1's x_min <- x_init).
template <int K>
__global__ void __launch_bounds__(kRowsPerBlock) k_bstart_scale(const BatchItem* items,
                                                                const int32_t* blk_item,
                                                                const int32_t* blk_row0,
                                                                const double* inv) {
  const int b = blockIdx.x, i = blk_item[b];
  const BatchItem& it = items[i];
  const int64_t j = (int64_t)blk_row0[b] + threadIdx.x;
  if (j >= it.n_cols) return;
#pragma unroll
  for (int c = 0; c < K; ++c) {
    const size_t o = (size_t)j * K + c;
    const double v = it.X0[o] * inv[i * K + c];
    it.X0[o] = v;
    it.XMIN[o] = v;
  }
}

// sigma partials: block b covers slices [row0/32, row0/32 + 8) of P A Q^T
// and x rows [row0, row0 + 256) of item i.
template <int K, bool DD>
__global__ void __launch_bounds__(kRowsPerBlock) k_bsigma_part(const BatchItem* items,
                                                               const int32_t* blk_item,
                                                               const int32_t* blk_row0,
                                                               double* blockpart) {
  __shared__ double sh[2][K][kRowsPerBlock];
  const int b = blockIdx.x, i = blk_item[b];
  const BatchItem& it = items[i];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int s = blk_row0[b] / 32 + warp;
  double y2[K], x2[K];
#pragma unroll
  for (int c = 0; c < K; ++c) y2[c] = x2[c] = 0.0;
  if (s < it.n_slices_a) {
    const int w0 = __ldg(it.a_wp + s), w = __ldg(it.a_wp + s + 1) - w0;
    const int64_t base = 32ll * w0 + lane;
    double acc[K], cmp[K];
#pragma unroll
    for (int c = 0; c < K; ++c) acc[c] = cmp[c] = 0.0;
    for (int k = 0; k < w; ++k) {
      const double a = __ldg(it.a_val + base + 32ll * k);
      const double* xr = it.XMIN + (size_t)__ldg(it.a_col + base + 32ll * k) * K;
#pragma unroll
      for (int c = 0; c < K; ++c) {
        if (DD) dot2_step(a, xr[c], acc[c], cmp[c]);
        else acc[c] = fma(a, xr[c], acc[c]);
      }
    }
    if (DD) {  // y rounded from its double-double value
#pragma unroll
      for (int c = 0; c < K; ++c) {
        double hi, lo;
        two_sum(acc[c], cmp[c], hi, lo);
        acc[c] = hi;
      }
    }
    if (32 * s + lane < it.n_rows)
#pragma unroll
      for (int c = 0; c < K; ++c) y2[c] = acc[c] * acc[c];
  }
  const int64_t j = (int64_t)blk_row0[b] + threadIdx.x;
  if (j < it.n_cols)
#pragma unroll
    for (int c = 0; c < K; ++c) {
      const double v = it.XMIN[(size_t)j * K + c];
      x2[c] = v * v;
    }
#pragma unroll
  for (int c = 0; c < K; ++c) {
    sh[0][c][threadIdx.x] = y2[c];
    sh[1][c][threadIdx.x] = x2[c];
  }
  __syncthreads();
  for (int q = warp; q < 2 * K; q += kRowsPerBlock / 32) {
    const double* slot = sh[q / K][q % K];
    double a = 0.0;
    for (int t = lane; t < kRowsPerBlock; t += 32) a += slot[t];
    a = warp_sum(a);
    if (lane == 0) blockpart[(size_t)b * 2 * K + q] = a;
  }
}

template <int K>
__global__ void k_bsigma_final(int n_items, const int32_t* item_blk0, const double* blockpart,
                               double* out) {
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (gw >= n_items * K) return;
  const int i = gw / K, c = gw % K;
  const int b0 = item_blk0[i], nb = item_blk0[i + 1] - b0;
  const double s = ordered_sum(blockpart + (size_t)b0 * 2 * K, nb, 2 * K, c);
  const double q = ordered_sum(blockpart + (size_t)b0 * 2 * K, nb, 2 * K, K + c);
  if ((threadIdx.x & 31) == 0) out[gw] = sqrt(s) / sqrt(q);
}

template <int K>
cudaError_t batch_start_k(const BatchItem* items, int n_items, int k_used, int k_stride, int i0,
                          int r0, uint64_t seed, const int32_t* blk_item, const int32_t* blk_row0, int nb,
                          double* blockpart, const int32_t* item_blk0, cudaStream_t s,
                          int64_t* launches) {
  double* inv = blockpart + (size_t)nb * K;  // n_items * K after the partials
  k_bstart_raw<K><<<nb, kRowsPerBlock, 0, s>>>(items, k_used, k_stride, i0, r0, seed, blk_item,
                                               blk_row0, blockpart);
  const int warps = n_items * K;
  k_bstart_norm<K><<<(warps * 32 + 255) / 256, 256, 0, s>>>(n_items, item_blk0, blockpart, inv);
  k_bstart_scale<K><<<nb, kRowsPerBlock, 0, s>>>(items, blk_item, blk_row0, inv);
  *launches += 3;
  return cudaGetLastError();
}

template <int K>
cudaError_t batch_sigma_k(const BatchItem* items, int n_items, const int32_t* blk_item,
                          const int32_t* blk_row0, int nb, double* blockpart,
                          const int32_t* item_blk0, double* out, bool dd, cudaStream_t s,
                          int64_t* launches) {
  if (dd) k_bsigma_part<K, true><<<nb, kRowsPerBlock, 0, s>>>(items, blk_item, blk_row0, blockpart);
  else k_bsigma_part<K, false><<<nb, kRowsPerBlock, 0, s>>>(items, blk_item, blk_row0, blockpart);
  const int warps = n_items * K;
  k_bsigma_final<K><<<(warps * 32 + 255) / 256, 256, 0, s>>>(n_items, item_blk0, blockpart, out);
  *launches += 2;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_batch_start(const BatchItem* items_dev, int n_items, int K, int k_used,
                               int k_stride, int i0, int r0, uint64_t seed, const int32_t* blk_item,
                               const int32_t* blk_row0, int nb, int /*rows_per_block*/,
                               double* blockpart, const int32_t* item_blk0, cudaStream_t s,
                               int64_t* launches) {
  switch (K) {
    case 1: return batch_start_k<1>(items_dev, n_items, k_used, k_stride, i0, r0, seed, blk_item, blk_row0, nb, blockpart, item_blk0, s, launches);
    case 2: return batch_start_k<2>(items_dev, n_items, k_used, k_stride, i0, r0, seed, blk_item, blk_row0, nb, blockpart, item_blk0, s, launches);
    case 4: return batch_start_k<4>(items_dev, n_items, k_used, k_stride, i0, r0, seed, blk_item, blk_row0, nb, blockpart, item_blk0, s, launches);
    case 8: return batch_start_k<8>(items_dev, n_items, k_used, k_stride, i0, r0, seed, blk_item, blk_row0, nb, blockpart, item_blk0, s, launches);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_batch_sigma(const BatchItem* items_dev, int n_items, int K,
                               const int32_t* blk_item, const int32_t* blk_row0, int nb,
                               int /*rows_per_block*/, double* blockpart,
                               const int32_t* item_blk0, double* out, bool dd, cudaStream_t s,
                               int64_t* launches) {
  switch (K) {
    case 1: return batch_sigma_k<1>(items_dev, n_items, blk_item, blk_row0, nb, blockpart, item_blk0, out, dd, s, launches);
    case 2: return batch_sigma_k<2>(items_dev, n_items, blk_item, blk_row0, nb, blockpart, item_blk0, out, dd, s, launches);
    case 4: return batch_sigma_k<4>(items_dev, n_items, blk_item, blk_row0, nb, blockpart, item_blk0, out, dd, s, launches);
    case 8: return batch_sigma_k<8>(items_dev, n_items, blk_item, blk_row0, nb, blockpart, item_blk0, out, dd, s, launches);
    default: return cudaErrorInvalidValue;
  }
}

static void* batched_fn(int k, bool dd) {
  switch (k) {
    case 1: return dd ? (void*)k_batched<1, true> : (void*)k_batched<1, false>;
    case 2: return dd ? (void*)k_batched<2, true> : (void*)k_batched<2, false>;
    case 4: return dd ? (void*)k_batched<4, true> : (void*)k_batched<4, false>;
    case 8: return dd ? (void*)k_batched<8, true> : (void*)k_batched<8, false>;
    default: return nullptr;
  }
}

int batched_threads() { return kBT; }

int batched_max_blocks(int k, bool dd) {
  void* fn = batched_fn(k, dd);
  if (!fn) return -1;
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kBT, 0) != cudaSuccess) return -1;
  return per * sms;
}

cudaError_t launch_batched(const BatchParams& p, int k, int G, bool dd, cudaStream_t s,
                           int64_t* launches) {
  void* fn = batched_fn(k, dd);
  if (!fn) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(kBT);
  cfg.dynamicSmemBytes = 0;
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
