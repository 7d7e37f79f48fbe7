// pa_iter2.cu -- the merged-phase persistent Projected Adam kernel (the
// paper's Algorithm 1 with the gradient of Eq. nabla_loss) for one vector,
// in an FP64 and a double-float (PA_DF64) variant.
//
// It computes the same iteration as k_persistent (pa_iter.cu) but moves the
// update and normalisation of x -- Algorithm 1's last two lines -- out of a
// pass of their own and into the next product.  With dx_t the Adam step,
// c = x_{t-1} . dx_t the tangent projection's coefficient and
// u_t = x_{t-1} - dx_t, Algorithm 1 sets
//     x_t = ((1 + c) x_{t-1} - dx_t) / ||.|| = inv (u_t + c x_{t-1}),
// and since A is linear,
//     y_t = A x_t = inv (A u_t + c y_{t-1}).
// A u_t needs only u_t, which every CTA writes at the end of its phase B
// without waiting for the grid, so the product of iteration t+1 starts as
// soon as the neighbours' u_t rows are written; c and inv (grid sums of
// phase B) are needed only to finish the rows.  Per iteration t:
//
//   A  wait for the neighbours' u_{t-1} flags; w = A u_{t-1} for the CTA's
//      first kMergedWin slices (kept in shared memory); wait for the grid's
//      phase-B arrivals of iteration t-1 (normally complete by then) and sum
//      its partials -> c, inv; y_{t-1} = inv (w + c y_{t-2}) for the own rows
//      of A (slices beyond the window are multiplied and finished at once);
//      x_{t-1} = inv (u_{t-1} + c x_{t-2}) for the own x rows; partials
//      ||y||^2, ||x||^2                                      | grid barrier
//      every CTA sums the partials in the same order: L(x_{t-1}) is scored
//      (Algorithm 1's tracking) and the gradient coefficients formed
//   B  z = A^T y over the explicit transpose, g = a x + b z, Adam's moments
//      and step dx, u_t = x_{t-1} - dx, partials x.dx and dx.dx; the CTA then
//      publishes "u_t written" and arrives on the split barrier without
//      waiting.
//
// One full grid barrier per iteration instead of two, and no pass of its own
// for the update of x.  The recursion for y carries y_{t-2}'s rounding error
// times c inv into y_{t-1}; Adam's early steps on large matrices have a big
// radial part (|c inv| > 1, so that error would grow geometrically), and an
// iteration whose |c inv| exceeds 1/2 therefore writes x_{t-1} first,
// publishes it and multiplies x_{t-1} itself (a refresh).  The error carried
// by y then stays below twice one iteration's rounding.  To keep such
// iterations rare, phase B folds the previous iteration's coefficient c_hat
// into u = (1 + c_hat) x - dx, so that only the change c - c_hat multiplies
// the carried error (c moves slowly once Adam's moments have settled).  At t = 1 phase A multiplies x_0 itself.  The first
// iteration that scores x_T runs phase A only.  Every wait is bounded by a
// %globaltimer budget and the shared abort flag (PA_ERR_TIMEOUT, no hang).
//
// The double-float variant stores the sliced values of 2^-k A (k from the
// largest |a_ij|, an exact power-of-two scaling that leaves the log-ratio
// iterates unchanged) and every vector as (hi, lo) float pairs -- the same
// 8 bytes per value as FP64 -- and runs the products and the per-row Adam
// arithmetic on the FP32 pipe (pa_df.cuh); partial sums, the grid sums and
// the per-iteration scalars stay in FP64.  A run whose ||y||^2 leaves
// [2^-100, 2^100] ends with kStatusDfRange and the host reruns it in FP64.
#include <math.h>

#include <algorithm>
#include <climits>
#include <type_traits>

#include "pa_device.cuh"
#include "pa_df.cuh"
#include "pa_internal.h"

namespace pa {

namespace {

constexpr int kU = 1;  // rows per thread and pass in the row loops of phase A

struct SharedM {
  double scratch[2 * kBlock];
  double ca, cb;    // g' = ca x + cb z
  df ca2, cb2;
  double c, inv;    // c - c_hat and 1 / ||x'|| of the previous iteration
  df c2, inv2;
  double chat;      // c_hat: the projection coefficient folded into u by phase B
  df chat2;
  double q_keep;    // ||x_{t-1}||^2 from the latest scalar step
  int brk, cur, nb, ok, refresh, refreshes, prev_refresh;
  double best_s, best_q, last_s, last_q;
  int have_best, have_last;
  int minb, t_min, iters_run, status;
  unsigned long long busy_a, busy_b, lat_a;
  long long tmark, tendb, twait;
};

template <bool DF>
struct Arith;

template <>
struct Arith<false> {
  using W = double;
};
template <>
struct Arith<true> {
  using W = df;
};

__device__ __forceinline__ double loss_value2(int mode, int loss, double s, double q) {
  if (loss == PA_LOSS_QUADRATIC) return mode == PA_SIGMA_MAX ? -s : s;
  const double lx = log(sqrt(q)), lax = log(sqrt(s));
  return mode == PA_SIGMA_MAX ? lx - lax : lax - lx;
}

// Double-float product of lane `lane`'s row of slice s with x (both as
// (hi, lo) pairs), entries in storage order.
__device__ __forceinline__ df slice_dot_df(const int32_t* __restrict__ wp,
                                           const int32_t* __restrict__ col,
                                           const float2* __restrict__ val, int s, int lane,
                                           const float2* x) {
  const int w0 = __ldg(wp + s), w = __ldg(wp + s + 1) - w0;
  const int64_t base = 32ll * w0 + lane;
  const int32_t* __restrict__ c = col + base;
  const float2* __restrict__ v = val + base;
  DfAcc acc;
  int k = 0;
  for (; k + 4 <= w; k += 4) {
    const int c0 = __ldg(c + 32 * k), c1 = __ldg(c + 32 * (k + 1)), c2 = __ldg(c + 32 * (k + 2)),
              c3 = __ldg(c + 32 * (k + 3));
    const float2 v0 = __ldg(v + 32 * k), v1 = __ldg(v + 32 * (k + 1)),
                 v2 = __ldg(v + 32 * (k + 2)), v3 = __ldg(v + 32 * (k + 3));
    const float2 x0 = x[c0], x1 = x[c1], x2 = x[c2], x3 = x[c3];
    acc.add_prod(df{v0.x, v0.y}, df{x0.x, x0.y});
    acc.add_prod(df{v1.x, v1.y}, df{x1.x, x1.y});
    acc.add_prod(df{v2.x, v2.y}, df{x2.x, x2.y});
    acc.add_prod(df{v3.x, v3.y}, df{x3.x, x3.y});
  }
  for (; k < w; ++k) {
    const float2 a = __ldg(v + 32 * k), xx = x[__ldg(c + 32 * k)];
    acc.add_prod(df{a.x, a.y}, df{xx.x, xx.y});
  }
  return acc.value();
}

// Every thread of the CTA asks L2 for every 128-byte line of [base, base +
// bytes): issued ahead of a pass over the CTA's own rows, so that the pass
// finds them in L2 instead of waiting one HBM latency per row it handles.
__device__ __forceinline__ void prefetch_range_l2(const void* base, size_t bytes) {
  const char* b = static_cast<const char*>(base);
  for (size_t off = 128 * (size_t)threadIdx.x; off < bytes; off += 128 * (size_t)blockDim.x)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(b + off));
}

// Wait until the arrival counter reaches `target` (thread 0 only); bounded
// like grid_barrier.  Returns 0 when the wait gave up.
__device__ __forceinline__ int wait_count(RunState* st, unsigned target, long long timeout_ns,
                                          int site) {
  const long long t0 = globaltimer_ns();
  int spins = 0;
  while (true) {
    const unsigned c = ld_acquire_u32(&st->barrier);
    if ((int)(c - target) >= 0) break;
    if ((++spins & 7) == 0) {
      if (ld_relaxed_u32(&st->abort) != 0u) return 0;
      if (spins > 64) {
        if (globaltimer_ns() - t0 > timeout_ns) {
          if (atomicExch(&st->abort, 1u) == 0u) st->timeout_site = site;
          return 0;
        }
        __nanosleep(64);
      }
    }
  }
  __threadfence();
  return 1;
}

template <int LOSS, bool DF, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) k_merged(const IterParams p) {
  using W = typename Arith<DF>::W;
  __shared__ SharedM sh;
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  W* const wbuf = reinterpret_cast<W*>(dyn_smem);  // [32 * win_slices]
  constexpr int NW = kBlock / 32;
  const unsigned G = gridDim.x;
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int sa0 = p.part_a[b], sa1 = p.part_a[b + 1];
  const int st0 = p.part_t[b], st1 = p.part_t[b + 1];
  const int n = p.n_cols;
  const int r0 = 32 * st0, r1 = min(32 * st1, n);  // own rows of x (positions)
  RunState* st = p.st;
  double* __restrict__ part = p.partials;
  // iterate buffer k (selects instead of an indexed array: no local memory)
  auto X64 = [&](int k) { return k == 0 ? p.X0 : (k == 1 ? p.X1 : p.X2); };
  auto X32 = [&](int k) { return k == 0 ? p.XD0 : (k == 1 ? p.XD1 : p.XD2); };

  unsigned target = 0;  // thread 0: arrivals the next wait needs
  int site = 0;
  int status = PA_OK;
  if (tid == 0) {
    sh.cur = 0;
    sh.brk = 0;
    sh.minb = 0;
    sh.t_min = 0;
    sh.iters_run = 0;
    sh.status = PA_OK;
    sh.have_best = 0;
    sh.have_last = 0;
    sh.busy_a = sh.busy_b = sh.lat_a = 0;
    sh.tendb = 0;
    sh.c = 0.0;
    sh.inv = 1.0;
    sh.chat = 0.0;
    sh.chat2 = df{0.f, 0.f};
    sh.q_keep = 1.0;
    sh.refresh = 0;
    sh.refreshes = 0;
    sh.prev_refresh = 0;
  }
  const int dlo = p.dep[2 * b], dhi = p.dep[2 * b + 1];
  // Adam constants as double-word pairs (each thread, once)
  df b1d{}, b2d{}, w2d{};
  if (DF) {
    b1d = df_from_double(p.beta1);
    b2d = df_from_double(p.beta2);
    w2d = df_from_double(p.w2);
  }
  __syncthreads();

  for (int t = 1;; ++t) {
    // ================= phase A(t): x_{t-1}, y_{t-1} = A x_{t-1}
    // flags: phase B of iteration t publishes 2t (u_t written), a refreshing
    // phase A(t) publishes 2t - 1 (x_{t-1} written)
    if (t > 1 && !wait_ready(st, p.ready, dlo, dhi, (unsigned)(2 * t - 2), p.timeout_ns, site++,
                             sh.ok)) {
      status = PA_ERR_TIMEOUT;
      break;
    }
    if (tid == 0) sh.tmark = globaltimer_ns();
    const int cur = sh.cur;  // x_{t-2} (t > 1) or x_0
    // products of the loops below: the slice at entry k of this warp's list
    // times u_{t-1} (from < 0) or times iterate buffer `from`;
    // this warp's share of the CTA's slices of P A Q^T: a_list[ka0 .. ka1)
    const int ka0 = p.a_woff[b * (NW + 1) + warp], ka1 = p.a_woff[b * (NW + 1) + warp + 1];
    auto product = [&](int k, int from) -> W {
      const int sl = __ldg(p.a_list + k);
      if (k + 1 < ka1) {
        const int nx = __ldg(p.a_list + k + 1);
        if (DF) prefetch_slice_l2(p.a_wp, p.a_col, p.a_val2, nx, lane);
        else prefetch_slice_l2(p.a_wp, p.a_col, p.a_val, nx, lane);
      }
      if constexpr (DF)
        return slice_dot_df(p.a_wp, p.a_col, p.a_val2, sl, lane, from < 0 ? p.ud : X32(from));
      else
        return slice_dot(p.a_wp, p.a_col, p.a_val, sl, lane, from < 0 ? p.u : X64(from));
    };
    // Speculative products w = A u_{t-1} of the CTA's first win_slices
    // slices, into shared memory, while the grid's phase-B arrivals complete.
    // Skipped after an iteration that refreshed (the next one most likely
    // refreshes too, and would drop them).
    const bool spec = t > 1 && !sh.prev_refresh;
    const int swin = spec ? min(sa1, sa0 + p.win_slices) : sa0;
    if (spec)
      for (int k = ka0; k < ka1; ++k) {
        const int sl = __ldg(p.a_list + k);
        if (sl < swin) wbuf[32 * (sl - sa0) + lane] = product(k, -1);
      }
    if (t > 1) {  // what the row passes below read: y_{t-2}, x_{t-2} and u_{t-1} rows
      const int ra = 32 * sa0, rb = min(32 * sa1, p.n_rows);
      if (rb > ra) prefetch_range_l2(DF ? (const void*)(p.yd + ra) : (const void*)(p.y + ra),
                                     (size_t)(rb - ra) * 8);
      if (r1 > r0) {
        prefetch_range_l2(DF ? (const void*)(X32(cur) + r0) : (const void*)(X64(cur) + r0),
                          (size_t)(r1 - r0) * 8);
        prefetch_range_l2(DF ? (const void*)(p.ud + r0) : (const void*)(p.u + r0),
                          (size_t)(r1 - r0) * 8);
      }
    }
    int xb = cur;  // buffer that receives x_{t-1}
    int refresh = 0;
    if (t > 1) {
      // the split barrier of iteration t-1: every CTA's phase B has arrived
      if (tid == 0) {
        target += G;
        const long long tw = globaltimer_ns();
        sh.ok = wait_count(st, target, p.timeout_ns, site);
        sh.twait = globaltimer_ns() - tw;
      }
      ++site;
      __syncthreads();
      if (!sh.ok) {
        status = PA_ERR_TIMEOUT;
        break;
      }
      if (tid < 32) {
        const double p1 = ordered_sum(part, G, kPartSlots, 2);
        const double p2 = ordered_sum(part, G, kPartSlots, 3);
        if (tid == 0) {
          int brk = 0;
          if (!isfinite(p1) || !isfinite(p2)) {
            sh.status = DF ? kStatusDfRange : PA_ERR_NONFINITE;
            brk = 1;
          }
          const double c = (p.ablation & PA_ABLATE_NO_TANGENT) ? 0.0 : p1;
          double inv = 1.0;
          if (!(p.ablation & PA_ABLATE_NO_NORMALISE)) {
            const double a1c = 1.0 + c;
            // ||(1+c) x - dx||^2 = (1+c)^2 q - 2 (1+c) p1 + p2
            const double nrm2 = fma(a1c * a1c, sh.q_keep, fma(-2.0 * a1c, p1, p2));
            inv = rsqrt(nrm2);  // scales x only: the loss and Adam's step are scale-free
          }
          // phase B folded c_hat (the previous iteration's c) into u, so
          // x_{t-1} = inv (u + (c - c_hat) x_{t-2}) and likewise for y
          const double cr = c - sh.chat;
          sh.c = cr;
          sh.inv = inv;
          sh.chat = c;
          // y_{t-1} = inv (A u + cr y_{t-2}) carries y_{t-2}'s rounding error
          // times cr inv: past 1/2, multiply x_{t-1} itself instead
          sh.refresh = fabs(cr) * inv > 0.5;
          sh.refreshes += sh.refresh;
          sh.prev_refresh = sh.refresh;
          if (DF) {
            sh.c2 = df_from_double(cr);
            sh.inv2 = df_from_double(inv);
            sh.chat2 = df_from_double(c);
          }
          const int minb = sh.minb;
          sh.nb = (cur != 0 && minb != 0) ? 0 : ((cur != 1 && minb != 1) ? 1 : 2);
          sh.brk = brk;
        }
      }
      __syncthreads();
      if (sh.brk) break;
      xb = sh.nb;
      refresh = sh.refresh;
    }
    {
      double v[2] = {0.0, 0.0};
      const double c = sh.c, inv = sh.inv;
      const df c2 = sh.c2, inv2 = sh.inv2;
      DfAcc sacc, qacc;
      // row r of y: the product itself (t == 1, refresh) or inv (w + c y_{t-2});
      // y_{t-2} is loaded by the caller ahead of its use
      using S = typename std::conditional<DF, float2, double>::type;
      S* const ybuf = DF ? (S*)p.yd : (S*)p.y;
      auto finish_row = [&](int r, W wv, S yo, bool direct) {
        if constexpr (DF) {
          df yn = wv;
          if (!direct) yn = df_mul(inv2, df_add(wv, df_mul(c2, df{yo.x, yo.y})));
          df_store(p.yd + r, yn);
          sacc.add_prod(yn, yn);
        } else {
          double yn = wv;
          if (!direct) yn = fma(c, yo, wv) * inv;
          p.y[r] = yn;
          v[0] = fma(yn, yn, v[0]);
        }
      };
      // slice sl's row of this lane, multiplied now (y_{t-2} loaded first)
      // entry k of this warp's list, multiplied now (y_{t-2} loaded first)
      auto multiply_finish = [&](int k, int from, bool direct) {
        const int r = 32 * __ldg(p.a_list + k) + lane;
        S yo{};
        if (!direct && r < p.n_rows) yo = ybuf[r];
        const W wv = product(k, from);
        if (r < p.n_rows) finish_row(r, wv, yo, direct);
      };
      // own x rows: x_{t-1} (written into buffer xb for t > 1) and ||x||^2
      // (kU rows per thread and pass, their loads issued before any use)
      auto finish_x = [&]() {
        double* tr = (p.x_trace && t > 1 && t - 1 <= p.n_trace)
                         ? p.x_trace + (size_t)(t - 2) * n : nullptr;
        S* const xo_buf = DF ? (S*)X32(cur) : (S*)X64(cur);
        S* const xn_buf = DF ? (S*)X32(xb) : (S*)X64(xb);
        const S* const u_buf = DF ? (const S*)p.ud : (const S*)p.u;
        for (int j0 = r0 + tid; j0 < r1; j0 += kU * kBlock) {
          S xo[kU], uu[kU];
#pragma unroll
          for (int k = 0; k < kU; ++k) {
            const int j = j0 + k * kBlock;
            if (j < r1) {
              xo[k] = xo_buf[j];
              if (t > 1) uu[k] = u_buf[j];
            }
          }
#pragma unroll
          for (int k = 0; k < kU; ++k) {
            const int j = j0 + k * kBlock;
            if (j >= r1) continue;
            if constexpr (DF) {
              df xn{xo[k].x, xo[k].y};
              if (t > 1) {
                xn = df_mul(inv2, df_add(df{uu[k].x, uu[k].y}, df_mul(c2, xn)));
                xn_buf[j] = make_float2(xn.hi, xn.lo);
                if (tr) tr[j] = df_to_double(xn);
              }
              qacc.add_prod(xn, xn);
            } else {
              double xn = xo[k];
              if (t > 1) {
                xn = fma(c, xn, uu[k]) * inv;
                xn_buf[j] = xn;
                if (tr) tr[j] = xn;
              }
              v[1] = fma(xn, xn, v[1]);
            }
          }
        }
      };
      if (refresh) {
        // x_{t-1} first, published, then y_{t-1} = A x_{t-1} from it (any
        // speculative products of u are dropped)
        finish_x();
        __syncthreads();
        if (tid == 0) publish_ready(p.ready + b, (unsigned)(2 * t - 1));
        if (!wait_ready(st, p.ready, dlo, dhi, (unsigned)(2 * t - 1), p.timeout_ns, site++,
                        sh.ok)) {
          status = PA_ERR_TIMEOUT;
          break;
        }
        for (int k = ka0; k < ka1; ++k) multiply_finish(k, xb, true);
      } else {
        // the speculative rows from shared memory (all threads, coalesced),
        // then the remaining slices multiplied and finished at once
        const int rw = min(32 * (swin - sa0), p.n_rows - 32 * sa0);
        const int rbase = 32 * sa0;
        for (int i0 = tid; i0 < rw; i0 += kU * kBlock) {
          S yo[kU];
#pragma unroll
          for (int k = 0; k < kU; ++k)
            if (i0 + k * kBlock < rw) yo[k] = ybuf[rbase + i0 + k * kBlock];
#pragma unroll
          for (int k = 0; k < kU; ++k)
            if (i0 + k * kBlock < rw)
              finish_row(rbase + i0 + k * kBlock, wbuf[i0 + k * kBlock], yo[k], false);
        }
        for (int k = ka0; k < ka1; ++k)
          if (__ldg(p.a_list + k) >= swin) multiply_finish(k, t == 1 ? cur : -1, t == 1);
        finish_x();
      }
      if (DF) {
        v[0] = df_to_double(sacc.value());
        v[1] = df_to_double(qacc.value());
      }
      block_sum_to0<2>(v, sh.scratch);
      if (tid == 0) {
        part[b * kPartSlots + 0] = v[0];
        part[b * kPartSlots + 1] = v[1];
        const long long now = globaltimer_ns();
        sh.busy_a += (unsigned long long)(now - sh.tmark - (t > 1 ? sh.twait : 0));
        if (sh.tendb) sh.lat_a += (unsigned long long)(now - sh.tendb);
        sh.cur = xb;
        if (t > 1) sh.iters_run = t - 1;
      }
    }
    const bool skip = (p.skip_arrival == t) && (b == 0);
    if (!grid_barrier(st, target, G, p.timeout_ns, skip, site++, sh.ok)) {
      status = PA_ERR_TIMEOUT;
      break;
    }
    // ---- scalar step: sums, scoring of x_{t-1}, gradient coefficients
    if (tid < 32) {
      const double s_ = ordered_sum(part, G, kPartSlots, 0);
      const double q = ordered_sum(part, G, kPartSlots, 1);
      double coef = 0.0;
      if (LOSS != PA_LOSS_QUADRATIC && lane < 2) coef = p.omb1 / (lane == 0 ? q : -s_);
      const double cb_lr = __shfl_sync(0xffffffffu, coef, 1);
      if (tid == 0) {
        int brk = 0;
        const int xc = sh.cur;
        if (!isfinite(s_) || !isfinite(q)) {
          sh.status = DF ? kStatusDfRange : PA_ERR_NONFINITE;
          brk = 1;
        } else if (DF && !(s_ >= 0x1.0p-100 && s_ <= 0x1.0p100)) {
          sh.status = kStatusDfRange;  // outside what the double-float variant covers
          brk = 1;
        } else {
          const double s_true = s_ * p.s_scale;
          if (t > 1) {  // score x_{t-1}
            bool better;
            if (LOSS == PA_LOSS_QUADRATIC) {
              const double L = loss_value2(p.mode, LOSS, s_true, q);
              better = !sh.have_best ||
                       L < loss_value2(p.mode, LOSS, sh.best_s * p.s_scale, sh.best_q);
            } else if (!sh.have_best) {
              better = p.mode == PA_SIGMA_MIN || s_ > 0.0;
            } else {
              better = p.mode == PA_SIGMA_MAX ? q * sh.best_s < sh.best_q * s_
                                              : s_ * sh.best_q < sh.best_s * q;
            }
            if (better) {
              sh.best_s = s_;
              sh.best_q = q;
              sh.have_best = 1;
              sh.t_min = t - 1;
              sh.minb = xc;
            }
            sh.last_s = s_;
            sh.last_q = q;
            sh.have_last = 1;
            if (p.L_trace && b == 0) p.L_trace[t - 2] = loss_value2(p.mode, LOSS, s_true, q);
          }
          if (s_ == 0.0) {
            if (p.mode == PA_SIGMA_MIN && t == 1) {
              sh.best_s = s_;
              sh.best_q = q;
              sh.have_best = 1;
              sh.t_min = 0;
              sh.minb = xc;
            }
            sh.status = PA_WARN_SINGULAR;
            brk = 1;
          } else if (t == p.iters + 1) {
            brk = 1;
          }
        }
        double ca, cb;
        if (LOSS == PA_LOSS_QUADRATIC) { ca = 0.0; cb = -2.0 * p.omb1; }
        else { ca = coef; cb = cb_lr; }
        if (p.mode == PA_SIGMA_MIN) { ca = -ca; cb = -cb; }
        sh.ca = ca;
        sh.cb = cb;
        if (DF && !brk) {
          sh.ca2 = df_from_double(ca);
          sh.cb2 = df_from_double(cb);
        }
        sh.q_keep = q;
        sh.brk = brk;
      }
    }
    __syncthreads();
    if (sh.brk) break;

    // ================= phase B(t): z, gradient, Adam, u_t, partials
    if (tid == 0) sh.tmark = globaltimer_ns();
    {
      const int xc = sh.cur;  // x_{t-1}
      if (r1 > r0) {  // the rows of x, m and v that the loop below reads
        const size_t nb8 = (size_t)(r1 - r0) * 8;
        prefetch_range_l2(DF ? (const void*)(X32(xc) + r0) : (const void*)(X64(xc) + r0), nb8);
        prefetch_range_l2(DF ? (const void*)(p.md + r0) : (const void*)(p.m + r0), nb8);
        prefetch_range_l2(DF ? (const void*)(p.vd + r0) : (const void*)(p.v + r0), nb8);
      }
      double v[2] = {0.0, 0.0};
      if constexpr (DF) {
        const df ca = sh.ca2, cb = sh.cb2, chat = sh.chat2;
        const float4 bq = p.bias2[p.t0 + t - 1];
        const df K1{bq.x, bq.y}, K2{bq.z, bq.w};
        DfAcc a1, a2;
        const float2* xs = X32(xc);
        const int kt0 = p.t_woff[b * (NW + 1) + warp], kt1 = p.t_woff[b * (NW + 1) + warp + 1];
        for (int k = kt0; k < kt1; ++k) {
          const int sl = __ldg(p.t_list + k);
          if (k + 1 < kt1) prefetch_slice_l2(p.t_wp, p.t_col, p.t_val2, __ldg(p.t_list + k + 1), lane);
          const int j = 32 * sl + lane;
          const df z = slice_dot_df(p.t_wp, p.t_col, p.t_val2, sl, lane, p.yd);
          if (j < n) {
            const df xj = df_load(xs + j);
            const df g = df_add(df_mul(ca, xj), df_mul(cb, z));
            const df mj = df_add(df_mul(b1d, df_load(p.md + j)), g);
            const df vj = df_add(df_mul(b2d, df_load(p.vd + j)), df_mul(w2d, df_mul(g, g)));
            df_store(p.md + j, mj);
            df_store(p.vd + j, vj);
            const df d = df_div(df_mul(K1, mj), df_add(df_sqrt(vj), K2));
            // u = (1 + c_hat) x - dx
            df_store(p.ud + j, df_add(df_sub(xj, d), df_mul(chat, xj)));
            a1.add_prod(xj, d);
            a2.add_prod(d, d);
          }
        }
        v[0] = df_to_double(a1.value());
        v[1] = df_to_double(a2.value());
      } else {
        const double ca = sh.ca, cb = sh.cb, chat = sh.chat;
        const double2 bc = p.bias[p.t0 + t - 1];
        const double b1 = p.beta1, b2 = p.beta2, w2 = p.w2;
        const double* xs = X64(xc);
        const int kt0 = p.t_woff[b * (NW + 1) + warp], kt1 = p.t_woff[b * (NW + 1) + warp + 1];
        for (int k = kt0; k < kt1; ++k) {
          const int sl = __ldg(p.t_list + k);
          if (k + 1 < kt1) prefetch_slice_l2(p.t_wp, p.t_col, p.t_val, __ldg(p.t_list + k + 1), lane);
          const int j = 32 * sl + lane;
          const double z = slice_dot(p.t_wp, p.t_col, p.t_val, sl, lane, p.y);
          if (j < n) {
            const double xj = xs[j], mo = p.m[j], vo = p.v[j];
            const double g = (LOSS == PA_LOSS_QUADRATIC) ? cb * z : fma(ca, xj, cb * z);
            const double mj = fma(b1, mo, g);
            const double vj = fma(b2, vo, w2 * (g * g));
            p.m[j] = mj;
            p.v[j] = vj;
            const double d = adam_quotient(bc.x * mj, vj, bc.y);
            p.u[j] = fma(chat, xj, xj - d);  // u = (1 + c_hat) x - dx
            v[0] = fma(xj, d, v[0]);
            v[1] = fma(d, d, v[1]);
          }
        }
      }
      block_sum_to0<2>(v, sh.scratch);  // its barriers order every u_t write of the CTA
      if (tid == 0) {
        part[b * kPartSlots + 2] = v[0];
        part[b * kPartSlots + 3] = v[1];
        const long long now = globaltimer_ns();
        sh.busy_b += (unsigned long long)(now - sh.tmark);
        sh.tendb = now;
        // "u_t written" for the neighbours, then the arrival on the split
        // barrier that the next phase A waits for
        publish_ready(p.ready + b, (unsigned)(2 * t));
        atomicAdd(&st->barrier, 1u);
      }
    }
  }

  if (tid == 0 && p.cta_ns) {
    p.cta_ns[2 * b] = sh.busy_a;
    p.cta_ns[2 * b + 1] = sh.busy_b;
  }
  if (tid == 0 && p.cta_lat) p.cta_lat[b] = sh.lat_a;
  if (b == 0 && tid == 0) {
    if (status == PA_ERR_TIMEOUT || ld_relaxed_u32(&st->abort) != 0u) sh.status = PA_ERR_TIMEOUT;
    st->status = sh.status;
    st->minb = sh.minb;
    st->cur = sh.cur;
    st->t_min = sh.t_min;
    st->L_min = sh.have_best
                    ? loss_value2(p.mode, LOSS, sh.best_s * p.s_scale, sh.best_q) : INFINITY;
    st->L_last = sh.have_last
                     ? loss_value2(p.mode, LOSS, sh.last_s * p.s_scale, sh.last_q) : NAN;
    st->iters_run = sh.iters_run;
    st->refreshes = sh.refreshes;
  }
}

// ---- double-float set-up and conversions

__device__ __forceinline__ int biased_exponent(double v) {
  return (int)((__double_as_longlong(v) >> 52) & 0x7ff);
}

__global__ void k_exp_range(int64_t n, const double* __restrict__ va, int* out) {
  int hi = INT_MIN, lo = INT_MAX;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double a = va[i];
    if (a != 0.0) {
      const int e = isfinite(a) ? biased_exponent(a) : 4096;  // non-finite: out of range
      hi = max(hi, e);
      lo = min(lo, e);
    }
  }
  for (int d = 16; d > 0; d >>= 1) {
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, d));
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, d));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, hi);
    atomicMin(out + 1, lo);
  }
}

// out[i] = (hi, lo) of in[i] * 2^-k (power-of-two scaling: exact)
__global__ void k_split_df(int64_t n, const double* __restrict__ in, double scale, float2* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const df d = df_from_double(in[i] * scale);
    out[i] = make_float2(d.hi, d.lo);
  }
}

__global__ void k_join_df(int64_t n, const float2* __restrict__ in, double* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = in[i];
    out[i] = (double)v.x + (double)v.y;
  }
}

int conv_blocks(int64_t n) { return (int)std::min<int64_t>(4096, (n + 255) / 256 + 1); }

}  // namespace

// The double-float variant runs two CTAs of 512 threads per SM (64
// registers, no spills): measured faster than one CTA per SM with its full
// register set (77.7 against 97.5 us per iteration on the 401 x 401
// operator), the memory latency of the products needing the warps.
static void* merged_fn(int loss, bool df) {
  if (df) return (void*)k_merged<PA_LOSS_LOGRATIO, true, 2>;
  return loss == PA_LOSS_QUADRATIC ? (void*)k_merged<PA_LOSS_QUADRATIC, false, kMinBlocksPerSM>
                                   : (void*)k_merged<PA_LOSS_LOGRATIO, false, kMinBlocksPerSM>;
}

// Shared memory for the speculative products: kMergedWin slices of 32
// values (FP64 or a double-float pair, 8 bytes each) = 64 KiB per CTA.
constexpr int kMergedWin = 256;
constexpr size_t kMergedSmem = (size_t)32 * 8 * kMergedWin;

static void* merged_fn_ready(int loss, bool df) {
  void* fn = merged_fn(loss, df);
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMergedSmem);
  return fn;
}

int merged_max_blocks(int loss, bool df) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, merged_fn_ready(loss, df), kBlock,
                                                    kMergedSmem) != cudaSuccess)
    return -1;
  return per * sms;
}

cudaError_t launch_merged(const IterParams& p, int loss, bool df, int G, cudaStream_t s,
                          int64_t* launches) {
  IterParams q = p;
  q.win_slices = kMergedWin;
  void* args[] = {(void*)&q};
  ++*launches;
  return cudaLaunchCooperativeKernel(merged_fn_ready(loss, df), dim3(G), dim3(kBlock), args,
                                     kMergedSmem, s);
}

cudaError_t launch_exp_range(int64_t n, const double* vals, int* out, cudaStream_t s,
                             int64_t* launches) {
  if (n <= 0) return cudaSuccess;
  k_exp_range<<<conv_blocks(n), 256, 0, s>>>(n, vals, out);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_split_df(int64_t n, const double* in, int k, float2* out, cudaStream_t s,
                            int64_t* launches) {
  if (n <= 0) return cudaSuccess;
  k_split_df<<<conv_blocks(n), 256, 0, s>>>(n, in, ldexp(1.0, -k), out);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_join_df(int64_t n, const float2* in, double* out, cudaStream_t s,
                           int64_t* launches) {
  if (n <= 0) return cudaSuccess;
  k_join_df<<<conv_blocks(n), 256, 0, s>>>(n, in, out);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace pa
