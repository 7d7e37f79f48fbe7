// pa_iter_sp.cu -- the single-pass engine: Algorithm 1 with the gradient of
// Eq. nabla_loss, reading A once per iteration and keeping no transposed copy.
//
// Eq. nabla_loss needs y = A x and z = A^T y.  CTA b owns a contiguous block
// of rows of P A Q^T (slices [part[b], part[b+1])) and the same range of x
// positions.  The rows of a banded operator touch a window of columns around
// that range, and the host keeps, per CTA, a plan of the window: for each
// window column the block's entries in that column, in row order, as
// (row - first row of the block) << 8 | slot of the entry in its row.  The
// plan holds no values (4 bytes per entry against 12 for a transposed copy).
// Per iteration t:
//
//   A  y = A x_{t-1} over the own rows (values read from HBM once), partials
//      s = ||y||^2 and q = ||x||^2; after a block barrier, one thread per
//      window column sums a_ij y_i over the column's plan entries in row
//      order (the values come back from L2, the y_i are the block's own)
//      into the CTA's halo slot for that column               | grid barrier
//      every CTA sums the partials in the same fixed order; L(x_{t-1}) is
//      scored as in the three-phase kernel
//   B  z_j for the own positions: the halo slots of every CTA whose window
//      holds j, added in CTA order; then g = a x + b z, Adam's moments and
//      step dx, partials x.dx and dx.dx                       | grid barrier
//   C  x_t = ((1 + p1) x - dx) / ||.||; publish the ready flag; the next
//      phase A waits for the flags of the CTAs owning its window's columns.
//
// Every sum has a fixed order (rows ascending inside a CTA's window column,
// CTAs ascending across the halo), so runs are bit-reproducible.
#include <math.h>

#include "pa_device.cuh"
#include "pa_internal.h"

namespace pa {

namespace {

struct SharedSP {
  double scratch[2 * kBlock];
  double ca, cb;      // g = ca * x + cb * z
  double c, inv;      // 1 + the projection coefficient, and 1 / ||x'||
  int brk;
  int cur, nb;        // buffer of x_{t-1}, buffer for x_t
  int ok;
  double best_s, best_q, last_s, last_q;  // Algorithm 1's tracking (thread 0)
  int have_best, have_last;
  int minb, t_min, iters_run, status;
  unsigned long long busy_a, busy_b;
  long long tmark;
};

__device__ __forceinline__ double* pick_sp(const IterParams& p, int k) {
  return k == 0 ? p.X0 : (k == 1 ? p.X1 : p.X2);
}

__device__ __forceinline__ double loss_sp(int mode, int loss, double s, double q) {
  if (loss == PA_LOSS_QUADRATIC) return mode == PA_SIGMA_MAX ? -s : s;
  const double lx = log(sqrt(q)), lax = log(sqrt(s));
  return mode == PA_SIGMA_MAX ? lx - lax : lax - lx;
}

// Prefetch [base, base + bytes) into L2, one 128-byte line per thread per step.
__device__ __forceinline__ void prefetch_l2(const void* base, size_t bytes) {
  const char* c = static_cast<const char*>(base);
  for (size_t off = 128 * (size_t)threadIdx.x; off < bytes; off += 128 * (size_t)blockDim.x)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(c + off));
}

// One plan slot: the entry's value and its row's y (both 0 for padding).
__device__ __forceinline__ void plan_slot(const IterParams& p, const int32_t* __restrict__ wpb,
                                          const double* y, int row0, uint32_t ent, double& a,
                                          double& yi) {
  a = yi = 0.0;
  if (ent != kPlanPad) {
    const int rl = (int)(ent >> 8);
    a = __ldg(p.a_val + 32ll * (__ldg(wpb + (rl >> 5)) + (int)(ent & 255u)) + (rl & 31));
    yi = y[row0 + rl];
  }
}

// CTA b's share of z = A^T y over its column window.  Warp w takes the
// CTA's plan groups in pairs (w, w + NW), (w + 2 NW, w + 3 NW), ...; lane l
// sums its column's entries in row order, one fused multiply-add each
// (groups hold columns of equal or nearly equal entry counts, so the warp's
// lanes stay busy).  The two groups' loads are issued together, two slots
// each, before their multiply-adds.  y holds the block's rows.
__device__ __forceinline__ void window_products(const IterParams& p, int b, int sa0,
                                                const double* y) {
  const int NW = blockDim.x >> 5, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g0 = p.sp_goff[b], g1 = p.sp_goff[b + 1];
  const int hbase = p.sp_woff[b], row0 = 32 * sa0;
  const int32_t* __restrict__ wpb = p.a_wp + sa0;
  for (int g = g0 + warp; g < g1; g += 2 * NW) {
    const int h = g + NW;
    const bool two = h < g1;
    const int ka = __ldg(p.sp_gp + g), wa = __ldg(p.sp_gp + g + 1) - ka;
    const int kb = two ? __ldg(p.sp_gp + h) : 0, wb = two ? __ldg(p.sp_gp + h + 1) - kb : 0;
    const uint32_t* __restrict__ ea = p.sp_ent + 32ll * ka + lane;
    const uint32_t* __restrict__ eb = p.sp_ent + 32ll * kb + lane;
    double acc_a = 0.0, acc_b = 0.0;
    const int wm = max(wa, wb);
    for (int k = 0; k < wm; k += 2) {
      double a[4], yi[4];
      const uint32_t n0 = k < wa ? __ldg(ea + 32 * k) : kPlanPad;
      const uint32_t n1 = k + 1 < wa ? __ldg(ea + 32 * (k + 1)) : kPlanPad;
      const uint32_t n2 = k < wb ? __ldg(eb + 32 * k) : kPlanPad;
      const uint32_t n3 = k + 1 < wb ? __ldg(eb + 32 * (k + 1)) : kPlanPad;
      plan_slot(p, wpb, y, row0, n0, a[0], yi[0]);
      plan_slot(p, wpb, y, row0, n1, a[1], yi[1]);
      plan_slot(p, wpb, y, row0, n2, a[2], yi[2]);
      plan_slot(p, wpb, y, row0, n3, a[3], yi[3]);
      if (k < wa) acc_a = fma(a[0], yi[0], acc_a);
      if (k + 1 < wa) acc_a = fma(a[1], yi[1], acc_a);
      if (k < wb) acc_b = fma(a[2], yi[2], acc_b);
      if (k + 1 < wb) acc_b = fma(a[3], yi[3], acc_b);
    }
    const int ca = __ldg(p.sp_gcol + 32 * g + lane);
    if (ca >= 0) p.sp_halo[hbase + ca] = acc_a;
    if (two) {
      const int cb = __ldg(p.sp_gcol + 32 * h + lane);
      if (cb >= 0) p.sp_halo[hbase + cb] = acc_b;
    }
  }
}

// The CTA's plan slots and group columns into L2 (issued before its
// products, so the window pass finds them there).
__device__ __forceinline__ void prefetch_plan(const IterParams& p, int b) {
  const int g0 = p.sp_goff[b], g1 = p.sp_goff[b + 1];
  const int64_t s0 = 32ll * __ldg(p.sp_gp + g0), s1 = 32ll * __ldg(p.sp_gp + g1);
  prefetch_l2(p.sp_ent + s0, sizeof(uint32_t) * (size_t)(s1 - s0));
  prefetch_l2(p.sp_gcol + 32ll * g0, sizeof(int32_t) * 32 * (size_t)(g1 - g0));
}

// z_j of an own position: the halo slots of CTAs [lo, hi] whose windows hold
// j, in CTA order.
__device__ __forceinline__ double halo_sum(const IterParams& p, int lo, int hi, int j) {
  double z = 0.0;
  for (int c = lo; c <= hi; ++c) {
    const int o0 = __ldg(p.sp_woff + c), w = j - __ldg(p.sp_cmin + c);
    if (w >= 0 && w < __ldg(p.sp_woff + c + 1) - o0) z += p.sp_halo[o0 + w];
  }
  return z;
}

template <int LOSS>
__global__ void __launch_bounds__(kBlock, kMinBlocksPerSM) k_single(const IterParams p) {
  __shared__ SharedSP sh;
  constexpr int NW = kBlock / 32;
  const unsigned G = gridDim.x;
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int sa0 = p.part_a[b], sa1 = p.part_a[b + 1];
  const int n = p.n_cols;
  const int c0 = min(32 * sa0, n), c1 = min(32 * sa1, n);  // own x positions
  RunState* st = p.st;
  double* __restrict__ part = p.partials;
  unsigned target = 0;
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
    sh.best_s = sh.best_q = 0.0;
    sh.have_last = 0;
    sh.busy_a = sh.busy_b = 0;
  }
  const int dlo = p.dep[2 * b], dhi = p.dep[2 * b + 1];
  const int rlo = p.sp_rdep[2 * b], rhi = p.sp_rdep[2 * b + 1];
  __syncthreads();  // sh.cur is read by every thread at t = 1

  double qloc = 0.0;
  {
    const double* x = pick_sp(p, 0);
    for (int j = c0 + tid; j < c1; j += kBlock) qloc = fma(x[j], x[j], qloc);
  }

  for (int t = 1;; ++t) {
    if (t > 1 && !wait_ready(st, p.ready, dlo, dhi, (unsigned)(t - 1), p.timeout_ns, site++, sh.ok)) {
      status = PA_ERR_TIMEOUT;
      break;
    }
    const double* x = pick_sp(p, sh.cur);
    if (tid == 0) sh.tmark = globaltimer_ns();
    // ---- phase A: y = A x (own rows), the window's share of A^T y
    {
      double v[2] = {0.0, qloc};
      prefetch_plan(p, b);
      const int k0 = p.a_woff[b * (NW + 1) + warp], k1 = p.a_woff[b * (NW + 1) + warp + 1];
      for (int k = k0; k < k1; ++k) {
        const int s = __ldg(p.a_list + k);
        if (k + 1 < k1) prefetch_slice_l2(p.a_wp, p.a_col, p.a_val, __ldg(p.a_list + k + 1), lane);
        const int r = 32 * s + lane;
        const double yr = slice_dot(p.a_wp, p.a_col, p.a_val, s, lane, x);
        if (r < p.n_rows) {  // rows past the end have no entries in the plan
          p.y[r] = yr;
          v[0] = fma(yr, yr, v[0]);
        }
      }
      __syncthreads();  // every y row of the block is written
      window_products(p, b, sa0, p.y);
      block_sum_to0<2>(v, sh.scratch);
      if (tid == 0) {
        part[b * kPartSlots + 0] = v[0];
        part[b * kPartSlots + 1] = v[1];
        sh.busy_a += (unsigned long long)(globaltimer_ns() - sh.tmark);
      }
    }
    if (!grid_barrier(st, target, G, p.timeout_ns, false, site++, sh.ok)) { status = PA_ERR_TIMEOUT; break; }
    if (tid < 32) {
      const double s_ = ordered_sum(part, G, kPartSlots, 0);
      const double q = ordered_sum(part, G, kPartSlots, 1);
      double coef = 0.0;
      if (LOSS != PA_LOSS_QUADRATIC && lane < 2) coef = p.omb1 / (lane == 0 ? q : -s_);
      const double cb_lr = __shfl_sync(0xffffffffu, coef, 1);
      if (tid == 0) {
        int brk = 0;
        const int cur = sh.cur;
        if (!isfinite(s_) || !isfinite(q)) {
          sh.status = PA_ERR_NONFINITE;
          brk = 1;
        } else {
          if (t > 1) {  // score x_{t-1}: L < L_min through the monotone map of the loss
            bool better;
            if (LOSS == PA_LOSS_QUADRATIC) {
              const double L = loss_sp(p.mode, LOSS, s_, q);
              better = !sh.have_best || L < loss_sp(p.mode, LOSS, sh.best_s, sh.best_q);
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
              sh.minb = cur;
            }
            sh.last_s = s_;
            sh.last_q = q;
            sh.have_last = 1;
            if (p.L_trace && b == 0) p.L_trace[t - 2] = loss_sp(p.mode, LOSS, s_, q);
          }
          if (s_ == 0.0) {
            if (p.mode == PA_SIGMA_MIN && t == 1) {  // x_init itself is a null vector
              sh.best_s = s_;
              sh.best_q = q;
              sh.have_best = 1;
              sh.t_min = 0;
              sh.minb = cur;
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
        sh.scratch[0] = q;
        sh.brk = brk;
      }
    }
    __syncthreads();
    if (sh.brk) break;
    const double q_keep = (tid == 0) ? sh.scratch[0] : 0.0;

    // ---- phase B: z from the halo, gradient, Adam, partials x.dx and dx.dx
    if (tid == 0) sh.tmark = globaltimer_ns();
    {
      const double ca = sh.ca, cb = sh.cb;
      const double2 bc = p.bias[p.t0 + t - 1];
      const double b1 = p.beta1, b2 = p.beta2, w2 = p.w2;
      double v[2] = {0.0, 0.0};
      for (int j = c0 + tid; j < c1; j += kBlock) {
        const double z = halo_sum(p, rlo, rhi, j);
        const double xj = x[j];
        const double g = (LOSS == PA_LOSS_QUADRATIC) ? cb * z : fma(ca, xj, cb * z);
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
        part[b * kPartSlots + 2] = v[0];
        part[b * kPartSlots + 3] = v[1];
        sh.busy_b += (unsigned long long)(globaltimer_ns() - sh.tmark);
      }
    }
    if (!grid_barrier(st, target, G, p.timeout_ns, false, site++, sh.ok)) { status = PA_ERR_TIMEOUT; break; }
    if (tid < 32) {
      const double p1 = ordered_sum(part, G, kPartSlots, 2);
      const double p2 = ordered_sum(part, G, kPartSlots, 3);
      if (tid == 0) {
        int brk = 0;
        if (!isfinite(p1) || !isfinite(p2)) {
          sh.status = PA_ERR_NONFINITE;
          brk = 1;
        }
        const double c = (p.ablation & PA_ABLATE_NO_TANGENT) ? 0.0 : p1;
        double inv = 1.0;
        if (!(p.ablation & PA_ABLATE_NO_NORMALISE)) {
          const double a1c = 1.0 + c;
          const double nrm2 = fma(a1c * a1c, q_keep, fma(-2.0 * a1c, p1, p2));
          inv = rsqrt(nrm2);
        }
        sh.c = 1.0 + c;
        sh.inv = inv;
        const int cur = sh.cur, minb = sh.minb;
        sh.nb = (cur != 0 && minb != 0) ? 0 : ((cur != 1 && minb != 1) ? 1 : 2);
        sh.brk = brk;
      }
    }
    __syncthreads();
    if (sh.brk) break;

    // ---- phase C: project, update, normalise; partial ||x_t||^2
    if (tid == 0) sh.tmark = globaltimer_ns();
    {
      const double a1c = sh.c, inv = sh.inv;
      double* xo = pick_sp(p, sh.nb);
      double* tr = (p.x_trace && t <= p.n_trace) ? p.x_trace + (size_t)(t - 1) * n : nullptr;
      qloc = 0.0;
      for (int j = c0 + tid; j < c1; j += kBlock) {
        const double xn = fma(a1c, x[j], -p.dx[j]) * inv;
        xo[j] = xn;
        if (tr) tr[j] = xn;
        qloc = fma(xn, xn, qloc);
      }
      __syncthreads();  // every x_t position of this CTA is written
      if (tid == 0) {
        publish_ready(p.ready + b, (unsigned)t);
        sh.cur = sh.nb;
        sh.iters_run = t;
        sh.busy_b += (unsigned long long)(globaltimer_ns() - sh.tmark);
      }
      __syncthreads();
    }
  }

  if (tid == 0 && p.cta_ns) {
    p.cta_ns[2 * b] = sh.busy_a;
    p.cta_ns[2 * b + 1] = sh.busy_b;
  }
  if (b == 0 && tid == 0) {
    if (status == PA_ERR_TIMEOUT || ld_relaxed_u32(&st->abort) != 0u) sh.status = PA_ERR_TIMEOUT;
    st->status = sh.status;
    st->minb = sh.minb;
    st->cur = sh.cur;
    st->t_min = sh.t_min;
    st->L_min = sh.have_best ? loss_sp(p.mode, LOSS, sh.best_s, sh.best_q) : INFINITY;
    st->L_last = sh.have_last ? loss_sp(p.mode, LOSS, sh.last_s, sh.last_q) : NAN;
    st->iters_run = sh.iters_run;
    st->best_s = sh.best_s;
    st->best_q = sh.best_q;
    st->have_best = sh.have_best;
  }
}

// One product z = A^T (A x) through the same plan, outside the iteration:
// y over the own rows and the window sums (k_single_rows), then each own
// position adds the halo slots (k_single_cols).
__global__ void __launch_bounds__(kBlock) k_single_rows(const IterParams p, const double* x) {
  constexpr int NW = kBlock / 32;
  const int b = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sa0 = p.part_a[b], sa1 = p.part_a[b + 1];
  for (int s = sa0 + warp; s < sa1; s += NW) {
    const int r = 32 * s + lane;
    const double yr = slice_dot(p.a_wp, p.a_col, p.a_val, s, lane, x);
    if (r < p.n_rows) p.y[r] = yr;
  }
  __syncthreads();
  window_products(p, b, sa0, p.y);
}

__global__ void __launch_bounds__(kBlock) k_single_cols(const IterParams p, double* z) {
  const int b = blockIdx.x;
  const int n = p.n_cols;
  const int c0 = min(32 * p.part_a[b], n), c1 = min(32 * p.part_a[b + 1], n);
  const int lo = p.sp_rdep[2 * b], hi = p.sp_rdep[2 * b + 1];
  for (int j = c0 + (int)threadIdx.x; j < c1; j += blockDim.x) z[j] = halo_sum(p, lo, hi, j);
}

}  // namespace

static void* single_fn(int loss) {
  return loss == PA_LOSS_QUADRATIC ? (void*)k_single<PA_LOSS_QUADRATIC>
                                   : (void*)k_single<PA_LOSS_LOGRATIO>;
}

int single_max_blocks(int loss) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, single_fn(loss), kBlock, 0) != cudaSuccess)
    return -1;
  return per * sms;
}

cudaError_t launch_single(const IterParams& p, int loss, int G, cudaStream_t s, int64_t* launches) {
  void* args[] = {(void*)&p};
  ++*launches;
  return cudaLaunchCooperativeKernel(single_fn(loss), dim3(G), dim3(kBlock), args, 0, s);
}

cudaError_t launch_single_product(const IterParams& p, int G, const double* x, double* z,
                                  cudaStream_t s, int64_t* launches) {
  k_single_rows<<<G, kBlock, 0, s>>>(p, x);
  k_single_cols<<<G, kBlock, 0, s>>>(p, z);
  *launches += 2;
  return cudaGetLastError();
}

}  // namespace pa
