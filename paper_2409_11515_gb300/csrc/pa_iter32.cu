// pa_iter32.cu -- the mixed-precision sigma_max iteration: Algorithm 1 (the
// paper's Projected Adam with the gradient of Eq. nabla_loss) with FP32
// products and FP32 Adam state on the power-of-two-equilibrated matrix
// A_hat = D_r^-1 A D_c^-1 (the paper's "Row and Column Scaling"), while every
// norm that scales the gradient or the step (||y||^2, ||x||^2, x.dx, dx.dx) is
// reduced in FP64 across threads.
//
// With power-of-two D the products are exact rescalings of A's:
//   y = A x = D_r (A_hat (D_c x)),   z = A^T y = D_c (A_hat^T (D_r y)),
// so the kernel keeps w = D_c x (FP32) as the gather source of phase A, forms
// y_i = D_r,i u_i, and in phase B gathers (D_r,i lambda) y_i with a
// power-of-two lambda ~ 1/||y|| chosen after the barrier, which keeps every
// FP32 intermediate of both products within range.
//
// Structure (CTA ranges, ready flags, barriers with time limits, fixed-order
// reductions, three rotating iterate buffers) follows the FP64 kernel.
#include <math.h>

#include "pa_device.cuh"
#include "pa_internal.h"

namespace pa {

namespace {

struct Shared32 {
  double scratch[2 * kBlock];
  float ca, cbz;      // g' = ca x + cbz (D_c,j t_j)  (g' = (1 - beta1) g)
  float lam;          // power-of-two scale of phase B's gathered y
  float c, inv;       // projection coefficient, 1 / ||x'||
  int brk, cur, nb, ok;
  double best_s, best_q, last_s, last_q;  // best and latest scored (||y||^2, ||x||^2)
  int have_best, have_last;
  int minb, t_min, iters_run, status;
  unsigned long long busy_a, busy_b;
  long long tmark;
};

__device__ __forceinline__ float* pick32(const IterParams32& p, int k) {
  return k == 0 ? p.X0 : (k == 1 ? p.X1 : p.X2);
}

__device__ __forceinline__ float slice_dot32(const int32_t* __restrict__ wp,
                                             const int32_t* __restrict__ col,
                                             const float* __restrict__ val, int s, int lane,
                                             const float* x) {
  const int w0 = __ldg(wp + s), w = __ldg(wp + s + 1) - w0;
  const int64_t base = 32ll * w0 + lane;
  const int32_t* __restrict__ c = col + base;
  const float* __restrict__ v = val + base;
  float acc = 0.f;
  int k = 0;
  for (; k + 4 <= w; k += 4) {
    const int c0 = __ldg(c + 32 * k), c1 = __ldg(c + 32 * (k + 1)), c2 = __ldg(c + 32 * (k + 2)),
              c3 = __ldg(c + 32 * (k + 3));
    const float v0 = __ldg(v + 32 * k), v1 = __ldg(v + 32 * (k + 1)), v2 = __ldg(v + 32 * (k + 2)),
                v3 = __ldg(v + 32 * (k + 3));
    const float x0 = x[c0], x1 = x[c1], x2 = x[c2], x3 = x[c3];
    acc = fmaf(v0, x0, acc);
    acc = fmaf(v1, x1, acc);
    acc = fmaf(v2, x2, acc);
    acc = fmaf(v3, x3, acc);
  }
  for (; k < w; ++k) acc = fmaf(__ldg(v + 32 * k), x[__ldg(c + 32 * k)], acc);
  return acc;
}

// Transposed slice product with the gathered vector rescaled on the fly:
// sum_k val_k * ((d[i_k] * lam) * y[i_k]).
__device__ __forceinline__ float slice_dot32_scaled(const int32_t* __restrict__ wp,
                                                    const int32_t* __restrict__ col,
                                                    const float* __restrict__ val, int s,
                                                    int lane, const float* y,
                                                    const float* __restrict__ d, float lam) {
  const int w0 = __ldg(wp + s), w = __ldg(wp + s + 1) - w0;
  const int64_t base = 32ll * w0 + lane;
  const int32_t* __restrict__ c = col + base;
  const float* __restrict__ v = val + base;
  float acc = 0.f;
  int k = 0;
  for (; k + 4 <= w; k += 4) {  // all loads of four entries issued before any use
    const int i0 = __ldg(c + 32 * k), i1 = __ldg(c + 32 * (k + 1)), i2 = __ldg(c + 32 * (k + 2)),
              i3 = __ldg(c + 32 * (k + 3));
    const float v0 = __ldg(v + 32 * k), v1 = __ldg(v + 32 * (k + 1)), v2 = __ldg(v + 32 * (k + 2)),
                v3 = __ldg(v + 32 * (k + 3));
    const float d0 = __ldg(d + i0), d1 = __ldg(d + i1), d2 = __ldg(d + i2), d3 = __ldg(d + i3);
    const float y0 = y[i0], y1 = y[i1], y2 = y[i2], y3 = y[i3];
    acc = fmaf(v0, (d0 * lam) * y0, acc);
    acc = fmaf(v1, (d1 * lam) * y1, acc);
    acc = fmaf(v2, (d2 * lam) * y2, acc);
    acc = fmaf(v3, (d3 * lam) * y3, acc);
  }
  for (; k < w; ++k) {
    const int32_t i = __ldg(c + 32 * k);
    acc = fmaf(__ldg(v + 32 * k), (__ldg(d + i) * lam) * y[i], acc);
  }
  return acc;
}

__global__ void __launch_bounds__(kBlock, kMinBlocksPerSM) k_persistent32(const IterParams32 p) {
  __shared__ Shared32 sh;
  constexpr int NW = kBlock / 32;
  const unsigned G = gridDim.x;
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int sa0 = p.part_a[b], sa1 = p.part_a[b + 1];
  const int st0 = p.part_t[b], st1 = p.part_t[b + 1];
  const int n = p.n_cols;
  const int r0 = 32 * st0, r1 = min(32 * st1, n);
  const int dlo = p.dep[2 * b], dhi = p.dep[2 * b + 1];
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
    sh.have_last = 0;
    sh.busy_a = sh.busy_b = 0;
  }

  // w = D_c x_init and the ||x||^2 partial over the own rows; then publish
  Kahan32 qk;
  {
    const float* x = pick32(p, 0);
    for (int j = r0 + tid; j < r1; j += kBlock) {
      const float xj = x[j];
      p.W[j] = p.dc[j] * xj;
      qk.add(__fmul_rn(xj, xj));
    }
  }
  __syncthreads();
  if (tid == 0) publish_ready(p.ready + b, 1u);

  for (int t = 1;; ++t) {
    // w of the iterate to differentiate must be written by the neighbours
    if (!wait_ready(st, p.ready, dlo, dhi, (unsigned)t, p.timeout_ns, site++, sh.ok)) {
      status = PA_ERR_TIMEOUT;
      break;
    }
    if (tid == 0) sh.tmark = globaltimer_ns();
    // ---- phase A: y = D_r (A_hat w); ||y||^2 in FP64, ||x||^2 carried in
    {
      double v[2] = {0.0, qk.value()};
      for (int s = sa0 + warp; s < sa1; s += NW) {
        if (s + NW < sa1) prefetch_slice_l2(p.a_wp, p.a_col, p.a_val, s + NW, lane);
        const float u = slice_dot32(p.a_wp, p.a_col, p.a_val, s, lane, p.W);
        const int r = 32 * s + lane;
        if (r < p.n_rows) {
          const float yr = p.dr[r] * u;
          p.y[r] = yr;
          const double yd = (double)yr;
          v[0] = fma(yd, yd, v[0]);
        }
      }
      block_sum_to0<2>(v, sh.scratch);
      if (tid == 0) {
        part[b * kPartSlots + 0] = v[0];
        part[b * kPartSlots + 1] = v[1];
        sh.busy_a += (unsigned long long)(globaltimer_ns() - sh.tmark);
      }
    }
    const bool skip = (p.skip_arrival == t) && (b == 0);
    if (!grid_barrier(st, target, G, p.timeout_ns, skip, site++, sh.ok)) { status = PA_ERR_TIMEOUT; break; }
    double q_keep = 0.0;
    if (tid < 32) {
      const double s_ = ordered_sum(part, G, kPartSlots, 0);
      const double q = ordered_sum(part, G, kPartSlots, 1);
      // lambda = 2^-e with 2^(e-1) <= ||y|| < 2^e keeps (D_r,i lambda) y_i
      // within FP32 range; e from the exponent of ||y||^2 (no square root)
      int es;
      frexp(s_, &es);
      const double lam = ldexp(1.0, -((es + 1) >> 1));
      // lanes 0 and 1 run one division sequence for both gradient
      // coefficients: (1 - beta1) / q and, with z_j / s = D_c,j t_j /
      // (lambda s), -(1 - beta1) / (lambda s)
      double coef = 0.0;
      if (lane < 2) coef = p.omb1 / (lane == 0 ? q : -(lam * s_));
      const double cbz = __shfl_sync(0xffffffffu, coef, 1);
      if (tid == 0) {
        int brk = 0;
        const int cur = sh.cur;
        if (!isfinite(s_) || !isfinite(q)) {
          sh.status = PA_ERR_NONFINITE;
          brk = 1;
        } else {
          if (t > 1) {
            // L = log||x|| - log||y|| < L_min iff ||x||^2 ||y_b||^2 < ||x_b||^2 ||y||^2
            const bool better = sh.have_best ? q * sh.best_s < sh.best_q * s_ : s_ > 0.0;
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
            if (p.L_trace && b == 0) p.L_trace[t - 2] = log(sqrt(q)) - log(sqrt(s_));
          }
          if (s_ == 0.0) {
            sh.status = PA_WARN_SINGULAR;
            brk = 1;
          } else if (t == p.iters + 1) {
            brk = 1;
          }
        }
        if (!brk) {
          sh.lam = (float)lam;
          sh.ca = (float)coef;
          sh.cbz = (float)cbz;
        }
        q_keep = q;
        sh.brk = brk;
      }
    }
    __syncthreads();
    if (sh.brk) break;
    const float* x = pick32(p, sh.cur);

    // ---- phase B: z, gradient, FP32 Adam, x.dx and dx.dx
    if (tid == 0) sh.tmark = globaltimer_ns();
    {
      const float ca = sh.ca, cbz = sh.cbz, lam = sh.lam;
      const double2 bc = p.bias[t - 1];
      const float K1 = (float)bc.x, K2 = (float)bc.y;
      const float b1 = (float)p.beta1, b2 = (float)p.beta2;
      const float w2 = (float)p.w2;
      Kahan32 k1, k2;
      for (int s = st0 + warp; s < st1; s += NW) {
        if (s + NW < st1) prefetch_slice_l2(p.t_wp, p.t_col, p.t_val, s + NW, lane);
        const float tj = slice_dot32_scaled(p.t_wp, p.t_col, p.t_val, s, lane, p.y, p.dr, lam);
        const int j = 32 * s + lane;
        if (j < n) {
          const float xj = x[j];
          // D_c,j t_j = lambda z_j is bounded like z; scaling it last keeps
          // the product clear of FP32 underflow
          const float g = fmaf(ca, xj, cbz * (p.dc[j] * tj));
          const float mj = fmaf(b1, p.m[j], g);
          const float vj = fmaf(b2, p.v[j], w2 * (g * g));
          p.m[j] = mj;
          p.v[j] = vj;
          const float d = __fdiv_rn(K1 * mj, __fadd_rn(__fsqrt_rn(vj), K2));
          p.dx[j] = d;
          k1.add(__fmul_rn(xj, d));
          k2.add(__fmul_rn(d, d));
        }
      }
      double v[2] = {k1.value(), k2.value()};
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
          inv = rsqrt(nrm2);  // scales x only
        }
        sh.c = (float)c;
        sh.inv = (float)inv;
        const int cur = sh.cur, minb = sh.minb;
        sh.nb = (cur != 0 && minb != 0) ? 0 : ((cur != 1 && minb != 1) ? 1 : 2);
        sh.brk = brk;
      }
    }
    __syncthreads();
    if (sh.brk) break;

    // ---- phase C: x_t, w = D_c x_t, ||x_t||^2; publish
    if (tid == 0) sh.tmark = globaltimer_ns();
    {
      const float a1c = 1.f + sh.c, inv = sh.inv;
      const int nb = sh.nb;
      float* xo = pick32(p, nb);
      qk = Kahan32();
      for (int j = r0 + tid; j < r1; j += kBlock) {
        const float xn = fmaf(a1c, x[j], -p.dx[j]) * inv;
        xo[j] = xn;
        p.W[j] = p.dc[j] * xn;
        qk.add(__fmul_rn(xn, xn));
      }
      __syncthreads();
      if (tid == 0) {
        publish_ready(p.ready + b, (unsigned)(t + 1));
        sh.cur = nb;
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
    st->L_min = sh.have_best ? log(sqrt(sh.best_q)) - log(sqrt(sh.best_s)) : INFINITY;
    st->L_last = sh.have_last ? log(sqrt(sh.last_q)) - log(sqrt(sh.last_s)) : NAN;
    st->iters_run = sh.iters_run;
  }
}

}  // namespace

int persistent32_max_blocks(int* blocks_per_sm) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_persistent32, kBlock, 0) != cudaSuccess)
    return -1;
  if (blocks_per_sm) *blocks_per_sm = per;
  return per * sms;
}

cudaError_t launch_persistent32(const IterParams32& p, int G, cudaStream_t s, int64_t* launches) {
  void* args[] = {(void*)&p};
  cudaError_t e = cudaLaunchCooperativeKernel((void*)k_persistent32, dim3(G), dim3(kBlock), args,
                                              0, s);
  ++*launches;
  return e;
}

}  // namespace pa
