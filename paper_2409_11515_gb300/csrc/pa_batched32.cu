// pa_batched32.cu -- the mixed-precision sigma_max stage of a batch: for
// every (matrix, restart) item, Algorithm 1 of the paper (gradient
// Eq. nabla_loss) with FP32 products and FP32 Adam state on the
// power-of-two-equilibrated matrix A_hat = D_r^-1 A D_c^-1 (the paper's "Row
// and Column Scaling"), the K restarts of a matrix advancing together as an
// n x K block (SpMM), while every norm that scales the gradient or the step
// (||y||^2, ||x||^2, x.dx, dx.dx) is reduced in FP64.
//
// The arithmetic per column is that of the single-vector FP32 kernel: the
// gather source of phase A is w = D_c x, y_i = D_r,i (A_hat w)_i, and phase B
// gathers (D_r,i lambda_c) y_i with a power-of-two lambda_c ~ 1 / ||y_c||, so
// every FP32 intermediate stays in range.  The CTA groups, partitions, group
// barriers, fixed-order reductions and per-column tracking are those of the
// FP64 batched kernel, so each column is bit-reproducible.  The caller
// continues from the FP32 state in FP64 (k_batched with t0) for the last
// iterations.
#include <math.h>

#include "pa_device.cuh"
#include "pa_internal.h"

namespace pa {

namespace {

constexpr int kBT32 = 256;  // threads per CTA (the FP64 batched kernel's)

template <int K>
struct SharedB32 {
  double part[2][K][kBT32];  // per-thread partials, two quantities per phase
  float ca[K], cbz[K];       // g' = ca x + cbz (D_c,j t_j), per column
  float lam[K];              // power-of-two scale of phase B's gathered y
  float c[K], inv[K];        // projection coefficient, 1 / ||x'||
  double q[K];               // ||x_{t-1}||^2
  double best_s[K], best_q[K], last_s[K], last_q[K];
  int have_best[K], have_last[K];
  int t_min[K], improved[K];
  int brk, ok, status;
  int iters_run;
};

template <int K>
__global__ void __launch_bounds__(kBT32, 2) k_batched32(const BatchParams bp) {
  __shared__ SharedB32<K> sh;
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = kBT32 / 32;
  const int item = bp.cta_item[b];
  const BatchItem& it = bp.items[item];
  const int lb = b - it.cta0;
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
  int cur = 0;
  if (tid == 0) {
    sh.brk = 0;
    sh.status = PA_OK;
    sh.iters_run = 0;
  }
  // w = D_c x_init and ||x_init||^2 per column over the own rows; the other
  // CTAs' w is read in phase A, hence the group barrier
  {
    Kahan32 qk[K];
    for (int j = r0 + tid; j < r1; j += kBT32) {
      const float dcj = it.dc32[j];
#pragma unroll
      for (int c = 0; c < K; ++c) {
        const size_t o = (size_t)j * K + c;
        const float xj = it.X0f[o];
        it.Wf[o] = dcj * xj;
        qk[c].add(__fmul_rn(xj, xj));
      }
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < K; ++c) sh.part[1][c][tid] = qk[c].value();
  }
  if (!group_barrier(counter, target, G, st, bp.timeout_ns, sh.ok)) status = PA_ERR_TIMEOUT;

  for (int t = 1; status == PA_OK; ++t) {
    const float* x = cur == 0 ? it.X0f : it.X1f;
    // ---- phase A: Y = D_r (A_hat W), ||y_c||^2 in FP64 (||x||^2 partials in slot 1)
    {
      double sv[K];
#pragma unroll
      for (int c = 0; c < K; ++c) sv[c] = 0.0;
      for (int s = sa0 + warp; s < sa1; s += NW) {
        if (s + NW < sa1) prefetch_slice_l2(it.a_wp, it.a_col, it.a_val32, s + NW, lane);
        const int w0 = __ldg(it.a_wp + s), w = __ldg(it.a_wp + s + 1) - w0;
        const int64_t base = 32ll * w0 + lane;
        float acc[K];
#pragma unroll
        for (int c = 0; c < K; ++c) acc[c] = 0.f;
        for (int k = 0; k < w; ++k) {
          const float a = __ldg(it.a_val32 + base + 32ll * k);
          const float* wr = it.Wf + (size_t)__ldg(it.a_col + base + 32ll * k) * K;
#pragma unroll
          for (int c = 0; c < K; ++c) acc[c] = fmaf(a, wr[c], acc[c]);
        }
        const int r = 32 * s + lane;
        if (r < it.n_rows) {
          const float dr = it.dr32[r];
#pragma unroll
          for (int c = 0; c < K; ++c) {
            const float yr = dr * acc[c];
            it.Yf[(size_t)r * K + c] = yr;
            const double yd = (double)yr;
            sv[c] = fma(yd, yd, sv[c]);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < K; ++c) sh.part[0][c][tid] = sv[c];
      __syncthreads();
      for (int c = warp; c < K; c += NW) {
        const double a0 = slot_sum(sh.part[0][c], kBT32);
        const double a1 = slot_sum(sh.part[1][c], kBT32);
        if (lane == 0) {
          part[((size_t)lb * 4 + 0) * K + c] = a0;
          part[((size_t)lb * 4 + 1) * K + c] = a1;
        }
      }
    }
    if (!group_barrier(counter, target, G, st, bp.timeout_ns, sh.ok)) { status = PA_ERR_TIMEOUT; break; }
    // ---- per-column scalars: score x_{t-1}, lambda_c, gradient coefficients
    for (int c = warp; c < K; c += NW) {
      const double s_ = ordered_sum(part, G, 4 * K, c);
      const double q = ordered_sum(part, G, 4 * K, K + c);
      if (lane == 0) {
        int imp = 0;
        if (!isfinite(s_) || !isfinite(q)) {
          atomicExch(&sh.status, PA_ERR_NONFINITE);
        } else if (t > 1) {
          // log||x|| - log||y|| < L_min iff ||x||^2 ||y_b||^2 < ||x_b||^2 ||y||^2
          const bool better = sh.have_best[c] ? q * sh.best_s[c] < sh.best_q[c] * s_ : s_ > 0.0;
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
        // lambda = 2^-e with 2^(e-1) <= ||y|| < 2^e, from the exponent of ||y||^2
        int es;
        frexp(s_, &es);
        const double lam = ldexp(1.0, -((es + 1) >> 1));
        const double omb1 = 1.0 - bp.beta1;
        sh.lam[c] = (float)lam;
        sh.ca[c] = (float)(omb1 / q);
        sh.cbz[c] = (float)(-omb1 / (lam * s_));
        sh.q[c] = q;
      }
    }
    __syncthreads();
    if (tid == 0) sh.brk = (sh.status != PA_OK) || (t == bp.iters + 1);
    __syncthreads();
    if (sh.brk) {
      if (sh.status == PA_OK || sh.status == PA_WARN_SINGULAR) {
        for (int j = r0 + tid; j < r1; j += kBT32)
#pragma unroll
          for (int c = 0; c < K; ++c)
            if (sh.improved[c]) it.XMINf[(size_t)j * K + c] = x[(size_t)j * K + c];
      }
      break;
    }

    // ---- phase B: T = A_hat^T ((D_r lambda) Y), gradient, FP32 Adam, x.dx, dx.dx
    {
      const double2 bc = bp.bias[bp.t0 + t - 1];
      const float K1 = (float)bc.x, K2 = (float)bc.y;
      const float b1 = (float)bp.beta1, b2 = (float)bp.beta2, w2 = (float)bp.w2;
      float lam[K], ca[K], cbz[K];
#pragma unroll
      for (int c = 0; c < K; ++c) {
        lam[c] = sh.lam[c];
        ca[c] = sh.ca[c];
        cbz[c] = sh.cbz[c];
      }
      Kahan32 k1[K], k2[K];
      for (int s = st0 + warp; s < st1; s += NW) {
        if (s + NW < st1) prefetch_slice_l2(it.t_wp, it.t_col, it.t_val32, s + NW, lane);
        const int w0 = __ldg(it.t_wp + s), w = __ldg(it.t_wp + s + 1) - w0;
        const int64_t base = 32ll * w0 + lane;
        float tz[K];
#pragma unroll
        for (int c = 0; c < K; ++c) tz[c] = 0.f;
        for (int k = 0; k < w; ++k) {
          const float a = __ldg(it.t_val32 + base + 32ll * k);
          const int32_t i = __ldg(it.t_col + base + 32ll * k);
          const float di = __ldg(it.dr32 + i);
          const float* yr = it.Yf + (size_t)i * K;
#pragma unroll
          for (int c = 0; c < K; ++c) tz[c] = fmaf(a, (di * lam[c]) * yr[c], tz[c]);
        }
        const int j = 32 * s + lane;
        if (j < n) {
          const float dcj = it.dc32[j];
#pragma unroll
          for (int c = 0; c < K; ++c) {
            const size_t o = (size_t)j * K + c;
            const float xj = x[o];
            if (sh.improved[c]) it.XMINf[o] = xj;
            // D_c,j t_j = lambda z_j is bounded like z; scaled last
            const float g = fmaf(ca[c], xj, cbz[c] * (dcj * tz[c]));
            const float mj = fmaf(b1, it.Mf[o], g);
            const float vj = fmaf(b2, it.Vf[o], w2 * (g * g));
            it.Mf[o] = mj;
            it.Vf[o] = vj;
            const float d = __fdiv_rn(K1 * mj, __fadd_rn(__fsqrt_rn(vj), K2));
            it.DXf[o] = d;
            k1[c].add(__fmul_rn(xj, d));
            k2[c].add(__fmul_rn(d, d));
          }
        }
      }
#pragma unroll
      for (int c = 0; c < K; ++c) {
        sh.part[0][c][tid] = k1[c].value();
        sh.part[1][c][tid] = k2[c].value();
      }
      __syncthreads();
      for (int c = warp; c < K; c += NW) {
        const double a0 = slot_sum(sh.part[0][c], kBT32);
        const double a1 = slot_sum(sh.part[1][c], kBT32);
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
          inv = rsqrt(fma(a1c * a1c, sh.q[c], fma(-2.0 * a1c, p1, p2)));  // scales x only
        }
        sh.c[c] = (float)cc;
        sh.inv[c] = (float)inv;
      }
    }
    __syncthreads();
    if (sh.status != PA_OK && sh.status != PA_WARN_SINGULAR) break;

    // ---- phase C: x_t, w = D_c x_t, ||x_t||^2 partials (slot 1 of phase A)
    {
      float* xo = cur == 0 ? it.X1f : it.X0f;
      float a1c[K], inv[K];
#pragma unroll
      for (int c = 0; c < K; ++c) {
        a1c[c] = 1.f + sh.c[c];
        inv[c] = sh.inv[c];
      }
      Kahan32 qk[K];
      for (int j = r0 + tid; j < r1; j += kBT32) {
        const float dcj = it.dc32[j];
#pragma unroll
        for (int c = 0; c < K; ++c) {
          const size_t o = (size_t)j * K + c;
          const float xn = fmaf(a1c[c], x[o], -it.DXf[o]) * inv[c];
          xo[o] = xn;
          it.Wf[o] = dcj * xn;
          qk[c].add(__fmul_rn(xn, xn));
        }
      }
#pragma unroll
      for (int c = 0; c < K; ++c) sh.part[1][c][tid] = qk[c].value();
      cur ^= 1;
      if (tid == 0) sh.iters_run = t;
    }
    if (!group_barrier(counter, target, G, st, bp.timeout_ns, sh.ok)) { status = PA_ERR_TIMEOUT; break; }
  }

  // results of the group, written by its first CTA (log-ratio sigma_max)
  if (lb == 0 && tid < K) {
    double* out = it.result + (size_t)tid * 4;
    out[0] = sh.have_best[tid] ? log(sqrt(sh.best_q[tid])) - log(sqrt(sh.best_s[tid])) : INFINITY;
    out[1] = sh.t_min[tid];
    out[2] = sh.have_last[tid] ? log(sqrt(sh.last_q[tid])) - log(sqrt(sh.last_s[tid])) : NAN;
    out[3] = sh.iters_run;
  }
  if (lb == 0 && tid == 0) {
    int s = sh.status;
    if (status == PA_ERR_TIMEOUT || ld_relaxed_u32(&st->abort) != 0u) s = PA_ERR_TIMEOUT;
    it.status[0] = s;
  }
}

void* batched32_fn(int k) {
  switch (k) {
    case 1: return (void*)k_batched32<1>;
    case 2: return (void*)k_batched32<2>;
    case 4: return (void*)k_batched32<4>;
    case 8: return (void*)k_batched32<8>;
    default: return nullptr;
  }
}

}  // namespace

int batched32_max_blocks(int k) {
  void* fn = batched32_fn(k);
  if (!fn) return -1;
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kBT32, 0) != cudaSuccess) return -1;
  return per * sms;
}

cudaError_t launch_batched32(const BatchParams& p, int k, int G, cudaStream_t s, int64_t* launches) {
  void* fn = batched32_fn(k);
  if (!fn) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(kBT32);
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
