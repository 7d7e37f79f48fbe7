// pa_iter.cu -- the persistent cooperative Projected Adam kernel (the paper's
// Algorithm 1 with the gradient of Eq. nabla_loss) for one vector.
//
// One launch runs every iteration without returning to the host.  CTA b owns
// a contiguous block of rows of A (phase A) and of A^T (phases B and C); the
// blocks are balanced by non-zeros.  Per iteration t:
//
//   A  y = A x_{t-1} (own rows); partial s = sum y_i^2         | grid barrier
//      every CTA sums the partials in the same fixed order -> s, q = ||x||^2;
//      L(x_{t-1}) is scored against L_min (Algorithm 1's tracking, lagged by
//      one product so that y serves both the score and the gradient).
//   B  z = A^T y over the explicit CSR of A^T (own rows), the gradient
//      g = a x + b z, Adam's moments and step dx (kept in `dx`), partials
//      p1 = x.dx, p2 = dx.dx                                  | grid barrier
//   C  x_t = ((1 + p1) x - dx) / ||.||, the tangent projection and the
//      normalisation of Algorithm 1 in one pass; ||.||^2 comes from the
//      partials: (1 + p1)^2 q - 2 (1 + p1) p1 + p2; partial q of x_t  | barrier
//
// Three iterate buffers rotate so that x_min never needs a copy: the buffer
// holding the best iterate is kept out of the rotation until it is beaten.
//
// The grid barrier counts arrivals on one monotone counter; every wait is
// bounded by a %globaltimer budget and an abort flag, so a lost arrival ends
// the kernel with PA_ERR_TIMEOUT instead of a hang.
#include <math.h>

#include "pa_device.cuh"
#include "pa_internal.h"

namespace pa {

namespace {

struct Shared {
  double scratch[4 * kBlock / 32];
  int ok;
};

// Grid-wide barrier with a time limit.  Returns false when the wait gave up
// (this CTA's or another's), after which the caller must leave the kernel.
__device__ __forceinline__ bool grid_barrier(RunState* st, unsigned& target, unsigned G,
                                             long long timeout_ns, bool skip_arrival,
                                             int site, Shared& sh) {
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
      if (ld_relaxed_u32(&st->abort) != 0u) { ok = 0; break; }
      if (++spins > 64) {
        if (globaltimer_ns() - t0 > timeout_ns) {
          if (atomicExch(&st->abort, 1u) == 0u) st->timeout_site = site;
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    sh.ok = ok;
  }
  __syncthreads();
  return sh.ok != 0;
}

__device__ __forceinline__ double* pick(const IterParams& p, int k) {
  return k == 0 ? p.X0 : (k == 1 ? p.X1 : p.X2);
}

__device__ __forceinline__ double loss_value(int mode, int loss, double s, double q) {
  if (loss == PA_LOSS_QUADRATIC) return mode == PA_SIGMA_MAX ? -s : s;
  const double lx = log(sqrt(q)), lax = log(sqrt(s));
  return mode == PA_SIGMA_MAX ? lx - lax : lax - lx;
}

template <int LOSS>
__global__ void __launch_bounds__(kBlock, kMinBlocksPerSM) k_persistent(const IterParams p) {
  __shared__ Shared sh;
  const unsigned G = gridDim.x;
  const int b = blockIdx.x, tid = threadIdx.x;
  const int a0 = p.part_a[b], a1 = p.part_a[b + 1];
  const int c0 = p.part_t[b], c1 = p.part_t[b + 1];
  const int n = p.n_cols;
  RunState* st = p.st;
  double* __restrict__ part = p.partials;

  int cur = 0, minb = 0, t_min = 0, iters_run = 0;
  double L_min = INFINITY, L_last = NAN;
  int status = PA_OK;
  unsigned target = 0;
  int site = 0;

  // ||x_init||^2, partial over the own rows of A^T
  {
    double v[1] = {0.0};
    const double* x = pick(p, cur);
    for (int j = c0 + tid; j < c1; j += kBlock) v[0] = fma(x[j], x[j], v[0]);
    block_sum<1>(v, sh.scratch);
    if (tid == 0) part[b * kPartSlots + 1] = v[0];
  }

  for (int t = 1;; ++t) {
    const double* x = pick(p, cur);
    // ---- phase A: y = A x, partial ||y||^2
    {
      double v[1] = {0.0};
      for (int r = a0 + tid; r < a1; r += kBlock) {
        const double yr = row_dot(p.ci, p.va, __ldg(p.rp + r), __ldg(p.rp + r + 1), x);
        p.y[r] = yr;
        v[0] = fma(yr, yr, v[0]);
      }
      block_sum<1>(v, sh.scratch);
      if (tid == 0) part[b * kPartSlots + 0] = v[0];
    }
    const bool skip = (p.skip_arrival == t) && (b == 0);
    if (!grid_barrier(st, target, G, p.timeout_ns, skip, site++, sh)) { status = PA_ERR_TIMEOUT; break; }
    double s, q;
    {
      if (tid < 32) {
        const double s_ = ordered_sum(part, G, kPartSlots, 0);
        const double q_ = ordered_sum(part, G, kPartSlots, 1);
        if (tid == 0) { sh.scratch[0] = s_; sh.scratch[1] = q_; }
      }
      __syncthreads();
      s = sh.scratch[0];
      q = sh.scratch[1];
      __syncthreads();
    }
    if (!isfinite(s) || !isfinite(q)) { status = PA_ERR_NONFINITE; break; }
    if (t > 1) {  // score x_{t-1}, the iterate produced by the previous iteration
      const double L = loss_value(p.mode, LOSS, s, q);
      L_last = L;
      if (p.L_trace && b == 0 && tid == 0) p.L_trace[t - 2] = L;
      if (L < L_min) { L_min = L; t_min = t - 1; minb = cur; }
    }
    if (s == 0.0) {
      if (p.mode == PA_SIGMA_MIN && t == 1) {
        L_min = loss_value(p.mode, LOSS, s, q);
        t_min = 0;
        minb = cur;
      }
      status = PA_WARN_SINGULAR;
      break;
    }
    if (t == p.iters + 1) break;

    // ---- phase B: z = A^T y, gradient, Adam, partial x.dx and dx.dx
    {
      double ca, cb;  // g = ca * x + cb * z
      if (LOSS == PA_LOSS_QUADRATIC) { ca = 0.0; cb = -2.0; }
      else { ca = 1.0 / q; cb = -1.0 / s; }
      if (p.mode == PA_SIGMA_MIN) { ca = -ca; cb = -cb; }
      const double2 bc = p.bias[t - 1];  // {lr/(1-b1^t), 1/(1-b2^t)}
      const double b1 = p.beta1, b2 = p.beta2, omb1 = 1.0 - b1, omb2 = 1.0 - b2, eps = p.eps;
      double v[2] = {0.0, 0.0};
      for (int j = c0 + tid; j < c1; j += kBlock) {
        const double z = row_dot(p.cit, p.vat, __ldg(p.rpt + j), __ldg(p.rpt + j + 1), p.y);
        const double xj = x[j];
        const double g = (LOSS == PA_LOSS_QUADRATIC) ? cb * z : fma(ca, xj, cb * z);
        const double mj = fma(b1, p.m[j], omb1 * g);
        const double vj = fma(b2, p.v[j], omb2 * (g * g));
        p.m[j] = mj;
        p.v[j] = vj;
        const double d = (bc.x * mj) / (sqrt(bc.y * vj) + eps);
        p.dx[j] = d;
        v[0] = fma(xj, d, v[0]);
        v[1] = fma(d, d, v[1]);
      }
      block_sum<2>(v, sh.scratch);
      if (tid == 0) {
        part[b * kPartSlots + 2] = v[0];
        part[b * kPartSlots + 3] = v[1];
      }
    }
    if (!grid_barrier(st, target, G, p.timeout_ns, false, site++, sh)) { status = PA_ERR_TIMEOUT; break; }
    double p1, p2;
    {
      if (tid < 32) {
        const double a_ = ordered_sum(part, G, kPartSlots, 2);
        const double b_ = ordered_sum(part, G, kPartSlots, 3);
        if (tid == 0) { sh.scratch[0] = a_; sh.scratch[1] = b_; }
      }
      __syncthreads();
      p1 = sh.scratch[0];
      p2 = sh.scratch[1];
      __syncthreads();
    }
    if (!isfinite(p1) || !isfinite(p2)) { status = PA_ERR_NONFINITE; break; }

    // ---- phase C: project, update, normalise; partial ||x_t||^2
    {
      const double c = (p.ablation & PA_ABLATE_NO_TANGENT) ? 0.0 : p1;
      double inv = 1.0;
      if (!(p.ablation & PA_ABLATE_NO_NORMALISE)) {
        const double a1c = 1.0 + c;
        // ||(1+c) x - dx||^2 = (1+c)^2 q - 2 (1+c) p1 + p2
        const double nrm2 = fma(a1c * a1c, q, fma(-2.0 * a1c, p1, p2));
        inv = 1.0 / sqrt(nrm2);
      }
      const int nb = (cur != 0 && minb != 0) ? 0 : ((cur != 1 && minb != 1) ? 1 : 2);
      double* xo = pick(p, nb);
      double* tr = (p.x_trace && t <= p.n_trace) ? p.x_trace + (size_t)(t - 1) * n : nullptr;
      double v[1] = {0.0};
      for (int j = c0 + tid; j < c1; j += kBlock) {
        const double xj = x[j];
        const double xn = (xj - (p.dx[j] - c * xj)) * inv;
        xo[j] = xn;
        if (tr) tr[j] = xn;
        v[0] = fma(xn, xn, v[0]);
      }
      block_sum<1>(v, sh.scratch);
      if (tid == 0) part[b * kPartSlots + 1] = v[0];
      cur = nb;
      iters_run = t;
    }
    if (!grid_barrier(st, target, G, p.timeout_ns, false, site++, sh)) { status = PA_ERR_TIMEOUT; break; }
  }

  if (b == 0 && tid == 0) {
    if (status != PA_ERR_TIMEOUT && ld_relaxed_u32(&st->abort) != 0u) status = PA_ERR_TIMEOUT;
    st->status = status;
    st->minb = minb;
    st->cur = cur;
    st->t_min = t_min;
    st->L_min = L_min;
    st->L_last = L_last;
    st->iters_run = iters_run;
  }
}

}  // namespace

int persistent_max_blocks(int loss, int* blocks_per_sm) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e;
  if (loss == PA_LOSS_QUADRATIC)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_persistent<PA_LOSS_QUADRATIC>, kBlock, 0);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_persistent<PA_LOSS_LOGRATIO>, kBlock, 0);
  if (e != cudaSuccess) return -1;
  if (blocks_per_sm) *blocks_per_sm = per;
  return per * sms;
}

cudaError_t launch_persistent(const IterParams& p, int loss, int G, cudaStream_t s,
                              int64_t* launches) {
  void* args[] = {(void*)&p};
  void* fn = loss == PA_LOSS_QUADRATIC ? (void*)k_persistent<PA_LOSS_QUADRATIC>
                                       : (void*)k_persistent<PA_LOSS_LOGRATIO>;
  cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kBlock), args, 0, s);
  ++*launches;
  return e;
}

}  // namespace pa
