// pa_iter.cu -- the persistent cooperative Projected Adam kernel (the paper's
// Algorithm 1 with the gradient of Eq. nabla_loss) for one vector.
//
// The matrix is held as P A Q^T and Q A^T P^T in sliced ELL form (rows sorted
// by length inside windows, 32-row slices stored column-major), so the 32
// lanes of a warp walk rows of equal length with coalesced loads; sigma and
// Algorithm 1 are unchanged by the permutations, which only relabel the
// coordinates of x (Q) and of y (P).
//
// One launch runs every iteration without returning to the host.  CTA b owns
// a contiguous range of slices of P A Q^T (phase A) and of Q A^T P^T (phases
// B and C); the ranges are balanced by padded entries plus a per-row weight,
// and inside a CTA the host deals the slices to the warps by the same cost
// (longest first to the least loaded warp).
// Per iteration t:
//
//   A  y = A x_{t-1} (own rows); partials s = sum y_i^2, q = ||x||^2 | grid barrier
//      every CTA sums the partials in the same fixed order -> s, q = ||x||^2;
//      L(x_{t-1}) is scored against L_min (Algorithm 1's tracking, lagged by
//      one product so that y serves both the score and the gradient).
//   B  z = A^T y over the explicit transpose (own rows), the gradient
//      g = a x + b z, Adam's moments and step dx (kept in `dx`), partials
//      p1 = x.dx, p2 = dx.dx                                  | grid barrier
//   C  x_t = ((1 + p1) x - dx) / ||.||, the tangent projection and the
//      normalisation of Algorithm 1 in one pass; ||.||^2 comes from the
//      partials: (1 + p1)^2 q - 2 (1 + p1) p1 + p2.  The CTA then publishes
//      "x_t written" on its ready flag; the next phase A waits only for the
//      flags of the CTAs whose x rows its products read (a banded operator
//      reads a few neighbours), not for the whole grid.
//
// Three iterate buffers rotate so that x_min never needs a copy: the buffer
// holding the best iterate is kept out of the rotation until it is beaten.
//
// The grid barrier counts arrivals on one monotone counter; every wait is
// bounded by a %globaltimer budget and an abort flag, so a lost arrival ends
// the kernel with PA_ERR_TIMEOUT instead of a hang.
#include <math.h>

#include <cooperative_groups.h>
#include <type_traits>

#include "pa_device.cuh"
#include "pa_internal.h"

namespace pa {

namespace {

struct Shared {
  double scratch[2 * kBlock];
  // per-iteration scalars, computed once by thread 0 and read by all threads
  double ca, cb;      // g = ca * x + cb * z
  double c, inv;      // 1 + the projection coefficient, and 1 / ||x'||
  int brk;            // leave the iteration loop
  int cur, nb;        // buffer of x_{t-1}, buffer for x_t
  int ok;
  // Algorithm 1's tracking state, owned by thread 0: the best and the latest
  // scored (||y||^2, ||x||^2); L itself is formed once at the end
  double best_s, best_q, last_s, last_q;
  int have_best, have_last;
  int minb, t_min, iters_run, status;
  // busy time per phase (barrier waits excluded), read by the partition tuner
  unsigned long long busy_a, busy_b;
  unsigned long long lat_a;  // sum of (end of phase A - start of the previous phase C)
  long long tmark, tc;
};

// The cluster engine adds two tables of per-warp partial pairs, one slot per
// (CTA, warp) of the cluster: phase A's (||y||^2, ||x||^2) and phase B's
// (x.dx, dx.dx).  Every warp writes its pair into the slot of every CTA of
// the cluster (distributed shared memory) before the cluster barrier, and
// each CTA then sums its own table in a fixed order: no block barrier and no
// round trip through global memory on the reduction's path.  Two tables, so
// that a CTA already writing the next reduction never meets one still being
// read (a CTA passes the following cluster barrier only after every CTA has
// finished reading).
constexpr int kMaxCluster = 16;
struct SharedCL : Shared {
  double ctab[2][kMaxCluster * (kBlock / 32)][2];
};

// Cluster engine: this warp's two partial sums into slot (b, warp) of table
// `tab` in every CTA of the cluster.
__device__ __forceinline__ void cluster_scatter(double (*tab)[2], double v0, double v1, int b,
                                                int warp, int lane, unsigned G) {
  v0 = warp_sum(v0);
  v1 = warp_sum(v1);
  if (lane < (int)G) {
    double* dst = cooperative_groups::this_cluster().map_shared_rank(&tab[0][0], (unsigned)lane);
    const int slot = b * (kBlock / 32) + warp;
    dst[2 * slot] = v0;
    dst[2 * slot + 1] = v1;
  }
}

// Cluster engine: component k of the sum over the table's first n slots, in
// a fixed order (one warp; loads first, a pairwise tree, then the butterfly).
__device__ __forceinline__ double cluster_total(const double (*tab)[2], int n, int k) {
  const int lane = threadIdx.x & 31;
  double u[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int i = lane + 32 * j;
    u[j] = i < n ? tab[i][k] : 0.0;
  }
  u[0] += u[1]; u[2] += u[3]; u[4] += u[5]; u[6] += u[7];
  u[0] += u[2]; u[4] += u[6];
  return warp_sum(u[0] + u[4]);
}

__device__ __forceinline__ double* pick(const IterParams& p, int k) {
  return k == 0 ? p.X0 : (k == 1 ? p.X1 : p.X2);
}

__device__ __forceinline__ double loss_value(int mode, int loss, double s, double q) {
  if (loss == PA_LOSS_QUADRATIC) return mode == PA_SIGMA_MAX ? -s : s;
  const double lx = log(sqrt(q)), lax = log(sqrt(s));
  return mode == PA_SIGMA_MAX ? lx - lax : lax - lx;
}

// CL: the grid is one thread-block cluster (up to 16 CTAs) and every
// grid-wide synchronisation is the hardware cluster barrier (release/acquire
// at cluster scope), for matrices too small to fill the GPU.
template <int LOSS, bool DD, bool CL>
__global__ void __launch_bounds__(kBlock, kMinBlocksPerSM) k_persistent(const IterParams p) {
  __shared__ typename std::conditional<CL, SharedCL, Shared>::type sh;
  constexpr int NW = kBlock / 32;
  const unsigned G = gridDim.x;
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int sa0 = p.part_a[b], sa1 = p.part_a[b + 1];
  const int st0 = p.part_t[b], st1 = p.part_t[b + 1];
  const int n = p.n_cols;
  const int r0 = 32 * st0, r1 = min(32 * st1, n);  // own rows of x (positions)
  RunState* st = p.st;
  double* __restrict__ part = p.partials;

  // Algorithm 1's scalar state lives in shared memory, written by thread 0
  // of every CTA (each CTA computes the same values from the same
  // fixed-order sums).
  unsigned target = 0;
  int site = 0;
  int status = PA_OK;  // this thread's view; thread 0 keeps the run's status in sh
  if (tid == 0) {
    sh.cur = 0;
    sh.brk = 0;
    sh.minb = p.init_minb;   // a continued run starts with the tracked state
    sh.t_min = p.init_t_min; // of the run it continues (zeros for a fresh run)
    sh.iters_run = 0;
    sh.status = PA_OK;
    sh.have_best = p.init_have_best;
    sh.best_s = p.init_best_s;
    sh.best_q = p.init_best_q;
    sh.have_last = 0;
    sh.busy_a = sh.busy_b = 0;
    sh.lat_a = 0;
    sh.tc = 0;
  }

  const int dlo = p.dep[2 * b], dhi = p.dep[2 * b + 1];
  // every thread reads sh.cur at t = 1: shared memory starts with whatever
  // the SM's previous launch left there.  The cluster engine waits for the
  // whole cluster instead: its warps write into the other CTAs' shared
  // memory, which must have started.
  if constexpr (CL) cooperative_groups::this_cluster().sync();
  else __syncthreads();

  // per-thread partial of ||x||^2 over the own rows, carried into phase A
  double qloc = 0.0;
  {
    const double* x = pick(p, 0);
    for (int j = r0 + tid; j < r1; j += kBlock) qloc = fma(x[j], x[j], qloc);
  }

  for (int t = 1;; ++t) {
    // x_{t-1} of the neighbours must be written before the gathers below
    if (CL) {
      if (t > 1) cooperative_groups::this_cluster().sync();
    } else if (t > 1 &&
               !wait_ready(st, p.ready, dlo, dhi, (unsigned)(t - 1), p.timeout_ns, site++, sh.ok)) {
      status = PA_ERR_TIMEOUT;
      break;
    }
    const double* x = pick(p, sh.cur);
    if (tid == 0) sh.tmark = globaltimer_ns();
    // ---- phase A: y = A x, partials ||y||^2 and ||x||^2
    {
      double v[2] = {0.0, qloc};
      const int k0 = p.a_woff[b * (NW + 1) + warp], k1 = p.a_woff[b * (NW + 1) + warp + 1];
      for (int k = k0; k < k1; ++k) {  // this warp's share of the CTA's slices
        const int s = __ldg(p.a_list + k);
        if (k + 1 < k1) prefetch_slice_l2(p.a_wp, p.a_col, p.a_val, __ldg(p.a_list + k + 1), lane);
        const int r = 32 * s + lane;
        double yr;
        if (DD) {
          double lo;
          slice_dot_dd(p.a_wp, p.a_col, p.a_val, s, lane, x, yr, lo);
          if (r < p.n_rows) p.ylo[r] = lo;
        } else {
          yr = slice_dot(p.a_wp, p.a_col, p.a_val, s, lane, x);
        }
        if (r < p.n_rows) {
          p.y[r] = yr;
          v[0] = fma(yr, yr, v[0]);
        }
      }
      if constexpr (CL) {
        cluster_scatter(sh.ctab[0], v[0], v[1], b, warp, lane, G);
      } else {
        block_sum_to0<2>(v, sh.scratch);
      }
      if (tid == 0) {
        if (!CL) {
          part[b * kPartSlots + 0] = v[0];
          part[b * kPartSlots + 1] = v[1];
        }
        const long long now = globaltimer_ns();
        sh.busy_a += (unsigned long long)(now - sh.tmark);
        // how late this CTA's y is: phase C, the neighbour wait and phase A
        if (sh.tc) sh.lat_a += (unsigned long long)(now - sh.tc);
      }
    }
    const bool skip = (p.skip_arrival == t) && (b == 0);
    if (CL) cooperative_groups::this_cluster().sync();
    else if (!grid_barrier(st, target, G, p.timeout_ns, skip, site++, sh.ok)) { status = PA_ERR_TIMEOUT; break; }
    if (tid < 32) {
      double s_, q;
      if constexpr (CL) {
        s_ = cluster_total(sh.ctab[0], (int)G * NW, 0);
        q = cluster_total(sh.ctab[0], (int)G * NW, 1);
      } else {
        s_ = ordered_sum(part, G, kPartSlots, 0);
        q = ordered_sum(part, G, kPartSlots, 1);
      }
      // g' = (1 - beta1) g = ca x + cb z (the first moment's weight folded
      // in): lanes 0 and 1 run one division sequence for both coefficients
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
          if (t > 1) {  // score x_{t-1}, the iterate produced by the previous iteration
            // L(x) < L_min through the monotone map of the loss: for the
            // log-ratio loss log||x|| - log||y|| < log||x_b|| - log||y_b||
            // iff ||x||^2 ||y_b||^2 < ||x_b||^2 ||y||^2 (sigma_max; swapped
            // for sigma_min), so no logarithm is taken in the loop
            bool better;
            if (LOSS == PA_LOSS_QUADRATIC) {
              const double L = loss_value(p.mode, LOSS, s_, q);
              better = !sh.have_best || L < loss_value(p.mode, LOSS, sh.best_s, sh.best_q);
            } else if (!sh.have_best) {
              better = p.mode == PA_SIGMA_MIN || s_ > 0.0;  // L = +inf never beats +inf
            } else {
              better = p.mode == PA_SIGMA_MAX ? q * sh.best_s < sh.best_q * s_
                                              : s_ * sh.best_q < sh.best_s * q;
            }
            if (better) {
              sh.best_s = s_;
              sh.best_q = q;
              sh.have_best = 1;
              sh.t_min = p.t_min_base + t - 1;
              sh.minb = cur;
            }
            sh.last_s = s_;
            sh.last_q = q;
            sh.have_last = 1;
            if (p.L_trace && b == 0) p.L_trace[t - 2] = loss_value(p.mode, LOSS, s_, q);
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
        sh.scratch[0] = q;  // kept for the normalisation below
        sh.brk = brk;
      }
    }
    __syncthreads();
    if (sh.brk) break;
    const double q_keep = (tid == 0) ? sh.scratch[0] : 0.0;

    // ---- phase B: z = A^T y, gradient, Adam, partial x.dx and dx.dx
    if (tid == 0) sh.tmark = globaltimer_ns();
    {
      const double ca = sh.ca, cb = sh.cb;
      // lr m_hat / (sqrt(v_hat) + eps) = K1 m / (sqrt(v) + K2) with
      // K1 = lr sqrt(1-b2^t) / (1-b1^t) and K2 = eps sqrt(1-b2^t)
      const double2 bc = p.bias[p.t0 + t - 1];
      const double b1 = p.beta1, b2 = p.beta2;
      const double w2 = p.w2;  // (1 - beta2) g^2 = w2 g'^2 with g' = (1 - beta1) g
      double v[2] = {0.0, 0.0};
      const int k0 = p.t_woff[b * (NW + 1) + warp], k1 = p.t_woff[b * (NW + 1) + warp + 1];
      for (int k = k0; k < k1; ++k) {
        const int s = __ldg(p.t_list + k);
        if (!DD && k + 1 < k1) prefetch_slice_l2(p.t_wp, p.t_col, p.t_val, __ldg(p.t_list + k + 1), lane);
        const double z = DD ? slice_dot_dd2(p.t_wp, p.t_col, p.t_val, s, lane, p.y, p.ylo)
                            : slice_dot(p.t_wp, p.t_col, p.t_val, s, lane, p.y);
        const int j = 32 * s + lane;
        if (j < n) {
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
      }
      if constexpr (CL) {
        cluster_scatter(sh.ctab[1], v[0], v[1], b, warp, lane, G);
      } else {
        block_sum_to0<2>(v, sh.scratch);
      }
      if (tid == 0) {
        if (!CL) {
          part[b * kPartSlots + 2] = v[0];
          part[b * kPartSlots + 3] = v[1];
        }
        sh.busy_b += (unsigned long long)(globaltimer_ns() - sh.tmark);
      }
    }
    if (CL) cooperative_groups::this_cluster().sync();
    else if (!grid_barrier(st, target, G, p.timeout_ns, false, site++, sh.ok)) { status = PA_ERR_TIMEOUT; break; }
    if (tid < 32) {
      double p1, p2;
      if constexpr (CL) {
        p1 = cluster_total(sh.ctab[1], (int)G * NW, 0);
        p2 = cluster_total(sh.ctab[1], (int)G * NW, 1);
      } else {
        p1 = ordered_sum(part, G, kPartSlots, 2);
        p2 = ordered_sum(part, G, kPartSlots, 3);
      }
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
          // ||(1+c) x - dx||^2 = (1+c)^2 q - 2 (1+c) p1 + p2
          const double nrm2 = fma(a1c * a1c, q_keep, fma(-2.0 * a1c, p1, p2));
          inv = rsqrt(nrm2);  // scales x only: the loss and Adam's step are scale-free
        }
        sh.c = 1.0 + c;  // phase C uses 1 + c
        sh.inv = inv;
        const int cur = sh.cur, minb = sh.minb;
        sh.nb = (cur != 0 && minb != 0) ? 0 : ((cur != 1 && minb != 1) ? 1 : 2);
        sh.brk = brk;
      }
    }
    __syncthreads();
    if (sh.brk) break;

    // ---- phase C: project, update, normalise; partial ||x_t||^2
    if (tid == 0) sh.tc = sh.tmark = globaltimer_ns();
    {
      const double a1c = sh.c, inv = sh.inv;
      const int nb = sh.nb;
      double* xo = pick(p, nb);
      double* tr = (p.x_trace && t <= p.n_trace) ? p.x_trace + (size_t)(t - 1) * n : nullptr;
      qloc = 0.0;
      for (int j = r0 + tid; j < r1; j += kBlock) {
        const double xj = x[j];
        const double xn = fma(a1c, xj, -p.dx[j]) * inv;  // (x - (dx - c x)) / ||.||
        xo[j] = xn;
        if (tr) tr[j] = xn;
        qloc = fma(xn, xn, qloc);
      }
      __syncthreads();  // every x_t row of this CTA is written
      if (tid == 0) {
        publish_ready(p.ready + b, (unsigned)t);
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
  if (tid == 0 && p.cta_lat) p.cta_lat[b] = sh.lat_a;
  if (b == 0 && tid == 0) {
    if (status == PA_ERR_TIMEOUT || ld_relaxed_u32(&st->abort) != 0u) sh.status = PA_ERR_TIMEOUT;
    st->status = sh.status;
    st->minb = sh.minb;
    st->cur = sh.cur;
    st->t_min = sh.t_min;
    st->L_min = sh.have_best ? loss_value(p.mode, LOSS, sh.best_s, sh.best_q) : INFINITY;
    st->L_last = sh.have_last ? loss_value(p.mode, LOSS, sh.last_s, sh.last_q) : NAN;
    st->iters_run = sh.iters_run;
    st->best_s = sh.best_s;
    st->best_q = sh.best_q;
    st->have_best = sh.have_best;
  }
}

}  // namespace

static void* persistent_fn(int loss, bool dd, bool cl = false) {
  if (cl)
    return loss == PA_LOSS_QUADRATIC ? (void*)k_persistent<PA_LOSS_QUADRATIC, false, true>
                                     : (void*)k_persistent<PA_LOSS_LOGRATIO, false, true>;
  if (loss == PA_LOSS_QUADRATIC)
    return dd ? (void*)k_persistent<PA_LOSS_QUADRATIC, true, false>
              : (void*)k_persistent<PA_LOSS_QUADRATIC, false, false>;
  return dd ? (void*)k_persistent<PA_LOSS_LOGRATIO, true, false>
            : (void*)k_persistent<PA_LOSS_LOGRATIO, false, false>;
}

int persistent_max_blocks(int loss, bool dd, int* blocks_per_sm) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const cudaError_t e =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, persistent_fn(loss, dd), kBlock, 0);
  if (e != cudaSuccess) return -1;
  if (blocks_per_sm) *blocks_per_sm = per;
  return per * sms;
}

cudaError_t launch_persistent(const IterParams& p, int loss, bool dd, int G, cudaStream_t s,
                              int64_t* launches) {
  void* args[] = {(void*)&p};
  void* fn = persistent_fn(loss, dd);
  cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kBlock), args, 0, s);
  ++*launches;
  return e;
}

// Largest cluster (<= 16 CTAs) of the cluster variant that the GPU can hold.
int persistent_cluster_max(int loss) {
  void* fn = persistent_fn(loss, false, true);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return 8;
  }
  for (int c = 16; c >= 1; c /= 2) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c);
    cfg.blockDim = dim3(kBlock);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) == cudaSuccess && n >= 1) return c;
    cudaGetLastError();
  }
  return 1;
}

cudaError_t launch_persistent_cluster(const IterParams& p, int loss, int G, cudaStream_t s,
                                      int64_t* launches) {
  void* fn = persistent_fn(loss, false, true);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(kBlock);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = G;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[] = {(void*)&p};
  ++*launches;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace pa
