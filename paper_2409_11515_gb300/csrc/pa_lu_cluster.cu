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
// Here the single-CTA kernel's steps run on a cluster of up to 16 CTAs: the
// solve vector is spread over their shared memories (element i in CTA
// i mod C, slot i / C), every step's items are dealt over all the cluster's
// threads (an item reads its row's partial and the final values of its
// columns, in any CTA, and writes the row back; the items of a step have
// distinct rows), and the hardware cluster barrier (a quarter of a
// microsecond on GB300) ends the step.  Every solve of the chain
// L t = P x, U u = t, U^T a = u, L^T c = a starts from the previous
// solve's result at the same index (b_i / T_ii), so one vector serves the
// whole chain, transformed in place, and n may reach 16 x 27,000 rows.
// Nothing waits on anything but the cluster barrier, which every CTA passes
// the same number of times.  The reductions are the grid kernel's (fixed
// orders: runs are reproducible).
#include <math.h>

#include <cooperative_groups.h>

#include "pa_device.cuh"
#include "pa_internal.h"
#include "pa_lu_cluster.h"

namespace pa {

namespace {

constexpr int kLcThreads = 512;

struct LcShared {
  double scratch[2 * kLcThreads];
  double ca, cb, c, inv, q_keep, L_min, L_last;
  int brk, improved, t_min, iters_run, status;
};

extern __shared__ double lc_vec[];  // this CTA's slots of the solve vector

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

__device__ __forceinline__ void lc_store(uint32_t ra, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(ra), "d"(v) : "memory");
}

// Element i of the solve vector (slots start at shared address `base`, the
// same offset in every CTA of the cluster).
__device__ __forceinline__ uint32_t lc_elem(uint32_t base, int i, int lgC) {
  return lc_map(base + 8u * (uint32_t)(i >> lgC), (uint32_t)i & ((1u << lgC) - 1u));
}

__device__ __forceinline__ void lc_sync() { cooperative_groups::this_cluster().sync(); }

// One item of a step (a thread, or lane gl of a group of G for a longer
// segment, whose partial the caller sums): {row, column, value} or
// {~row, first entry, end entry}; lane 0 of a group starts from x[row].
__device__ __forceinline__ double lc_item(const int4& r, const TriSys& T, uint32_t base, int lgC,
                                          int gl, int G, int* row) {
  if (r.x >= 0) {
    *row = r.x;
    return gl == 0 ? fma(__hiloint2double(r.w, r.z), lc_load(lc_elem(base, r.y, lgC)),
                         lc_load(lc_elem(base, r.x, lgC)))
                   : 0.0;
  }
  *row = ~r.x;
  double acc = gl == 0 ? lc_load(lc_elem(base, ~r.x, lgC)) : 0.0;
  for (int e = r.y + gl; e < r.z; e += G)
    acc = fma(__ldg(T.va + e), lc_load(lc_elem(base, __ldg(T.ci + e), lgC)), acc);
  return acc;
}

// This thread's first item record of the step described by J (its index:
// the thread's global index for one thread per item, its group's for groups),
// or a record that is never used.
__device__ __forceinline__ int4 lc_first(const TriSys& T, const int4& J, int gt) {
  const int nit = (J.y & kItemMask) - J.x, lg = (J.y >> 27) & 7;
  const int k = gt >> lg;
  return k < nit ? __ldg(T.items + J.x + k) : make_int4(0, 0, 0, 0);
}

// T x = b for x holding b / diag on entry: the steps, each dealt over the
// cluster's C x kLcThreads threads and ended by the cluster barrier.  The
// records a step needs do not depend on the solve, so each thread loads the
// step record two steps ahead and its first item record one step ahead:
// their latency overlaps the current step instead of adding to the chain.
__device__ __forceinline__ void lc_steps(const TriSys& T, uint32_t base, int lgC) {
  cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
  const int GT = (int)cl.num_blocks() * kLcThreads;
  const int gt = (int)cl.block_rank() * kLcThreads + (int)threadIdx.x;
  const int np = T.nproc;
  int4 I = np > 0 ? __ldg(T.linfo) : make_int4(0, 0, 0, 0);
  int4 In = np > 1 ? __ldg(T.linfo + 1) : make_int4(0, 0, 0, 0);
  int4 rec = np > 0 ? lc_first(T, I, gt) : make_int4(0, 0, 0, 0);
  for (int l = 0; l < np; ++l) {
    const int4 Inn = l + 2 < np ? __ldg(T.linfo + l + 2) : make_int4(0, 0, 0, 0);
    const int4 recn = l + 1 < np ? lc_first(T, In, gt) : make_int4(0, 0, 0, 0);
    const int nit = (I.y & kItemMask) - I.x, lg = (I.y >> 27) & 7;
    const int4* IT = T.items + I.x;
    if (lg == 0) {  // a thread per item
      for (int k = gt; k < nit; k += GT) {
        int row;
        const double v = lc_item(k == gt ? rec : __ldg(IT + k), T, base, lgC, 0, 1, &row);
        lc_store(lc_elem(base, row, lgC), v);
      }
    } else {  // 2^lg lanes per item, then a butterfly inside the group
      const int G = 1 << lg, gid = gt >> lg, gl = gt & (G - 1), ng = GT >> lg;
      for (int k0 = 0; k0 < nit; k0 += ng) {  // the same trip count for every thread
        const int k = k0 + gid;
        double acc = 0.0;
        int row = 0;
        if (k < nit) acc = lc_item(k0 == 0 ? rec : __ldg(IT + k), T, base, lgC, gl, G, &row);
        for (int d = G >> 1; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
        if (k < nit && gl == 0) lc_store(lc_elem(base, row, lgC), acc);
      }
    }
    cl.sync();  // the step's rows are written before the next step reads them
    I = In;
    In = Inn;
    rec = recn;
  }
}

__global__ void __launch_bounds__(kLcThreads, 1) k_lu_cluster(const LuClusterParams P, int R,
                                                              int lgC) {
  __shared__ LcShared sh;
  const LuGridParams& p = P.g;
  const int n = p.n, tid = threadIdx.x;
  const unsigned C = gridDim.x;
  const int b = blockIdx.x;
  RunState* st = p.st;
  double* part = p.partials;
  const uint32_t V = (uint32_t)__cvta_generic_to_shared(lc_vec);
  const int32_t* perm = p.p;
  if (tid == 0) {
    sh.L_min = INFINITY;
    sh.L_last = NAN;
    sh.t_min = 0;
    sh.iters_run = 0;
    sh.status = PA_OK;
  }
  // every CTA has started (its shared memory exists) before any remote access
  lc_sync();
  // this CTA's slots: slot s holds element i = s C + b of the vector
  auto own = [&](int s) { return s * (int)C + b; };
  // r = A^{-1} v: L t = P v, U u = t in place; ||v||^2 and ||u||^2 per thread
  auto apply_inv = [&](const double* vsrc, double& q2, double& rr) {
    for (int s = tid; s < R; s += kLcThreads) {
      const int i = own(s);
      if (i < n) {
        const double bi = vsrc[perm ? __ldg(perm + i) : i];
        q2 = fma(bi, bi, q2);
        lc_vec[s] = bi * __ldg(P.sys[0].dinv + i);
      }
    }
    lc_sync();
    lc_steps(P.sys[0], V, lgC);
    for (int s = tid; s < R; s += kLcThreads) {
      const int i = own(s);
      if (i < n) lc_vec[s] *= __ldg(P.sys[1].dinv + i);
    }
    lc_sync();
    lc_steps(P.sys[1], V, lgC);
    for (int s = tid; s < R; s += kLcThreads) {
      const int i = own(s);
      if (i < n) rr = fma(lc_vec[s], lc_vec[s], rr);
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
      if (i < n) lc_vec[s] *= __ldg(P.sys[2].dinv + i);
    }
    lc_sync();
    lc_steps(P.sys[2], V, lgC);
    for (int s = tid; s < R; s += kLcThreads) {
      const int i = own(s);
      if (i < n) lc_vec[s] *= __ldg(P.sys[3].dinv + i);
    }
    lc_sync();
    lc_steps(P.sys[3], V, lgC);
    for (int s = tid; s < R; s += kLcThreads) {
      const int i = own(s);
      if (i < n) p.w[perm ? __ldg(perm + i) : i] = lc_vec[s];
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
}

size_t lc_smem(int R) { return sizeof(double) * (size_t)R; }

}  // namespace

int lu_cluster_plan(int n, int* lgC_out, int* R_out) {
  void* fn = (void*)k_lu_cluster;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  for (int lgC = 4; lgC >= 3; --lgC) {  // clusters of 16, else 8
    const int C = 1 << lgC;
    const int R = (n + C - 1) / C;
    const size_t dyn = lc_smem(R);
    if (dyn + sizeof(LcShared) > (size_t)optin) continue;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess) {
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
      if (lgC_out) *lgC_out = lgC;
      if (R_out) *R_out = R;
      return C;
    }
    cudaGetLastError();
  }
  return 0;
}

cudaError_t launch_lu_cluster(const LuClusterParams& p, int lgC, int R, cudaStream_t s,
                              int64_t* launches) {
  void* fn = (void*)k_lu_cluster;
  const int C = 1 << lgC;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(kLcThreads);
  cfg.dynamicSmemBytes = lc_smem(R);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[] = {(void*)&p, (void*)&R, (void*)&lgC};
  ++*launches;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace pa
