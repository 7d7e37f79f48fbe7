// pa_setup.cu -- one-time and auxiliary kernels of the Projected Adam library:
// CSR validation, the stable CSR transpose that gives the explicit A^T used by
// the transposed product, work partitions of the persistent grid, the seeded
// start vector, a standalone SpMV, and the final sigma = ||A x|| / ||x||.
#include "pa_device.cuh"
#include "pa_internal.h"

namespace pa {

namespace {

constexpr int kT = 256;            // threads per block of the setup kernels
constexpr int kScanPer = 4;        // elements per thread in the scan
constexpr int kScanChunk = 1024 * kScanPer;

inline int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }
inline int grid_for(int64_t n, int per_block = kT, int cap = 152 * 32) {
  int g = cdiv(n, per_block);
  return g < 1 ? 1 : (g > cap ? cap : g);
}

// ------------------------------------------------------------- validate --
// flag bit 1: row_ptr ends wrong, bit 2: row_ptr decreases, bit 4: column
// index out of range.
__global__ void k_validate(int32_t n_rows, int32_t n_cols, int64_t nnz,
                           const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           int* flag) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t0 == 0 && (rp[0] != 0 || (int64_t)rp[n_rows] != nnz)) atomicOr(flag, 1);
  for (int64_t r = t0; r < n_rows; r += stride)
    if (rp[r + 1] < rp[r]) atomicOr(flag, 2);
  for (int64_t k = t0; k < nnz; k += stride) {
    const int32_t c = ci[k];
    if (c < 0 || c >= n_cols) atomicOr(flag, 4);
  }
}

// ------------------------------------------------------------ transpose --
__global__ void k_count_cols(int64_t nnz, const int32_t* __restrict__ ci, int32_t* cnt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += stride)
    atomicAdd(&cnt[ci[k]], 1);
}

// Sum of each kScanChunk-element chunk of in[0, n).
__global__ void __launch_bounds__(1024) k_scan_sums(int64_t n, const int32_t* __restrict__ in,
                                                    int32_t* sums) {
  __shared__ int32_t ws[32];
  const int64_t base = (int64_t)blockIdx.x * kScanChunk;
  int32_t a = 0;
  for (int i = 0; i < kScanPer; ++i) {
    const int64_t idx = base + (int64_t)threadIdx.x * kScanPer + i;
    if (idx < n) a += in[idx];
  }
  for (int d = 16; d > 0; d >>= 1) a += __shfl_xor_sync(0xffffffffu, a, d);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x < 32) {
    int32_t b = ws[threadIdx.x];
    for (int d = 16; d > 0; d >>= 1) b += __shfl_xor_sync(0xffffffffu, b, d);
    if (threadIdx.x == 0) sums[blockIdx.x] = b;
  }
}

// Exclusive scan of sums[0, nb) in place, one block.
__global__ void __launch_bounds__(1024) k_scan_top(int nb, int32_t* sums) {
  __shared__ int32_t buf[1024];
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += 1024) {
    const int i = base + threadIdx.x;
    const int32_t v = i < nb ? sums[i] : 0;
    buf[threadIdx.x] = v;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {  // Hillis-Steele inclusive scan
      const int32_t add = threadIdx.x >= d ? buf[threadIdx.x - d] : 0;
      __syncthreads();
      buf[threadIdx.x] += add;
      __syncthreads();
    }
    if (i < nb) sums[i] = carry + buf[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += buf[1023];
    __syncthreads();
  }
}

// out[i] = exclusive prefix of in up to i (i < n), out[n] = total.
__global__ void __launch_bounds__(1024) k_scan_apply(int64_t n, const int32_t* __restrict__ in,
                                                     const int32_t* __restrict__ sums,
                                                     int32_t* out) {
  __shared__ int32_t ws[32];
  const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanPer;
  int32_t v[kScanPer];
  int32_t local = 0;
  for (int i = 0; i < kScanPer; ++i) {
    v[i] = (base + i < n) ? in[base + i] : 0;
    local += v[i];
  }
  // exclusive scan of `local` across the block
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t inc = local;
  for (int d = 1; d < 32; d <<= 1) {
    const int32_t o = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += o;
  }
  if (lane == 31) ws[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int32_t w = ws[lane];
    for (int d = 1; d < 32; d <<= 1) {
      const int32_t o = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= d) w += o;
    }
    ws[lane] = w;
  }
  __syncthreads();
  int32_t run = sums[blockIdx.x] + (warp > 0 ? ws[warp - 1] : 0) + inc - local;
  for (int i = 0; i < kScanPer; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
  if (base <= n - 1 && n - 1 < base + kScanPer) out[n] = run - 0;  // total after last element
}

__global__ void k_copy_i32(int64_t n, const int32_t* __restrict__ a, int32_t* b) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) b[i] = a[i];
}

__global__ void k_row_ids(int32_t n_rows, const int32_t* __restrict__ rp, int32_t* rowid) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_rows; r += stride)
    for (int32_t k = rp[r]; k < rp[r + 1]; ++k) rowid[k] = (int32_t)r;
}

__global__ void k_scatter(int64_t nnz, const int32_t* __restrict__ ci, int32_t* cursor,
                          int32_t* src) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += stride) {
    const int32_t pos = atomicAdd(&cursor[ci[k]], 1);
    src[pos] = (int32_t)k;
  }
}

// Sort each row segment of A^T by source position (= row-major order of A),
// which makes the transpose stable and independent of the scatter's timing.
// Short segments: insertion sort; long ones: heap sort (in place, O(L log L)).
__device__ void sift_down(int32_t* a, int root, int len) {
  while (true) {
    int c = 2 * root + 1;
    if (c >= len) return;
    if (c + 1 < len && a[c + 1] > a[c]) ++c;
    if (a[root] >= a[c]) return;
    const int32_t t = a[root];
    a[root] = a[c];
    a[c] = t;
    root = c;
  }
}

__global__ void k_segsort(int32_t n_cols, const int32_t* __restrict__ rpt, int32_t* src) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_cols; j += stride) {
    int32_t* a = src + rpt[j];
    const int len = rpt[j + 1] - rpt[j];
    if (len <= 32) {
      for (int i = 1; i < len; ++i) {
        const int32_t key = a[i];
        int p = i - 1;
        while (p >= 0 && a[p] > key) {
          a[p + 1] = a[p];
          --p;
        }
        a[p + 1] = key;
      }
    } else {
      for (int r = len / 2 - 1; r >= 0; --r) sift_down(a, r, len);
      for (int end = len - 1; end > 0; --end) {
        const int32_t t = a[0];
        a[0] = a[end];
        a[end] = t;
        sift_down(a, 0, end);
      }
    }
  }
}

__global__ void k_gather_t(int64_t nnz, const int32_t* __restrict__ src,
                           const int32_t* __restrict__ rowid, const double* __restrict__ va,
                           int32_t* cit, double* vat) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += stride) {
    const int32_t e = src[p];
    cit[p] = rowid[e];
    vat[p] = va[e];
  }
}

// ------------------------------------------------------------ partition --
// part[b] = first slice s with cost(s) >= b * cost(n_slices) / G, where
// cost(s) = 32 * wp[s] + w * 32 * s (padded entries plus a per-row weight).
__global__ void k_partition(const int32_t* __restrict__ wp, int32_t ns, int G, int w,
                            int32_t* part) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b > G) return;
  const double total = 32.0 * wp[ns] + 32.0 * w * ns;
  const double target = total * b / G;
  int lo = 0, hi = ns;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const double c = 32.0 * wp[mid] + 32.0 * w * mid;
    if (c >= target) hi = mid; else lo = mid + 1;
  }
  part[b] = (b == G) ? ns : lo;
}

// One block per CTA b of the persistent grid: smallest and largest x
// position read by a non-zero of b's slices, mapped to the owning CTAs
// (CTA j owns positions [32 part_t[j], 32 part_t[j+1])).
__global__ void __launch_bounds__(kT) k_dependencies(const int32_t* __restrict__ wp,
                                                     const int32_t* __restrict__ col,
                                                     const double* __restrict__ val,
                                                     const int32_t* __restrict__ part_a,
                                                     const int32_t* __restrict__ part_t, int G,
                                                     int32_t* dep) {
  __shared__ int32_t smin[kT], smax[kT];
  const int b = blockIdx.x;
  const int64_t e0 = 32ll * wp[part_a[b]], e1 = 32ll * wp[part_a[b + 1]];
  int32_t lo = 0x7fffffff, hi = -1;
  for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    if (val[e] != 0.0) {
      const int32_t c = col[e];
      lo = c < lo ? c : lo;
      hi = c > hi ? c : hi;
    }
  }
  smin[threadIdx.x] = lo;
  smax[threadIdx.x] = hi;
  __syncthreads();
  for (int d = blockDim.x / 2; d > 0; d >>= 1) {
    if (threadIdx.x < d) {
      smin[threadIdx.x] = min(smin[threadIdx.x], smin[threadIdx.x + d]);
      smax[threadIdx.x] = max(smax[threadIdx.x], smax[threadIdx.x + d]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (smax[0] < 0) {  // no non-zero: depends on nobody
      dep[2 * b] = 1;
      dep[2 * b + 1] = 0;
      return;
    }
    // owner(p) = largest j with 32 part_t[j] <= p
    auto owner = [&](int32_t p) {
      int l = 0, h = G - 1;
      while (l < h) {
        const int m = (l + h + 1) >> 1;
        if (32 * part_t[m] <= p) l = m; else h = m - 1;
      }
      return l;
    };
    dep[2 * b] = owner(smin[0]);
    dep[2 * b + 1] = owner(smax[0]);
  }
}

// -------------------------------------------------------- equilibration --
// Nearest power of two to r > 0: r = f 2^e with f in [0.5, 1); 2^e when
// f >= sqrt(1/2), else 2^(e-1).  Zero, negative or non-finite r give 1.
__device__ __forceinline__ double nearest_pow2(double r) {
  if (!(r > 0.0) || !isfinite(r)) return 1.0;
  int e;
  const double f = frexp(r, &e);
  return f >= 0.70710678118654752440 ? ldexp(1.0, e) : ldexp(1.0, e - 1);
}

// Row 2-norms: squares summed in storage order without FMA (the oracle's order).
__global__ void k_row_norm_pow2(int32_t n, const int32_t* __restrict__ rp,
                                const double* __restrict__ va, double* d) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    double s = 0.0;
    for (int32_t k = rp[r]; k < rp[r + 1]; ++k) s = __dadd_rn(s, __dmul_rn(va[k], va[k]));
    d[r] = nearest_pow2(sqrt(s));
  }
}

// Column 2-norms of D_row^-1 A over the rows of A^T (contributions in
// increasing row order, as the oracle's scatter adds them).
__global__ void k_col_norm_pow2(int32_t n_cols, const int32_t* __restrict__ rpt,
                                const int32_t* __restrict__ cit, const double* __restrict__ vat,
                                const double* __restrict__ d_row, double* d_col) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_cols; j += stride) {
    double s = 0.0;
    for (int32_t k = rpt[j]; k < rpt[j + 1]; ++k) {
      const double a = __ddiv_rn(vat[k], d_row[cit[k]]);
      s = __dadd_rn(s, __dmul_rn(a, a));
    }
    d_col[j] = nearest_pow2(sqrt(s));
  }
}

// In-place A_hat = D_row^-1 A D_col^-1 over a CSR whose rows are the rows of A
// (row_is_a = true: entry (r, ci[k])) or the columns of A (its transpose:
// entry (ci[k], r)).  Each value is divided by its row-of-A factor, then by
// its column-of-A factor; both are powers of two, so the result is exact.
__global__ void k_scale_csr(int32_t n, const int32_t* __restrict__ rp,
                            const int32_t* __restrict__ ci, double* va,
                            const double* __restrict__ d_row, const double* __restrict__ d_col,
                            bool row_is_a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    for (int32_t k = rp[r]; k < rp[r + 1]; ++k) {
      const double dr = row_is_a ? d_row[r] : d_row[ci[k]];
      const double dc = row_is_a ? d_col[ci[k]] : d_col[r];
      va[k] = __ddiv_rn(__ddiv_rn(va[k], dr), dc);
    }
  }
}

__global__ void k_permute_factors(int32_t n, const int32_t* __restrict__ perm,
                                  const double* __restrict__ d, float* out, int* flag) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride) {
    const double v = d[perm[q]];
    if (!(v >= 0x1.0p-126 && v <= 0x1.0p+126)) atomicOr(flag, 1);
    out[q] = (float)v;
  }
}

// One thread per (slice, lane) of m: scale the lane's entries by its row
// factor and each entry's column factor, round to FP32.
__global__ void k_sell_scale32(int32_t n_rows, int32_t ns, const int32_t* __restrict__ wp,
                               const int32_t* __restrict__ col, const double* __restrict__ val,
                               const float* __restrict__ drow, const float* __restrict__ dcol,
                               float* val32) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < 32ll * ns; t += stride) {
    const int64_t s = t >> 5;
    const int lane = (int)(t & 31);
    const int64_t p = 32 * s + lane;
    const int w0 = wp[s], w = wp[s + 1] - w0;
    const double dr = p < n_rows ? (double)drow[p] : 1.0;
    for (int k = 0; k < w; ++k) {
      const int64_t e = 32ll * (w0 + k) + lane;
      val32[e] = (float)(val[e] / dr / (double)dcol[col[e]]);
    }
  }
}

__global__ void k_f32_to_f64(int64_t n, const float* __restrict__ in, double* out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = (double)in[i];
}

__global__ void k_f64_to_f32(int64_t n, const double* __restrict__ in, float* out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = (float)in[i];
}

// ------------------------------------------------------ sliced ELL build --
// Stored non-zeros per row: explicit zeros are left out of the sliced copies
// (they add nothing to a product of finite vectors), so every unpadded entry
// of a slice is a real non-zero and the neighbour dependencies are exact.
__global__ void k_row_lengths(int32_t n, const int32_t* __restrict__ rp,
                              const double* __restrict__ va, int32_t* lens) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    int32_t c = 0;
    for (int32_t k = rp[r]; k < rp[r + 1]; ++k) c += va[k] != 0.0;
    lens[r] = c;
  }
}

// One block per window of kWindow rows: bitonic sort of the keys
// (INT32_MAX - len) << 32 | local index, i.e. length descending and, among
// equal lengths, source order (a stable sort).  perm[p] = source row at
// position p; pos[row] = p.
__global__ void __launch_bounds__(kWindow / 2) k_window_sort(int32_t n,
                                                             const int32_t* __restrict__ lens,
                                                             int32_t* perm, int32_t* pos) {
  __shared__ unsigned long long key[kWindow];
  const int64_t base = (int64_t)blockIdx.x * kWindow;
  for (int i = threadIdx.x; i < kWindow; i += blockDim.x) {
    const int64_t r = base + i;
    const unsigned long long len = r < n ? (unsigned long long)lens[r] : 0ull;
    key[i] = r < n ? (((0x7fffffffull - len) << 32) | (unsigned long long)i) : ~0ull;
  }
  __syncthreads();
  for (int k = 2; k <= kWindow; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < kWindow; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const bool up = (i & k) == 0;
          const unsigned long long a = key[i], b = key[ixj];
          if ((a > b) == up) { key[i] = b; key[ixj] = a; }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < kWindow; i += blockDim.x) {
    const unsigned long long k = key[i];
    if (k != ~0ull) {
      const int32_t src = (int32_t)(base + (int64_t)(k & 0xffffffffull));
      perm[base + i] = src;
      pos[src] = (int32_t)(base + i);
    }
  }
}

// Width of each slice = length of its first (longest) row; widths[ns] = 0.
__global__ void k_slice_widths(int32_t n, int32_t ns, const int32_t* __restrict__ perm,
                               const int32_t* __restrict__ lens, int32_t* widths) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s <= ns; s += stride)
    widths[s] = (s < ns) ? lens[perm[32 * s]] : 0;
}

// One thread per (slice, lane): copy the row's non-zero entries (in CSR
// order) column-major into the slice and pad with (column 0, value 0.0) up
// to the slice width.
__global__ void k_sell_fill(int32_t n, int32_t ns, const int32_t* __restrict__ rp,
                            const int32_t* __restrict__ ci, const double* __restrict__ va,
                            const int32_t* __restrict__ perm, const int32_t* __restrict__ col_pos,
                            const int32_t* __restrict__ wp, int32_t* col, double* val) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < 32ll * ns; t += stride) {
    const int64_t s = t >> 5;
    const int lane = (int)(t & 31);
    const int64_t p = 32 * s + lane;
    const int w0 = wp[s], w = wp[s + 1] - w0;
    const int64_t out = 32ll * w0 + lane;
    int k = 0;
    if (p < n) {
      const int32_t r = perm[p];
      for (int32_t q = rp[r]; q < rp[r + 1]; ++q) {
        if (va[q] == 0.0) continue;
        col[out + 32ll * k] = col_pos[ci[q]];
        val[out + 32ll * k] = va[q];
        ++k;
      }
    }
    for (; k < w; ++k) {
      col[out + 32ll * k] = 0;
      val[out + 32ll * k] = 0.0;
    }
  }
}

__global__ void k_permute(int32_t n, const int32_t* __restrict__ pos, const double* __restrict__ in,
                          double* out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[pos[i]] = in[i];
}

// `count` vectors of length n (row-major), each mapped back to source order.
__global__ void k_unpermute(int32_t n, int32_t count, const int32_t* __restrict__ pos,
                            const double* __restrict__ in, double* out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t total = (int64_t)n * count;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
    const int64_t v = t / n, i = t - v * n;
    out[t] = in[v * n + pos[i]];
  }
}

// --------------------------------------------------------- start vector --
__global__ void __launch_bounds__(kT) k_start_raw(int32_t n, uint64_t seed,
                                                  const int32_t* __restrict__ pos, double* x,
                                                  double* blockpart) {
  __shared__ double scratch[kT];
  double q[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double u = (double)(splitmix64_at(seed, (uint64_t)i) >> 11) * 0x1.0p-53;
    const double xi = 2.0 * u - 1.0;
    x[pos ? pos[i] : i] = xi;  // pos == null: source order
    q[0] = fma(xi, xi, q[0]);
  }
  block_sum_to0<1>(q, scratch);
  if (threadIdx.x == 0) blockpart[blockIdx.x] = q[0];
}

__global__ void __launch_bounds__(kT) k_start_scale(int32_t n, double* x,
                                                    const double* blockpart, int nb) {
  __shared__ double inv;
  if (threadIdx.x < 32) {
    const double q = ordered_sum(blockpart, nb, 1, 0);
    if (threadIdx.x == 0) inv = 1.0 / sqrt(q);
  }
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= inv;
}

// ------------------------------------------------------- sliced product --
__global__ void __launch_bounds__(kT) k_sell_spmv(int32_t n, int32_t ns,
                                                  const int32_t* __restrict__ wp,
                                                  const int32_t* __restrict__ col,
                                                  const double* __restrict__ val,
                                                  const double* __restrict__ x, double* y) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < ns;
       s += warps) {
    const double a = slice_dot(wp, col, val, (int)s, lane, x);
    const int64_t p = 32 * s + lane;
    if (p < n) y[p] = a;
  }
}

// ---------------------------------------------------------------- sigma --
__device__ __forceinline__ const double* select_x(const double* X0, const double* X1,
                                                  const double* X2, int k) {
  return k == 0 ? X0 : (k == 1 ? X1 : X2);
}

template <bool DD>
__global__ void __launch_bounds__(kT) k_sigma_part(int32_t n_rows, int32_t ns, int32_t n_cols,
                                                   const int32_t* __restrict__ wp,
                                                   const int32_t* __restrict__ col,
                                                   const double* __restrict__ val,
                                                   const double* X0, const double* X1,
                                                   const double* X2, int use_minb,
                                                   const RunState* st, double* blockpart) {
  __shared__ double scratch[2 * kT];
  const double* x = select_x(X0, X1, X2, use_minb ? st->minb : 0);
  double v[2] = {0.0, 0.0};
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < ns;
       s += warps) {
    double a, lo;
    if (DD) slice_dot_dd(wp, col, val, (int)s, lane, x, a, lo);
    else a = slice_dot(wp, col, val, (int)s, lane, x);
    if (32 * s + lane < n_rows) v[0] = fma(a, a, v[0]);
  }
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_cols; j += stride)
    v[1] = fma(x[j], x[j], v[1]);
  block_sum_to0<2>(v, scratch);
  if (threadIdx.x == 0) {
    blockpart[2 * blockIdx.x] = v[0];
    blockpart[2 * blockIdx.x + 1] = v[1];
  }
}

__global__ void k_sigma_final(const double* blockpart, int nb, RunState* st) {
  const double s = ordered_sum(blockpart, nb, 2, 0);
  const double q = ordered_sum(blockpart, nb, 2, 1);
  if (threadIdx.x == 0) st->sigma = sqrt(s) / sqrt(q);
}

}  // namespace

// ====================================================== launch wrappers ==

cudaError_t launch_validate_csr(int32_t n_rows, int32_t n_cols, int64_t nnz, const int32_t* rp,
                                const int32_t* ci, int* flag, cudaStream_t s, int64_t* launches) {
  k_validate<<<grid_for(n_rows > nnz ? n_rows : nnz), kT, 0, s>>>(n_rows, n_cols, nnz, rp, ci,
                                                                   flag);
  ++*launches;
  return cudaGetLastError();
}

int scan_blocks(int64_t n) { return cdiv(n, kScanChunk) < 1 ? 1 : cdiv(n, kScanChunk); }

cudaError_t launch_transpose(int32_t n_rows, int32_t n_cols, int64_t nnz, const int32_t* rp,
                             const int32_t* ci, const double* va, int32_t* rpt, int32_t* cit,
                             double* vat, int32_t* cursor, int32_t* src, int32_t* rowid,
                             int32_t* blocksums, int* /*long_flag*/, cudaStream_t s,
                             int64_t* launches) {
  cudaError_t e = cudaMemsetAsync(cursor, 0, sizeof(int32_t) * (size_t)n_cols, s);
  if (e != cudaSuccess) return e;
  if (nnz > 0) {
    k_count_cols<<<grid_for(nnz), kT, 0, s>>>(nnz, ci, cursor);
    ++*launches;
  }
  const int nb = scan_blocks(n_cols);
  k_scan_sums<<<nb, 1024, 0, s>>>(n_cols, cursor, blocksums);
  k_scan_top<<<1, 1024, 0, s>>>(nb, blocksums);
  k_scan_apply<<<nb, 1024, 0, s>>>(n_cols, cursor, blocksums, rpt);
  *launches += 3;
  if (n_cols == 0) {
    e = cudaMemsetAsync(rpt, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
  }
  if (nnz > 0) {
    k_copy_i32<<<grid_for(n_cols), kT, 0, s>>>(n_cols, rpt, cursor);
    k_row_ids<<<grid_for(n_rows), kT, 0, s>>>(n_rows, rp, rowid);
    k_scatter<<<grid_for(nnz), kT, 0, s>>>(nnz, ci, cursor, src);
    k_segsort<<<grid_for(n_cols), kT, 0, s>>>(n_cols, rpt, src);
    k_gather_t<<<grid_for(nnz), kT, 0, s>>>(nnz, src, rowid, va, cit, vat);
    *launches += 5;
  }
  return cudaGetLastError();
}

cudaError_t launch_partition(const int32_t* wp, int32_t n_slices, int G, int row_weight,
                             int32_t* part, cudaStream_t s, int64_t* launches) {
  k_partition<<<cdiv(G + 1, kT), kT, 0, s>>>(wp, n_slices, G, row_weight, part);
  ++*launches;
  return cudaGetLastError();
}

int32_t sell_slices(int32_t n_rows) { return (n_rows + 31) / 32; }

cudaError_t launch_equilibrate(int32_t n_rows, int32_t n_cols, const int32_t* rp,
                               const double* va, const int32_t* rpt, const int32_t* cit,
                               const double* vat, double* d_row, double* d_col, cudaStream_t s,
                               int64_t* launches) {
  k_row_norm_pow2<<<grid_for(n_rows), kT, 0, s>>>(n_rows, rp, va, d_row);
  k_col_norm_pow2<<<grid_for(n_cols), kT, 0, s>>>(n_cols, rpt, cit, vat, d_row, d_col);
  *launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_scale_csr(int32_t n_rows, int32_t n_cols, const int32_t* rp,
                             const int32_t* ci, double* va, const int32_t* rpt,
                             const int32_t* cit, double* vat, const double* d_row,
                             const double* d_col, cudaStream_t s, int64_t* launches) {
  k_scale_csr<<<grid_for(n_rows), kT, 0, s>>>(n_rows, rp, ci, va, d_row, d_col, true);
  k_scale_csr<<<grid_for(n_cols), kT, 0, s>>>(n_cols, rpt, cit, vat, d_row, d_col, false);
  *launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_permute_factors(int32_t n, const int32_t* perm, const double* d, float* out,
                                   int* range_flag, cudaStream_t s, int64_t* launches) {
  k_permute_factors<<<grid_for(n), kT, 0, s>>>(n, perm, d, out, range_flag);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_sell_scale32(const Sell& m, const float* d_rowpos, const float* d_colpos,
                                float* val32, cudaStream_t s, int64_t* launches) {
  k_sell_scale32<<<grid_for(32ll * m.n_slices), kT, 0, s>>>(m.n_rows, m.n_slices, m.wp, m.col,
                                                             m.val, d_rowpos, d_colpos, val32);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_convert(int64_t n, const float* in, double* out, cudaStream_t s,
                           int64_t* launches) {
  k_f32_to_f64<<<grid_for(n), kT, 0, s>>>(n, in, out);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_convert(int64_t n, const double* in, float* out, cudaStream_t s,
                           int64_t* launches) {
  k_f64_to_f32<<<grid_for(n), kT, 0, s>>>(n, in, out);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_dependencies(const int32_t* wp, const int32_t* col, const double* val,
                                const int32_t* part_a, const int32_t* part_t, int G,
                                int32_t* dep, cudaStream_t s, int64_t* launches) {
  k_dependencies<<<G, kT, 0, s>>>(wp, col, val, part_a, part_t, G, dep);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_row_lengths(int32_t n_rows, const int32_t* rp, const double* va,
                               int32_t* lens, cudaStream_t s, int64_t* launches) {
  k_row_lengths<<<grid_for(n_rows), kT, 0, s>>>(n_rows, rp, va, lens);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_window_sort(int32_t n, const int32_t* lens, int32_t* perm, int32_t* pos,
                               cudaStream_t s, int64_t* launches) {
  k_window_sort<<<cdiv(n, kWindow), kWindow / 2, 0, s>>>(n, lens, perm, pos);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_sell_build(int32_t n_rows, const int32_t* /*rp*/, const int32_t* /*ci*/,
                              const double* /*va*/, const int32_t* lens,
                              const int32_t* /*col_pos*/, Sell* out, int32_t* widths,
                              int32_t* blocksums, int64_t* total, cudaStream_t s,
                              int64_t* launches) {
  const int32_t ns = sell_slices(n_rows);
  out->n_rows = n_rows;
  out->n_slices = ns;
  k_slice_widths<<<grid_for((int64_t)ns + 1), kT, 0, s>>>(n_rows, ns, out->perm, lens, widths);
  // exclusive scan of the ns widths: wp[0..ns-1], and wp[ns] = total
  const int nb = scan_blocks((int64_t)ns);
  k_scan_sums<<<nb, 1024, 0, s>>>((int64_t)ns, widths, blocksums);
  k_scan_top<<<1, 1024, 0, s>>>(nb, blocksums);
  k_scan_apply<<<nb, 1024, 0, s>>>((int64_t)ns, widths, blocksums, out->wp);
  *launches += 4;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int32_t tot = 0;
  e = cudaMemcpyAsync(&tot, out->wp + ns, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  *total = 32ll * tot;
  return e;
}

cudaError_t launch_sell_fill(int32_t n_rows, const int32_t* rp, const int32_t* ci,
                             const double* va, const int32_t* /*lens*/, const int32_t* col_pos,
                             const Sell& out, cudaStream_t s, int64_t* launches) {
  k_sell_fill<<<grid_for(32ll * out.n_slices), kT, 0, s>>>(n_rows, out.n_slices, rp, ci, va,
                                                            out.perm, col_pos, out.wp, out.col,
                                                            out.val);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_permute(int32_t n, const int32_t* pos, const double* in, double* out,
                           cudaStream_t s, int64_t* launches) {
  k_permute<<<grid_for(n), kT, 0, s>>>(n, pos, in, out);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_unpermute(int32_t n, int32_t count, const int32_t* pos, const double* in,
                             double* out, cudaStream_t s, int64_t* launches) {
  k_unpermute<<<grid_for((int64_t)n * count), kT, 0, s>>>(n, count, pos, in, out);
  ++*launches;
  return cudaGetLastError();
}

int start_vector_blocks(int32_t n) { return grid_for(n, kT, 152 * 4); }

cudaError_t launch_start_vector(int32_t n, uint64_t seed, const int32_t* pos, double* x,
                                double* blockpart, cudaStream_t s, int64_t* launches) {
  const int nb = start_vector_blocks(n);
  k_start_raw<<<nb, kT, 0, s>>>(n, seed, pos, x, blockpart);
  k_start_scale<<<nb, kT, 0, s>>>(n, x, blockpart, nb);
  *launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_sell_spmv(const Sell& m, const double* x, double* y, cudaStream_t s,
                             int64_t* launches) {
  if (m.n_rows == 0) return cudaSuccess;
  k_sell_spmv<<<grid_for(32ll * m.n_slices), kT, 0, s>>>(m.n_rows, m.n_slices, m.wp, m.col,
                                                          m.val, x, y);
  ++*launches;
  return cudaGetLastError();
}

int sigma_blocks(int32_t n_slices, int32_t n_cols) {
  const int64_t a = 32ll * n_slices, b = n_cols;
  return grid_for(a > b ? a : b, kT, 152 * 4);
}

cudaError_t launch_sigma(const Sell& m, int32_t n_cols, const double* X0, const double* X1,
                         const double* X2, int use_minb, RunState* st, double* blockpart,
                         bool dd, cudaStream_t s, int64_t* launches) {
  const int nb = sigma_blocks(m.n_slices, n_cols);
  if (dd)
    k_sigma_part<true><<<nb, kT, 0, s>>>(m.n_rows, m.n_slices, n_cols, m.wp, m.col, m.val, X0,
                                         X1, X2, use_minb, st, blockpart);
  else
    k_sigma_part<false><<<nb, kT, 0, s>>>(m.n_rows, m.n_slices, n_cols, m.wp, m.col, m.val, X0,
                                          X1, X2, use_minb, st, blockpart);
  k_sigma_final<<<1, 32, 0, s>>>(blockpart, nb, st);
  *launches += 2;
  return cudaGetLastError();
}

}  // namespace pa
