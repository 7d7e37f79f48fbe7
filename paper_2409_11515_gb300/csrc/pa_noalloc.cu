// pa_noalloc.cu -- pa_sigma_noalloc: sigma = ||A x|| / ||x|| for a CSR matrix
// and a vector that the caller already holds in device memory, computed
// without allocating any memory.
//
// It is a variant of the library's sigma kernel (the last step of every
// Projected Adam run): the same deterministic two-stage reduction, but reading
// the caller's CSR directly and keeping its per-block partial sums in a
// file-scope device array instead of handle-owned buffers.
//
// Why: some callers cannot allocate device memory at the point where they
// need a norm -- for instance code whose device memory is entirely reserved
// by another allocator (a framework's caching pool), or loops that must not
// pay cudaMalloc's implicit device-wide synchronisation.  This entry point
// calls no cudaMalloc, cudaFree or allocating library routine.
//
// The scratch array below is loaded with the library and stays resident on
// every GPU that loads it until the process exits.  Every call shares it and
// it keeps the previous call's contents; each call writes every partial it
// later reads, so nothing has to start at zero.  Calls whose kernels overlap
// on the GPU (different streams, no ordering between them) race on the array.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "pa.h"
#include "pa_device.cuh"
#include "pa_internal.h"

namespace {

constexpr int kNoAllocThreads = 256;   // one row (and one column) per thread
constexpr int kNoAllocMaxBlocks = 8192;
constexpr int kMaxDevices = 64;

// Two partial sums per block: sum of (A x)_i^2 and sum of x_j^2.  128 KiB.
static __device__ __align__(256) double g_sigma_scratch[2 * kNoAllocMaxBlocks];

std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// Host code cannot use g_sigma_scratch's name as a device address; look the
// address up once per device, with that device current.  The cached address
// belongs to the device's primary context (the one the CUDA runtime uses):
// after a cudaDeviceReset, or from a context created through the driver API,
// it is stale, which the header states as a condition of use.
cudaError_t scratch_address(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_sigma_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// Block b covers rows and columns [256 b, 256 b + 256): one row dot product
// (entries in storage order) and one x_j^2 per thread, block sums in a fixed
// order into scratch[2b], scratch[2b+1].
__global__ void __launch_bounds__(kNoAllocThreads)
    k_csr_sigma_part(int32_t n_rows, int32_t n_cols, const int32_t* __restrict__ rp,
                     const int32_t* __restrict__ ci, const double* __restrict__ va,
                     const double* __restrict__ x, double* scratch) {
  __shared__ double sh[2 * kNoAllocThreads];
  const int64_t i = (int64_t)blockIdx.x * kNoAllocThreads + threadIdx.x;
  double v[2] = {0.0, 0.0};
  if (i < n_rows) {
    const double yi = pa::row_dot(ci, va, __ldg(rp + i), __ldg(rp + i + 1), x);
    v[0] = yi * yi;
  }
  if (i < n_cols) v[1] = x[i] * x[i];
  pa::block_sum_to0<2>(v, sh);
  if (threadIdx.x == 0) {
    scratch[2 * blockIdx.x] = v[0];
    scratch[2 * blockIdx.x + 1] = v[1];
  }
}

__global__ void k_csr_sigma_final(const double* scratch, int nb, double* sigma) {
  const double s = pa::ordered_sum(scratch, nb, 2, 0);
  const double q = pa::ordered_sum(scratch, nb, 2, 1);
  if (threadIdx.x == 0) *sigma = sqrt(s) / sqrt(q);
}

}  // namespace

extern "C" pa_status pa_sigma_noalloc(int32_t n_rows, int32_t n_cols, const int32_t* row_ptr,
                                      const int32_t* col_idx, const double* vals, const double* x,
                                      double* sigma, void* cuda_stream) {
  const int64_t n = n_rows > n_cols ? n_rows : n_cols;
  const int64_t max_n = (int64_t)kNoAllocThreads * kNoAllocMaxBlocks;
  if (n_rows <= 0 || n_cols <= 0 || !row_ptr || !col_idx || !vals || !x || !sigma)
    return pa::set_error(PA_ERR_INVALID_ARG, "pa_sigma_noalloc: empty matrix or NULL pointer");
  if (n > max_n)
    return pa::set_error(PA_ERR_INVALID_ARG,
                         "pa_sigma_noalloc: max(n_rows, n_cols) = %lld exceeds the fixed scratch "
                         "limit of %lld",
                         (long long)n, (long long)max_n);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return pa::set_error(PA_ERR_CUDA, "pa_sigma_noalloc: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices)
    return pa::set_error(PA_ERR_UNSUPPORTED, "pa_sigma_noalloc: device %d out of range", dev);
  double* scratch = nullptr;
  if ((e = scratch_address(dev, &scratch)) != cudaSuccess)
    return pa::set_error(PA_ERR_CUDA, "pa_sigma_noalloc: scratch address: %s", cudaGetErrorString(e));
  const int nb = (int)((n + kNoAllocThreads - 1) / kNoAllocThreads);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  k_csr_sigma_part<<<nb, kNoAllocThreads, 0, s>>>(n_rows, n_cols, row_ptr, col_idx, vals, x,
                                                   scratch);
  k_csr_sigma_final<<<1, 32, 0, s>>>(scratch, nb, sigma);
  if ((e = cudaGetLastError()) != cudaSuccess)
    return pa::set_error(PA_ERR_CUDA, "pa_sigma_noalloc: launch: %s", cudaGetErrorString(e));
  return PA_OK;
}
