// pa_bounds.cu -- kernels of pa_error_bounds: the residual of an approximate
// solution x_hat of A x = b and the error bounds of the paper's section
// "Error estimates and conditioning" (Theorems 1-4).
//
// The residual r_i = sum_k a_ik x_hat_k - b_i is accumulated in Dot2
// (Ogita, Rump & Oishi 2005): the row's products in CSR order, then -b_i as
// one more term, then s + c.  A plainly accumulated residual of a good
// solution of an ill-conditioned system is mostly rounding noise of A x_hat;
// the compensated one keeps the digits the bounds depend on.  The norms are
// reduced in a fixed order (per-block partials, then one ordered sum), so a
// call is bit-reproducible.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "pa_device.cuh"
#include "pa_internal.h"

namespace pa {

namespace {

constexpr int kRB = 256;

__global__ void __launch_bounds__(kRB)
    k_residual_part(int32_t n_rows, int32_t n_cols, const int32_t* __restrict__ rp,
                    const int32_t* __restrict__ ci, const double* __restrict__ va,
                    const double* __restrict__ x, const double* __restrict__ bv, double* part) {
  __shared__ double sh[3 * kRB];
  double v[3] = {0.0, 0.0, 0.0};  // ||r||^2, ||b||^2, ||x_hat||^2
  const int64_t n = n_rows > n_cols ? n_rows : n_cols;
  const int64_t stride = (int64_t)gridDim.x * kRB;
  for (int64_t i = (int64_t)blockIdx.x * kRB + threadIdx.x; i < n; i += stride) {
    if (i < n_rows) {
      double s = 0.0, c = 0.0, t, te;
      for (int32_t k = rp[i]; k < rp[i + 1]; ++k) dot2_step(va[k], x[ci[k]], s, c);
      two_sum(s, -bv[i], t, te);
      s = t;
      c = __dadd_rn(c, te);
      const double r = __dadd_rn(s, c);
      v[0] = fma(r, r, v[0]);
      v[1] = fma(bv[i], bv[i], v[1]);
    }
    if (i < n_cols) v[2] = fma(x[i], x[i], v[2]);
  }
  block_sum_to0<3>(v, sh);
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x + 0] = v[0];
    part[3 * blockIdx.x + 1] = v[1];
    part[3 * blockIdx.x + 2] = v[2];
  }
}

// The theorem formulas, in the order of the output vector of pa_error_bounds.
__global__ void k_bounds_final(const double* part, int nb, double kappa, double norm_a, double u,
                               double* out) {
  const double nr = sqrt(ordered_sum(part, nb, 3, 0));
  const double nb2 = sqrt(ordered_sum(part, nb, 3, 1));
  const double nx = sqrt(ordered_sum(part, nb, 3, 2));
  if (threadIdx.x != 0) return;
  out[0] = nr;
  out[1] = nb2;
  out[2] = nx;
  // Theorem 1: ||x_hat - x|| / ||x|| within [rel / kappa, kappa rel], rel = ||r|| / ||b||
  out[3] = (nr / nb2) / kappa;
  out[4] = kappa * (nr / nb2);
  // Theorem 2: ||x_hat - x|| / ||x_hat|| within [||r|| / (||A|| ||x_hat||), eps]
  out[5] = nr / (norm_a * nx);
  const double eps = kappa * (nr / (norm_a * nx));
  out[6] = eps;
  // Theorem 3: ||x_hat - x|| / ||x|| <= eps / (1 - eps) while eps < 1
  out[7] = eps < 1.0 ? eps / (1.0 - eps) : INFINITY;
  // Theorem 4: rounding at precision u costs at most 2 u kappa / (1 - kappa u);
  // kappa u >= 1 means A is numerically singular at that precision
  const double ku = kappa * u;
  out[8] = ku < 1.0 ? 2.0 * u * kappa / (1.0 - ku) : INFINITY;
  out[9] = ku >= 1.0 ? 1.0 : 0.0;
}

}  // namespace

int error_bound_blocks(int64_t n) {
  const int64_t want = (n + kRB - 1) / kRB;
  return (int)(want < kErrorBoundMaxBlocks ? (want > 0 ? want : 1) : kErrorBoundMaxBlocks);
}

cudaError_t launch_error_bounds(int32_t n_rows, int32_t n_cols, const int32_t* rp,
                                const int32_t* ci, const double* va, const double* x_hat,
                                const double* b, double kappa, double norm_a, double u,
                                double* part, double* out, cudaStream_t s, int64_t* launches) {
  const int nb = error_bound_blocks(n_rows > n_cols ? n_rows : n_cols);
  k_residual_part<<<nb, kRB, 0, s>>>(n_rows, n_cols, rp, ci, va, x_hat, b, part);
  k_bounds_final<<<1, 32, 0, s>>>(part, nb, kappa, norm_a, u, out);
  *launches += 2;
  return cudaGetLastError();
}

}  // namespace pa
