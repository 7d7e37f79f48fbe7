// pa_df.cuh -- double-float ("double-word") arithmetic on the FP32 pipe.
//
// A value is an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits with FP32's exponent range.  GB300 issues FP32
// fused multiply-adds 64 times faster than FP64 ones, so the Projected Adam
// iteration of the PA_DF64 precision mode carries its products and its
// per-row Adam arithmetic in this form and keeps only the reductions in FP64.
//
// The building blocks are the published error-free transformations and
// double-word algorithms, written here from their definitions:
//   * TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s + e = a + b exactly;
//   * Fast2Sum (Dekker 1971, "A floating-point technique for extending the
//     available precision"): the same when |a| >= |b| or a = 0;
//   * TwoProd with one FMA: p + e = a b exactly (no underflow);
//   * DW+DW, DW*DW, DW*FP and DW/DW as analysed by Joldes, Muller and Popescu,
//     "Tight and rigorous error bounds for basic building blocks of
//     double-word arithmetic", ACM TOMS 44 (2017): the accurate sum (relative
//     error below 3u^2, u = 2^-24), the FMA product (below 4u^2), the
//     product by a float (below 2u^2) and the quotient through one float
//     division and a correction (below 15u^2);
//   * the square root by one correction of the correctly rounded FP32 root
//     (Karp and Markstein, "High-precision division and square root", ACM
//     TOMS 23, 1997).
// Every addition and multiplication is written with the _rn intrinsics so
// that the compiler cannot contract or reassociate them.
#pragma once

#include <cuda_runtime.h>

namespace pa {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_make(float hi, float lo) { return df{hi, lo}; }

__device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df{s, e};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df df_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return df{p, __fmaf_rn(a, b, -p)};
}

// accurate double-word sum (relative error < 3u^2)
__device__ __forceinline__ df df_add(df x, df y) {
  const df s = df_two_sum(x.hi, y.hi);
  const df t = df_two_sum(x.lo, y.lo);
  const df v = df_fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return df_fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}

__device__ __forceinline__ df df_neg(df x) { return df{-x.hi, -x.lo}; }
__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }

// double-word times double-word with FMA (relative error < 4u^2)
__device__ __forceinline__ df df_mul(df x, df y) {
  const df c = df_two_prod(x.hi, y.hi);
  const float t = __fmaf_rn(x.hi, y.lo, __fmul_rn(x.lo, y.lo));
  const float cl = __fadd_rn(c.lo, __fmaf_rn(x.lo, y.hi, t));
  return df_fast_two_sum(c.hi, cl);
}

// double-word times float (relative error < 2u^2)
__device__ __forceinline__ df df_mul_f(df x, float y) {
  const df c = df_two_prod(x.hi, y);
  return df_fast_two_sum(c.hi, __fmaf_rn(x.lo, y, c.lo));
}

// double-word quotient: one float division, the residual x - q y in
// double-word, a second division for the correction (relative error < 15u^2)
__device__ __forceinline__ df df_div(df x, df y) {
  const float th = __fdiv_rn(x.hi, y.hi);
  const df r = df_mul_f(y, th);
  const float ph = __fsub_rn(x.hi, r.hi);  // exact (Sterbenz): r.hi is close to x.hi
  const float dl = __fsub_rn(x.lo, r.lo);
  const float tl = __fdiv_rn(__fadd_rn(ph, dl), y.hi);
  return df_fast_two_sum(th, tl);
}

// square root of a non-negative double-word: the correctly rounded float
// root s0 of x.hi, the residual x - s0^2 (s0^2 exactly by TwoProd), and one
// correction residual / (2 s0)
__device__ __forceinline__ df df_sqrt(df x) {
  if (!(x.hi > 0.f)) return df{0.f, 0.f};
  const float s0 = __fsqrt_rn(x.hi);
  const df p = df_two_prod(s0, s0);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p.hi), p.lo), x.lo);
  return df_fast_two_sum(s0, __fdiv_rn(r, __fmul_rn(2.f, s0)));
}

// FP64 -> double-word: hi = float(d), lo = float(d - hi).  The difference is
// formed in FP64 (exact), so this is for set-up and boundary conversions,
// not for the loop.
__device__ __forceinline__ df df_from_double(double d) {
  const float hi = __double2float_rn(d);
  return df{hi, __double2float_rn(d - (double)hi)};
}

__device__ __forceinline__ double df_to_double(df x) { return (double)x.hi + (double)x.lo; }

__device__ __forceinline__ df df_load(const float2* p) {
  const float2 v = *p;
  return df{v.x, v.y};
}
__device__ __forceinline__ df df_ldg(const float2* p) {
  const float2 v = __ldg(p);
  return df{v.x, v.y};
}
__device__ __forceinline__ void df_store(float2* p, df x) { *p = make_float2(x.hi, x.lo); }

// Running sum of products a_k x_k: each product split exactly by TwoProd
// plus its cross terms, the high parts added by TwoSum, every low part
// collected in one float; renormalised once at the end.
struct DfAcc {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add_prod(df a, df x) {
    const df p = df_two_prod(a.hi, x.hi);
    const float e = __fmaf_rn(a.hi, x.lo, __fmaf_rn(a.lo, x.hi, p.lo));
    const df t = df_two_sum(s, p.hi);
    s = t.hi;
    c = __fadd_rn(c, __fadd_rn(t.lo, e));
  }
  __device__ __forceinline__ void add(df x) {
    const df t = df_two_sum(s, x.hi);
    s = t.hi;
    c = __fadd_rn(c, __fadd_rn(t.lo, x.lo));
  }
  __device__ __forceinline__ df value() const { return df_fast_two_sum(s, c); }
};

}  // namespace pa
