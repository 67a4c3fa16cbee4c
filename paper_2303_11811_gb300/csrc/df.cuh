// df.cuh -- double-float arithmetic: a value is the unevaluated sum hi + lo of
// two FP32 numbers.  GB300 executes FP64 at 1/64 of its FP32 rate; the
// collision in this form runs on the FP32 pipes while keeping the PDFs to
// about 2^-47 relative precision.
//
// The operations are the error-free transformations of Knuth (TwoSum, 1969)
// and Dekker (Fast2Sum and the exact product, 1971), the product's error term
// taken from a fused multiply-add, as in the double-float arithmetic of Hida,
// Li and Bailey (QD library, ARITH 2001), but without renormalising each
// result (the compensated form of Ogita, Rump and Oishi, SIAM J. Sci. Comput.
// 2005): a sum keeps the exact error of its high parts plus the sum of the low
// parts, a product the exact error of the high product plus the cross terms.
// Each operation then errs by about 2^-47 of its operands' magnitude rather
// than of its result; the collision's inputs and outputs are deviations from
// the lattice weights, small next to the PDFs themselves, so this stays far
// below the FP64 path's bound on the PDFs.  Stored values are renormalised
// (renorm) so that the low part never accumulates over time steps.  Every
// FP32 step is an explicitly rounded intrinsic, so the compiler cannot
// contract or reassociate them.
#pragma once
#include <cuda_runtime.h>

namespace psm {

struct __align__(8) df {
  float hi, lo;
  df() = default;
  // exact split of a double into its nearest float and the rounded remainder
  __host__ __device__ constexpr explicit df(double d)
      : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
};

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df(s, e);
}
// |a| >= |b| or a = 0
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ df operator+(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  return df(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df(p, e);
}
// canonical pair: hi the FP32 rounding of hi + lo (exact for any magnitudes)
__device__ __forceinline__ df renorm(df a) { return two_sum(a.hi, a.lo); }
// the same by Fast2Sum, for results of a sum or product (|lo| <= a few
// ulp(hi); after a cancellation where |lo| > |hi| the pair is still put back
// into canonical form, its value kept to within ulp(lo), the form's own
// precision)
__device__ __forceinline__ df renorm_fast(df a) { return fast_two_sum(a.hi, a.lo); }
__device__ __forceinline__ df& operator+=(df& a, df b) { return a = a + b; }
__device__ __forceinline__ bool operator>(df a, df b) {
  a = renorm(a);
  b = renorm(b);
  return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo);
}
__device__ __forceinline__ double to_double(df a) { return (double)a.hi + (double)a.lo; }

}  // namespace psm
