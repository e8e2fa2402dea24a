// Double-float ("df64") arithmetic: a value is the unevaluated sum hi + lo of
// two fp32 numbers with |lo| <= ulp(hi)/2, about 48 significant bits.  It
// runs on the fp32 pipes, which on this GPU issue 58x more operations per
// clock than the fp64 pipe.
//
// Building blocks (error-free transformations):
//   * Knuth's TwoSum: s = fl(a + b), e = (a - (s - v)) + (b - v), v = s - a,
//     gives a + b = s + e exactly;
//   * the FMA product error: p = fl(a b), e = fma(a, b, -p) gives a b = p + e.
// A df64 value occupies the same 8 bytes as a double (float2 {hi, lo}).
#pragma once

#include <cuda_runtime.h>

namespace rsf {

struct df64 {
  float hi, lo;
};

__device__ __forceinline__ df64 df_from_double(double d) {
  float h = __double2float_rn(d);
  float l = __double2float_rn(d - (double)h);
  return {h, l};
}

__device__ __forceinline__ double df_to_double(df64 a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df64 df_fast_two_sum(float s, float e) {
  float h = __fadd_rn(s, e);
  float l = __fsub_rn(e, __fsub_rn(h, s));
  return {h, l};
}

__device__ __forceinline__ df64 df_add(df64 a, df64 b) {
  float s = __fadd_rn(a.hi, b.hi);
  float v = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df_fast_two_sum(s, e);
}

// a * f for an fp32 scalar f (exact for powers of two)
__device__ __forceinline__ df64 df_scale(df64 a, float f) {
  float p = __fmul_rn(a.hi, f);
  float e = __fmaf_rn(a.hi, f, -p);
  e = __fmaf_rn(a.lo, f, e);
  return df_fast_two_sum(p, e);
}

// Accumulator for sums of products: hi carries the running fp32 sum, lo the
// accumulated rounding errors (of the products and of the additions).
struct dfacc {
  float hi, lo;
};

__device__ __forceinline__ void df_mac(dfacc& c, df64 a, df64 b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float s = __fadd_rn(c.hi, p);
  float v = __fsub_rn(s, c.hi);
  float t = __fadd_rn(__fsub_rn(c.hi, __fsub_rn(s, v)), __fsub_rn(p, v));
  c.hi = s;
  c.lo = __fadd_rn(c.lo, __fadd_rn(t, e));
}

__device__ __forceinline__ df64 df_of_acc(dfacc c) { return df_fast_two_sum(c.hi, c.lo); }

}  // namespace rsf
