// Float-float arithmetic (Dekker 1971; Knuth, TAOCP vol. 2, 4.2.2) on the FP32 pipes: a
// value is the unevaluated sum hi + lo of two floats, |lo| <= ulp(hi) / 2, about 48
// significant bits. Products use the exact FMA residual of hi * hi; sums use TwoSum. Every
// operation uses the explicitly rounded intrinsics, so no multiply-add contraction alters
// them. On GB300 the FP32 pipes issue ~60x the FP64 rate, which makes these 10-15 instruction
// sequences several times faster than FP64 arithmetic.
#pragma once
#include <cuda_runtime.h>

namespace mrd {

struct FF {
  float hi, lo;
};

__device__ __forceinline__ FF ff_from(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}

// accumulator s + c: s collects the rounded partial sums, c their TwoSum errors and the
// low-order parts of the products
struct FFAcc {
  float s, c;
};

// acc += x * y
__device__ __forceinline__ void ff_mac(FFAcc& a, FF x, FF y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);         // x.hi * y.hi = p + e exactly
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  const float s = __fadd_rn(a.s, p);           // TwoSum(a.s, p)
  const float bp = __fsub_rn(s, a.s);
  const float err = __fadd_rn(__fsub_rn(a.s, __fsub_rn(s, bp)), __fsub_rn(p, bp));
  a.s = s;
  a.c = __fadd_rn(a.c, __fadd_rn(err, e));
}

// acc += x * c for an FP32 coefficient c (exact product of c with both parts of x)
__device__ __forceinline__ void ff_mac1(FFAcc& a, FF x, float c) {
  const float p = __fmul_rn(c, x.hi);
  float e = __fmaf_rn(c, x.hi, -p);
  e = __fmaf_rn(c, x.lo, e);
  const float s = __fadd_rn(a.s, p);
  const float bp = __fsub_rn(s, a.s);
  const float err = __fadd_rn(__fsub_rn(a.s, __fsub_rn(s, bp)), __fsub_rn(p, bp));
  a.s = s;
  a.c = __fadd_rn(a.c, __fadd_rn(err, e));
}

// x * c for an FP32 coefficient c as an accumulator (the exact product: no sum to form yet)
__device__ __forceinline__ FFAcc ff_prod1(FF x, float c) {
  const float p = __fmul_rn(c, x.hi);
  float e = __fmaf_rn(c, x.hi, -p);
  e = __fmaf_rn(c, x.lo, e);
  return {p, e};
}

// a * b of two FP32 numbers, exactly, as a float-float value
__device__ __forceinline__ FF ff_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ FF ff_norm(FFAcc a) {  // FastTwoSum(s, c)
  const float h = __fadd_rn(a.s, a.c);
  return {h, __fsub_rn(a.c, __fsub_rn(h, a.s))};
}

__device__ __forceinline__ FF ff_neg(FF a) { return {-a.hi, -a.lo}; }

// a + b (TwoSum of the high parts, low parts added to the error)
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bp = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bp)), __fsub_rn(b.hi, bp));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  const float h = __fadd_rn(s, e);
  return {h, __fsub_rn(e, __fsub_rn(h, s))};
}

__device__ __forceinline__ FF ff_warp_sum(FF v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const FF w = {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = ff_add(v, w);
  }
  return v;
}

}  // namespace mrd
