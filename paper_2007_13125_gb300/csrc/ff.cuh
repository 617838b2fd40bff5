// Double-float ("ff") arithmetic: a value is the unevaluated sum hi + lo of two floats,
// |lo| <= ulp(hi)/2, giving a ~48-bit significand. The all-at-once residual F_hat - K U
// of the refinement loop needs ~1e-13 relative accuracy in its largest terms; on GB300
// the FP32 pipes are ~64x faster than FP64, so the residual is evaluated with these
// error-free transformations on FP32 hardware instead of in native FP64.
//
// two_sum / fast_two_sum are Knuth's and Dekker's exact-addition transformations; two_prod
// uses a fused multiply-add to obtain the exact rounding error of a product.
#pragma once
#include <cuda_runtime.h>

namespace pint {

struct ff { float hi, lo; };

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// Accumulator of many terms: exact running sum of the high parts (two_sum chain) plus a
// float accumulator for everything of order eps * |term|.
struct ff_acc {
  float sh, sl;
  __device__ __forceinline__ void init(ff x) { sh = x.hi; sl = x.lo; }
  __device__ __forceinline__ void add_hi(float t) {
    float s, e;
    two_sum(sh, t, s, e);
    sh = s;
    sl = __fadd_rn(sl, e);
  }
  __device__ __forceinline__ void add(ff x) {
    add_hi(x.hi);
    sl = __fadd_rn(sl, x.lo);
  }
  __device__ __forceinline__ void sub(ff x) {
    add_hi(-x.hi);
    sl = __fsub_rn(sl, x.lo);
  }
  // acc += sign * c * u   (c, u double-float; error O(eps^2 |c u|))
  __device__ __forceinline__ void fma_term(ff c, ff u, float sign) {
    float p = __fmul_rn(c.hi, u.hi);
    float pe = __fmaf_rn(c.hi, u.hi, -p);                 // exact error of the product
    float low = __fmaf_rn(c.hi, u.lo, __fmaf_rn(c.lo, u.hi, pe));
    add_hi(sign * p);
    sl = __fmaf_rn(sign, low, sl);
  }
  __device__ __forceinline__ float value() const { return __fadd_rn(sh, sl); }
  __device__ __forceinline__ ff normalized() const {
    ff r;
    fast_two_sum(sh, sl, r.hi, r.lo);
    return r;
  }
};

// x + c for a double-float x and a float c
__device__ __forceinline__ ff ff_add_f(ff x, float c) {
  float s, e;
  two_sum(x.hi, c, s, e);
  e = __fadd_rn(e, x.lo);
  ff r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

// exact split of a double into hi = rn(x), lo = rn(x - hi)
__device__ __forceinline__ ff ff_from_double(double x) {
  ff r;
  r.hi = __double2float_rn(x);
  r.lo = __double2float_rn(x - (double)r.hi);
  return r;
}

__device__ __forceinline__ double ff_to_double(ff x) { return (double)x.hi + (double)x.lo; }

}  // namespace pint
