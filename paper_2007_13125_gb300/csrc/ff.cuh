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

// ---- double-float scalar and complex arithmetic (used by the FFTs of the CQ history) ----
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  ff r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff{-b.hi, -b.lo}); }
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  ff r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}

// complex double-float: (rh + rl) + i (ih + il)
struct ffc { float rh, rl, ih, il; };

__device__ __forceinline__ ffc ffc_make(ff re, ff im) { return ffc{re.hi, re.lo, im.hi, im.lo}; }
__device__ __forceinline__ ff ffc_re(ffc a) { return ff{a.rh, a.rl}; }
__device__ __forceinline__ ff ffc_im(ffc a) { return ff{a.ih, a.il}; }
__device__ __forceinline__ ffc cadd(ffc a, ffc b) {
  return ffc_make(ff_add(ffc_re(a), ffc_re(b)), ff_add(ffc_im(a), ffc_im(b)));
}
__device__ __forceinline__ ffc csub(ffc a, ffc b) {
  return ffc_make(ff_sub(ffc_re(a), ffc_re(b)), ff_sub(ffc_im(a), ffc_im(b)));
}
__device__ __forceinline__ ffc cmul(ffc a, ffc b) {
  const ff ar = ffc_re(a), ai = ffc_im(a), br = ffc_re(b), bi = ffc_im(b);
  return ffc_make(ff_sub(ff_mul(ar, br), ff_mul(ai, bi)), ff_add(ff_mul(ar, bi), ff_mul(ai, br)));
}
__device__ __forceinline__ ffc cmulc(ffc a, ffc b) {  // a * conj(b)
  const ff ar = ffc_re(a), ai = ffc_im(a), br = ffc_re(b), bi = ffc_im(b);
  return ffc_make(ff_add(ff_mul(ar, br), ff_mul(ai, bi)), ff_sub(ff_mul(ai, br), ff_mul(ar, bi)));
}

// Lazy complex double-float for FFT butterflies (the CQ history's transforms): the same
// unevaluated sums hi + lo, but sums and products skip the renormalisation, so within one FFT
// pass a low part may reach a few ulp of its high part. Every rounding error stays of order
// 2^-48 of the magnitudes entering the operation (the norm-wise error model of an FFT); the pass
// renormalises each value once when it stores it (fft_store, with an exact two_sum).
struct ffz { float rh, rl, ih, il; };
__device__ __forceinline__ void lazy_add(float ah, float al, float bh, float bl, float& sh, float& sl) {
  float e;
  two_sum(ah, bh, sh, e);
  sl = __fadd_rn(e, __fadd_rn(al, bl));
}
__device__ __forceinline__ void lazy_mul(float ah, float al, float bh, float bl, float& ph, float& pl) {
  ph = __fmul_rn(ah, bh);
  pl = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, __fmaf_rn(ah, bh, -ph)));
}
__device__ __forceinline__ ffz cadd(ffz a, ffz b) {
  ffz r;
  lazy_add(a.rh, a.rl, b.rh, b.rl, r.rh, r.rl);
  lazy_add(a.ih, a.il, b.ih, b.il, r.ih, r.il);
  return r;
}
__device__ __forceinline__ ffz csub(ffz a, ffz b) {
  ffz r;
  lazy_add(a.rh, a.rl, -b.rh, -b.rl, r.rh, r.rl);
  lazy_add(a.ih, a.il, -b.ih, -b.il, r.ih, r.il);
  return r;
}
__device__ __forceinline__ ffz cmul(ffz a, ffz b) {
  float p1h, p1l, p2h, p2l, p3h, p3l, p4h, p4l;
  lazy_mul(a.rh, a.rl, b.rh, b.rl, p1h, p1l);  // ar br
  lazy_mul(a.ih, a.il, b.ih, b.il, p2h, p2l);  // ai bi
  lazy_mul(a.rh, a.rl, b.ih, b.il, p3h, p3l);  // ar bi
  lazy_mul(a.ih, a.il, b.rh, b.rl, p4h, p4l);  // ai br
  ffz r;
  lazy_add(p1h, p1l, -p2h, -p2l, r.rh, r.rl);
  lazy_add(p3h, p3l, p4h, p4l, r.ih, r.il);
  return r;
}
__device__ __forceinline__ ffz cmulc(ffz a, ffz b) {  // a * conj(b)
  float p1h, p1l, p2h, p2l, p3h, p3l, p4h, p4l;
  lazy_mul(a.rh, a.rl, b.rh, b.rl, p1h, p1l);  // ar br
  lazy_mul(a.ih, a.il, b.ih, b.il, p2h, p2l);  // ai bi
  lazy_mul(a.ih, a.il, b.rh, b.rl, p3h, p3l);  // ai br
  lazy_mul(a.rh, a.rl, b.ih, b.il, p4h, p4l);  // ar bi
  ffz r;
  lazy_add(p1h, p1l, p2h, p2l, r.rh, r.rl);
  lazy_add(p3h, p3l, -p4h, -p4l, r.ih, r.il);
  return r;
}
__device__ __forceinline__ ffz fft_store(ffz v) {
  ffz r;
  two_sum(v.rh, v.rl, r.rh, r.rl);
  two_sum(v.ih, v.il, r.ih, r.il);
  return r;
}

// Split a double into hi + lo with integer operations only. On GB300 every FP64<->FP32
// conversion runs at the FP64 rate (~1/70 of FP32), so the bit patterns are taken apart
// directly: hi = x rounded to 24 significant bits (nearest, ties to even), exact as a float;
// the remainder x - hi is an integer of at most 29 bits in units of 2^(e-1075), converted to
// float (rounded: lo keeps 24 of those bits) and scaled: |hi + lo - x| <= 2^-48 |x| for
// |x| in [2^-74, 2^127). Below 2^-74 lo is dropped (hi stays exact down to 2^-126) and below
// 2^-126 the result is 0: absolute errors under 1e-37, far below every term of the method.
__device__ __forceinline__ ff ff_from_double(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned long long mag = b & 0x7FFFFFFFFFFFFFFFull;
  const int e = (int)(mag >> 52);
  ff r;
  if (e < 897) { r.hi = 0.f; r.lo = 0.f; return r; }
  const unsigned int sgn = (unsigned int)(b >> 32) & 0x80000000u;
  // round away the low 29 mantissa bits (nearest-even); a carry moves into the exponent
  const unsigned long long rm = (mag + 0x0FFFFFFFull + ((mag >> 29) & 1ull)) & ~0x1FFFFFFFull;
  const unsigned int er = (unsigned int)(rm >> 52);
  const unsigned int fm = (unsigned int)(rm >> 29) & 0x7FFFFFu;
  r.hi = __uint_as_float(sgn | ((er - 896u) << 23) | fm);
  // remainder in units of 2^(e-1075); |d| <= 2^28. Bit-pattern differences equal value
  // differences in those units even when the rounding carried into the exponent.
  const int d = (int)((long long)mag - (long long)rm);
  const int se = e - 948;  // biased float exponent of 2^(e-1075)
  const float scale = se >= 1 ? __uint_as_float((unsigned int)se << 23) : 0.f;
  const float lo = __int2float_rn(d) * scale;
  r.lo = sgn ? -lo : lo;
  return r;
}

// FP64 -> double-float by truncation, from the two 32-bit halves of the double: hi keeps the
// leading 24 significant bits (exact as a float), lo is the remaining 29-bit integer scaled by
// 2^(e-1075) and rounded once to 24 bits: |hi + lo - x| <= 2^-47 |x| for |x| in [2^-74, 2^127),
// |lo| < ulp(hi) (not normalised: fine as the start of an accumulation). Cheaper than
// ff_from_double (no 64-bit rounding carry). Below 2^-74 lo is dropped, below 2^-126 all is 0.
__device__ __forceinline__ ff ff_split_trunc(double x) {
  const unsigned h = (unsigned)__double2hiint(x), l = (unsigned)__double2loint(x);
  const unsigned e = (h >> 20) & 0x7FFu;
  const unsigned sgn = h & 0x80000000u;
  ff r;
  const unsigned hb = sgn | ((e - 896u) << 23) | ((h & 0xFFFFFu) << 3) | (l >> 29);
  r.hi = e >= 897u ? __uint_as_float(hb) : 0.f;
  const float scale = e >= 949u ? __uint_as_float((e - 948u) << 23) : 0.f;
  const float lo = __uint2float_rn(l & 0x1FFFFFFFu) * scale;
  r.lo = __uint_as_float(__float_as_uint(lo) | sgn);
  return r;
}

// Exact float -> double by bit construction (no FP64 conversion instruction).
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int ex = (u >> 23) & 0xFFu;
  if (ex == 0) return 0.0;  // zero (float subnormals flushed)
  const unsigned long long hi = ((unsigned long long)(u & 0x80000000u) << 32) |
                                ((unsigned long long)(ex + 896u) << 52) |
                                ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)hi);
}

// hi + lo as a double: two exact bit constructions and one FP64 add.
__device__ __forceinline__ double ff_to_double(ff x) { return f2d_bits(x.hi) + f2d_bits(x.lo); }

}  // namespace pint
