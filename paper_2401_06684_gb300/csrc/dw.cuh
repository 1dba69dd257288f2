// Double-word ("double-float") arithmetic on the FP32 pipes.
//
// GB300 executes FP64 at 1/64 of its FP32 rate, so an FP64 stencil or
// Gram-Schmidt sweep is bound by the FP64 ALU long before HBM.  A value is
// kept as an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2
// (about 48 significand bits, the same 8 bytes as an FP64).  The building
// blocks are the error-free transformations of Knuth (TwoSum), Dekker
// (FastTwoSum) and the FMA form of TwoProd; the compositions follow the
// "sloppy" double-word sum and the FMA-based double-word products analysed by
// Joldes, Muller and Popescu (ACM TOMS 44(2), 2017).  The sloppy sum's error
// is bounded by a small multiple of u^2 (|x| + |y|), u = 2^-24: a normwise
// bound of the same kind as an FP64 addition's, which is what the Krylov
// process needs.
//
// All operations use the _rn intrinsics so that the compiler neither
// contracts nor reassociates them.
#pragma once
#include <cuda_runtime.h>

struct __align__(8) dw {
  float hi, lo;
};

__device__ __forceinline__ dw dw_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// Requires |a| >= |b| (or a == 0) for exactness.
__device__ __forceinline__ dw dw_fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}

__device__ __forceinline__ dw operator+(dw x, dw y) {
  dw s = dw_two_sum(x.hi, y.hi);
  float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return dw_fast_two_sum(s.hi, e);
}

__device__ __forceinline__ dw operator-(dw x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ dw operator-(dw x, dw y) { return x + (-y); }

// double-word x double-word (FMA form)
__device__ __forceinline__ dw operator*(dw x, dw y) {
  float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return dw_fast_two_sum(p, e);
}

// double-word x float
__device__ __forceinline__ dw operator*(dw x, float y) {
  float p = __fmul_rn(x.hi, y);
  float e = __fmaf_rn(x.hi, y, -p);
  e = __fmaf_rn(x.lo, y, e);
  return dw_fast_two_sum(p, e);
}

__device__ __forceinline__ dw dw_from_double(double v) {
  float hi = __double2float_rn(v);
  float lo = __double2float_rn(v - (double)hi);
  return {hi, lo};
}

__device__ __forceinline__ double dw_to_double(dw x) { return (double)x.hi + (double)x.lo; }

// Host-side split of an FP64 constant (same rounding as dw_from_double).
static inline dw dw_split_host(double v) {
  float hi = (float)v;
  float lo = (float)(v - (double)hi);
  dw r;
  r.hi = hi;
  r.lo = lo;
  return r;
}

// Lazy compensated accumulator (the compensated dot-product scheme of Ogita,
// Rump and Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 26(6),
// 2005, with double-word operands): the running sum s collects the leading
// parts through TwoSum, every rounding error and every trailing part goes
// to e, and the pair is renormalised once at the end.  The result is as
// accurate as a computation in twice the float precision: error about
// n u^2 sum |terms|.
struct dwacc {
  float s, e;
};

__device__ __forceinline__ void acc_set(dwacc &a, dw x) {
  a.s = x.hi;
  a.e = x.lo;
}

__device__ __forceinline__ void acc_add(dwacc &a, dw x) {
  dw t = dw_two_sum(a.s, x.hi);
  a.s = t.hi;
  a.e = __fadd_rn(a.e, __fadd_rn(t.lo, x.lo));
}

__device__ __forceinline__ void acc_sub(dwacc &a, dw x) { acc_add(a, {-x.hi, -x.lo}); }

// product c*x as an unnormalised pair (p, pe): c.lo*x.lo is dropped (~u^2 |c x|)
__device__ __forceinline__ dw dw_prod_raw(dw c, dw x) {
  float p = __fmul_rn(c.hi, x.hi);
  float e = __fmaf_rn(c.hi, x.hi, -p);
  e = __fmaf_rn(c.hi, x.lo, e);
  e = __fmaf_rn(c.lo, x.hi, e);
  return {p, e};
}

__device__ __forceinline__ void acc_set_prod(dwacc &a, dw c, dw x) {
  dw p = dw_prod_raw(c, x);
  a.s = p.hi;
  a.e = p.lo;
}

__device__ __forceinline__ void acc_add_prod(dwacc &a, dw c, dw x) {
  dw p = dw_prod_raw(c, x);
  dw t = dw_two_sum(a.s, p.hi);
  a.s = t.hi;
  a.e = __fadd_rn(a.e, __fadd_rn(t.lo, p.lo));
}

// float coefficient c (exact in FP32, e.g. a link entry): c*x with one FMA
// fewer than the double-word product
__device__ __forceinline__ void acc_add_prod(dwacc &a, float c, dw x) {
  const float p = __fmul_rn(c, x.hi);
  float e = __fmaf_rn(c, x.hi, -p);
  e = __fmaf_rn(c, x.lo, e);
  dw t = dw_two_sum(a.s, p);
  a.s = t.hi;
  a.e = __fadd_rn(a.e, __fadd_rn(t.lo, e));
}

__device__ __forceinline__ dw acc_get(const dwacc &a) { return dw_fast_two_sum(a.s, a.e); }
// the unnormalised pair, usable as a product operand
__device__ __forceinline__ dw acc_raw(const dwacc &a) { return {a.s, a.e}; }
