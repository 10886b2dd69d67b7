// Float-float numbers: x = hi + lo, two FP32 values with |lo| <= ulp(hi) / 2,
// together a 48-bit significand (Dekker 1971).  GB300 retires FP32 FMAs at 64x
// the rate of FP64 ones (128 against 2 lanes per clock and SM), so an FFT kept in
// float-float arithmetic on the FP32 pipes outruns the same FFT on the FP64 pipe
// while staying within a few units of 2^-48 per operation.
//
// `ff` is the storage and constant type (one value); the arithmetic runs on
// `ff2`, two values at once, each pair of parts one 64-bit operand of the f32x2
// instructions (sm_100 and later: add/sub/mul/fma.rn.f32x2, one instruction for
// two lanes, each lane rounded as its scalar form), which halves the issue slots.
// The FFT packs the real and imaginary parts of a complex value into the lanes.
//
// Error-free transformations used (Knuth's two-sum, Dekker's fast two-sum, the
// exact product a b - fl(a b) as one FMA); sums take the "sloppy" form, whose
// error is bounded relative to |a| + |b|, which is what a transform's norm-wise
// error needs.  Every step is one inline-PTX .rn instruction, so the compiler
// never contracts a product and a sum into one FMA: the transformations rely on
// each rounding happening where it is written.
//
// The operators leave their result unnormalised: (s, e) with s the rounded sum
// (or product) of the high parts and e the exact error of that plus the low
// parts, |e| a few units of 2^-24 |s| (without cancellation) instead of at most
// half an ulp.  The two-sum of the high parts is exact for any inputs and every
// low-part rounding stays ~2^-24 of a term already ~2^-24 of the operands, so
// the norm-wise error is that of normalised arithmetic, while a sum costs 8
// instructions instead of 11, a product 4 (+1 sign flip) instead of 7, a fused
// a b + c 12 instead of 15 (per lane pair).  ff2_settle renormalises; a
// transform settles what its last stage stores, which bounds the growth of e to
// the few operations per element of one transform (the products that drop
// lo x lo take a normalised twiddle or potential as one factor).
#pragma once

#include <cuda_runtime.h>

namespace qe {

struct ff {
  float hi, lo;
  ff() = default;
  __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
  // nearest float, then the nearest float to the (exact) remainder
  __host__ __device__ constexpr explicit ff(double x)
      : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __host__ __device__ constexpr explicit ff(int x) : hi((float)x), lo(0.0f) {}   // |x| < 2^24
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};


// Scalar operations (the SIMT products of the FP64 path), unnormalised as the pair
// operations below: a sum 8 FP32 instructions, a product 4, a fused a b + c 12.
__device__ __forceinline__ ff operator+(ff a, ff b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float v = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
  return ff(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__device__ __forceinline__ ff operator*(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff(p, e);
}

// ---- two floats in one 64-bit register: the operands of the f32x2 instructions --

struct f2 {
  unsigned long long v;
};

__device__ __forceinline__ f2 f2_of(float a, float b) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_split(f2 a, float& x, float& y) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(a.v));
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
  f2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
  f2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}
// a b + c per lane
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return d;
}
// sign flips: both lanes, lane 0, lane 1
__device__ __forceinline__ f2 neg2(f2 a) { return {a.v ^ 0x8000000080000000ull}; }
__device__ __forceinline__ f2 neg2_0(f2 a) { return {a.v ^ 0x0000000080000000ull}; }
__device__ __forceinline__ f2 neg2_1(f2 a) { return {a.v ^ 0x8000000000000000ull}; }
// (a1, a0)
__device__ __forceinline__ f2 swap2(f2 a) {
  float x, y;
  f2_split(a, x, y);
  return f2_of(y, x);
}

// Two float-float numbers, lane by lane.
struct ff2 {
  f2 hi, lo;
};

__device__ __forceinline__ ff2 operator+(ff2 a, ff2 b) {
  const f2 s = add2(a.hi, b.hi);
  const f2 v = sub2(s, a.hi);
  const f2 e = add2(sub2(a.hi, sub2(s, v)), sub2(b.hi, v));
  return {s, add2(e, add2(a.lo, b.lo))};
}
// a - b: the two-sum of a.hi and -b.hi, written with subtractions
__device__ __forceinline__ ff2 operator-(ff2 a, ff2 b) {
  const f2 s = sub2(a.hi, b.hi);
  const f2 v = sub2(s, a.hi);
  const f2 e = sub2(sub2(a.hi, sub2(s, v)), add2(b.hi, v));
  return {s, add2(e, sub2(a.lo, b.lo))};
}
__device__ __forceinline__ ff2 operator*(ff2 a, ff2 b) {
  const f2 p = mul2(a.hi, b.hi);
  f2 e = fma2(a.hi, b.hi, neg2(p));
  e = fma2(a.hi, b.lo, e);
  e = fma2(a.lo, b.hi, e);
  return {p, e};
}
// a b + c (an overload beside the float and double fma, so that code templated
// on the element type calls fma for all of them)
using ::fma;
__device__ __forceinline__ ff2 fma(ff2 a, ff2 b, ff2 c) { return a * b + c; }
__device__ __forceinline__ ff fma(ff a, ff b, ff c) { return a * b + c; }
__device__ __forceinline__ ff2 ff2_settle(ff2 a) {
  const f2 h = add2(a.hi, a.lo);
  return {h, sub2(a.lo, sub2(h, a.hi))};
}
// (x, x) for a float-float x
__device__ __forceinline__ ff2 ff2_bcast(ff x) { return {f2_of(x.hi, x.hi), f2_of(x.lo, x.lo)}; }

}  // namespace qe
