// dfloat.cuh — double-float ("float-float") arithmetic: a value is carried as
// an unevaluated sum hi + lo of two floats (~48 significant bits), so that
// FP64-class dense products run on the FP32 pipe, which on B300 issues 64
// FMAs for every FP64 one.
//
// Multiply-accumulate (hi, lo) += a * b follows the classic error-free
// transformations: the high product's rounding error is recovered exactly by
// an FMA (Dekker / Kahan product), the high parts are added with Knuth's
// TwoSum, and the small terms (cross products, both rounding errors) go to the
// low accumulator; a_lo * b_lo (~2^-48 relative) is dropped. Accumulating K
// terms gives a relative error of order K 2^-48 in the worst case and
// sqrt(K) 2^-48 typically (about 1e-13 at K = 512), with the low word
// renormalised into the high word after every block of terms. Inputs must lie
// in the FP32 range; values below 2^-74 carry fewer than 48 bits.
#pragma once

namespace bipp {
namespace df {

// x = hi + lo with hi = fl32(x), lo = fl32(x - hi), through the FP64 pipe.
__device__ __forceinline__ void split_fp64(double x, float& hi, float& lo) {
  hi = __double2float_rn(x);
  lo = __double2float_rn(x - (double)hi);
}

// x = hi + lo from the bits of x, off the FP64 pipe (which converts at the
// DFMA rate on B300): hi keeps the sign, the exponent and the leading 23
// fraction bits (x truncated to 24 significant bits), lo is the remaining 29
// fraction bits, r 2^(e - 1075) with r < 2^29, converted to FP32 (24 of those
// bits kept) with the sign of x. hi + lo carries 48 significant bits. Values
// whose hi or lo would leave the FP32 normal range (|x| < 2^-74 or
// |x| >= 2^128, zero, inf, NaN) take split_fp64.
__device__ __forceinline__ void split(double x, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int hw = (unsigned int)(b >> 32), lw = (unsigned int)b;
  const int e = (int)((hw >> 20) & 0x7FFu);
  if (e < 1023 - 74 + 1 || e > 1023 + 127) {
    split_fp64(x, hi, lo);
    return;
  }
  const unsigned int sgn = hw & 0x80000000u;
  hi = __uint_as_float(sgn | ((unsigned int)(e - 1023 + 127) << 23) | ((hw & 0xFFFFFu) << 3) | (lw >> 29));
  const float scale = __uint_as_float((unsigned int)(e - 1075 + 127) << 23);  // 2^(e - 1075), e >= 950
  lo = __uint_as_float(__float_as_uint(__uint2float_rn(lw & 0x1FFFFFFFu) * scale) | sgn);
}

// (sh, sl) += (ah + al) * (bh + bl).
__device__ __forceinline__ void mac(float& sh, float& sl, float ah, float al, float bh, float bl) {
  const float ph = __fmul_rn(ah, bh);
  float pl = fmaf(ah, bh, -ph);
  pl = fmaf(ah, bl, pl);
  pl = fmaf(al, bh, pl);
  const float t = __fadd_rn(sh, ph);
  const float z = __fsub_rn(t, sh);
  const float e = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, z)), __fsub_rn(ph, z));
  sh = t;
  sl = __fadd_rn(sl, __fadd_rn(e, pl));
}

// Fold the low word into the high one (Fast2Sum, |sl| <= |sh| up to the
// accumulated small terms).
__device__ __forceinline__ void renorm(float& sh, float& sl) {
  const float t = __fadd_rn(sh, sl);
  sl = __fsub_rn(sl, __fsub_rn(t, sh));
  sh = t;
}

__device__ __forceinline__ double to_double(float hi, float lo) { return (double)hi + (double)lo; }

// Two independent accumulations at once on the packed FP32 pipe operations of
// sm_100+ (__fmul2_rn, __fadd2_rn, __ffma2_rn, per component the rounding of
// the scalar ones): component c of (sh, sl) += (ah + al) * (bh + bl), with the
// same roundings, term for term, as mac() above, in 12 instructions for the
// pair instead of 24. The packed operations take no negated operands, so the
// caller passes nah = -ah and nal = -al (exact) beside ah, and each
// subtraction x - y is the exact FMA y * (-1) + x.
__device__ __forceinline__ void mac2(float2& sh, float2& sl, float2 ah, float2 nah, float2 nal, float2 bh,
                                     float2 bl) {
  const float2 m1 = make_float2(-1.0f, -1.0f);
  const float2 ph = __fmul2_rn(ah, bh);
  float2 npl = __ffma2_rn(nah, bh, ph);  // -(ah bh - ph): the product's rounding error, negated
  npl = __ffma2_rn(nah, bl, npl);
  npl = __ffma2_rn(nal, bh, npl);
  const float2 t = __fadd2_rn(sh, ph);
  const float2 z = __ffma2_rn(sh, m1, t);                                    // t - sh
  const float2 e = __fadd2_rn(__ffma2_rn(__ffma2_rn(z, m1, t), m1, sh),     // sh - (t - z)
                              __ffma2_rn(z, m1, ph));                        // + (ph - z)
  sh = t;
  sl = __fadd2_rn(sl, __ffma2_rn(npl, m1, e));  // sl + (e + pl)
}

// renorm() on both components.
__device__ __forceinline__ void renorm2(float2& sh, float2& sl) {
  const float2 m1 = make_float2(-1.0f, -1.0f);
  const float2 t = __fadd2_rn(sh, sl);
  sl = __ffma2_rn(__ffma2_rn(sh, m1, t), m1, sl);  // sl - (t - sh)
  sh = t;
}

}  // namespace df
}  // namespace bipp
