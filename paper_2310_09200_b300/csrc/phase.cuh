// phase.cuh — exact phase reduction for the FP32 / tensor-core synthesis
// paths. The phasor of Eq. standard_synthesis, exp(-j 2 pi <r, p_i>/wl), only
// depends on the fractional part of t = <r, q_i> with q_i = p_i/wl (cycles).
// At 65 km baselines and wl = 1.5-3 m, |t| reaches ~4e4 cycles, so a plain
// FP32 product would lose ~1e-3 cycles; this reduction keeps ~2^-24.
#pragma once

namespace bipp {

// Fractional part of <r, q> in cycles, in [-0.5, 0.5]; r and q are given as
// float hi + lo splits (r[0..2] hi, r[3..5] lo; the same for q). Each hi*hi
// product p is formed rounded (never contracted into an FMA) with its exact
// residual fma(a, b, -p); p - rint(p) is exact in FP32; the residuals and the
// hi*lo cross terms are below 2^-8 cycles and are summed in FP32.
__device__ __forceinline__ float phase_frac_f32(const float* r, const float* q) {
  float f = 0.0f, small = 0.0f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float p = __fmul_rn(r[c], q[c]);
    const float e = fmaf(r[c], q[c], -p);
    f = __fadd_rn(f, __fsub_rn(p, rintf(p)));
    small = __fadd_rn(small, e);
    small = fmaf(r[c], q[c + 3], small);
    small = fmaf(r[c + 3], q[c], small);
  }
  f = __fadd_rn(f, small);
  return __fsub_rn(f, rintf(f));
}

// sin and cos of 2 pi f on the SFU (f in cycles, |f| <= 1/2).
__device__ __forceinline__ void sincos_cycles(float f, float* s, float* c) {
  __sincosf(6.28318530717958647692f * f, s, c);
}

}  // namespace bipp
