// tc_ptx.cuh — inline-PTX building blocks of the tcgen05 kernels (synth_tc.cu,
// adjoint_tc.cu): mbarriers with bounded waits, bulk copies, the UMMA
// shared-memory descriptor, tcgen05.mma / commit / ld, the hi/lo operand
// split and the 32-bit integer phase. Internal to libbipp_ss.so.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace bipp {
namespace tcx {

constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
// try_wait with a suspend-time hint (ns): a waiting warp sleeps in hardware
// until the phase completes or the hint expires instead of spinning on issue
// slots that the other producer warps need.
__device__ __forceinline__ bool mbar_test(uint32_t a, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(a), "r"(parity), "r"(1000000u)
      : "memory");
  return done != 0;
}
// Bounded wait for the phase of the given parity; false on expiry or abort.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, volatile int* abort_flag) {
  if (mbar_test(a, parity)) return true;
  const long long t0 = clock64();
  for (;;) {
    if (mbar_test(a, parity)) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > kWaitCycles) {
      *abort_flag = 1;
      return false;
    }
  }
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// UMMA shared-memory descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), version 1, leading offset unused for this layout.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Two 16-column loads (the two halves of a fused accumulator) under one wait,
// summed: v = acc[a] + acc[b], the sums on the packed FP32 operations.
__device__ __forceinline__ void tmem_ld16_sum2(uint32_t ta, uint32_t tb, float (&v)[16]) {
  uint32_t r[16], q[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(ta));
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]), "=r"(q[7]), "=r"(q[8]),
        "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]), "=r"(q[13]), "=r"(q[14]), "=r"(q[15])
      : "r"(tb));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; i += 2) {
    const float2 x = __fadd2_rn(make_float2(__uint_as_float(r[i]), __uint_as_float(r[i + 1])),
                                make_float2(__uint_as_float(q[i]), __uint_as_float(q[i + 1])));
    v[i] = x.x;
    v[i + 1] = x.y;
  }
}

// hi/lo split of two values in [-1, 1] into packed 16-bit pairs (element 0
// in the low half). hi is x rounded to a multiple of 2^-11 (FP16) or 2^-8
// (BF16), by adding and subtracting 1.5 * 2^12 (2^15), whose FP32 ulp is that
// step; such multiples in [-1, 1] are exact in the 16-bit type. lo = x - hi is
// exact in FP32 and |lo| <= 2^-12 (2^-9), so its 16-bit rounding costs at most
// 2^-24 (2^-17) absolute. The two values go through the packed FP32 pipe
// operations of sm_100+ (__fadd2_rn, __ffma2_rn: per component the same
// rounding as the scalar ones), three instructions instead of six.
template <bool FP16>
__device__ __forceinline__ void split2(float x0, float x1, uint32_t* hi, uint32_t* lo) {
  constexpr float M = FP16 ? 6144.0f : 49152.0f;
  const float2 x = make_float2(x0, x1);
  const float2 hh = __fadd2_rn(__fadd2_rn(x, make_float2(M, M)), make_float2(-M, -M));
  const float2 ll = __ffma2_rn(hh, make_float2(-1.0f, -1.0f), x);  // x - hi, exact
  const float h0 = hh.x, h1 = hh.y, l0 = ll.x, l1 = ll.y;
  if constexpr (FP16) {
    __half2 h = __floats2half2_rn(h0, h1);
    __half2 l = __floats2half2_rn(l0, l1);
    *hi = *reinterpret_cast<uint32_t*>(&h);
    *lo = *reinterpret_cast<uint32_t*>(&l);
  } else {
    __nv_bfloat162 h = __floats2bfloat162_rn(h0, h1);
    __nv_bfloat162 l = __floats2bfloat162_rn(l0, l1);
    *hi = *reinterpret_cast<uint32_t*>(&h);
    *lo = *reinterpret_cast<uint32_t*>(&l);
  }
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ uint4 ld_shared_v4(uint32_t a) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
  return v;
}
__device__ __forceinline__ uint2 ld_shared_v2(uint32_t a) {
  uint2 v;
  asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
  return v;
}

// Per-pixel constants of the 32-bit phase (see the header comment of
// synth_tc.cu): R = round(r 2^29) per component, and (r, r), (rl, rl) in FP32,
// rl = r - R 2^-29, duplicated for the packed FP32 operations.
struct PhasePix {
  int32_t R[3];
  float2 rf[3], rl[3];
};
__device__ __forceinline__ PhasePix phase_pix(const double (&r)[3]) {
  PhasePix p;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int R = __double2int_rn(r[c] * 536870912.0);  // |r| <= 1: |R| <= 2^29
    const float f = (float)r[c], l = (float)(r[c] - (double)R * 1.862645149230957e-09);
    p.R[c] = R;
    p.rf[c] = make_float2(f, f);
    p.rl[c] = make_float2(l, l);
  }
  return p;
}
// The 80-byte group of phase words of two stations (k_tc_pack: QH_x, QH_y,
// QH_z as 32-bit integers, then 2 pi ql and 2 pi q per component in FP32, each
// word for station 0 then station 1), from shared address a.
struct PhaseWords {
  uint4 w0, w1, w2, w3, w4;
};
__device__ __forceinline__ PhaseWords phase_words(uint32_t a) {
  PhaseWords q;
  q.w0 = ld_shared_v4(a);
  q.w1 = ld_shared_v4(a + 16u);
  q.w2 = ld_shared_v4(a + 32u);
  q.w3 = ld_shared_v4(a + 48u);
  q.w4 = ld_shared_v4(a + 64u);
  return q;
}
// 2 pi <r, q> mod 2 pi, in radians within about [-4.3, 4.3], of one pixel and
// the two stations of a group.
__device__ __forceinline__ float2 phase_rad_pair(const PhasePix& p, const PhaseWords& q) {
  const uint32_t acc0 = (uint32_t)p.R[0] * q.w0.x + (uint32_t)p.R[1] * q.w0.z + (uint32_t)p.R[2] * q.w1.x;
  const uint32_t acc1 = (uint32_t)p.R[0] * q.w0.y + (uint32_t)p.R[1] * q.w0.w + (uint32_t)p.R[2] * q.w1.y;
  float2 f = __fmul2_rn(p.rf[0], make_float2(__uint_as_float(q.w1.z), __uint_as_float(q.w1.w)));
  f = __ffma2_rn(p.rf[1], make_float2(__uint_as_float(q.w2.x), __uint_as_float(q.w2.y)), f);
  f = __ffma2_rn(p.rf[2], make_float2(__uint_as_float(q.w2.z), __uint_as_float(q.w2.w)), f);
  f = __ffma2_rn(p.rl[0], make_float2(__uint_as_float(q.w3.x), __uint_as_float(q.w3.y)), f);
  f = __ffma2_rn(p.rl[1], make_float2(__uint_as_float(q.w3.z), __uint_as_float(q.w3.w)), f);
  f = __ffma2_rn(p.rl[2], make_float2(__uint_as_float(q.w4.x), __uint_as_float(q.w4.y)), f);
  constexpr float k2pi32 = 1.4629180792671596e-09f;  // 2 pi 2^-32
  return __ffma2_rn(make_float2((float)(int32_t)acc0, (float)(int32_t)acc1), make_float2(k2pi32, k2pi32), f);
}

__device__ __forceinline__ void st_shared_v4(uint32_t a, const uint32_t (&w)[4]) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3])
               : "memory");
}

}  // namespace tcx
}  // namespace bipp
