// adjoint_tc.cu — the pixel contraction of the adjoint of the differentiable
// synthesis on the tcgen05 tensor cores.
//
// With Y_te(r) = d_te R_{l(te)}(r) z_te(r) from the first stage (k_synth_tc
// with EPI = 1, which recomputes z on the tensor cores), the gradient with
// respect to the gain-corrected eigenvectors W' is (Eq. standard_synthesis
// differentiated; the complex gradient convention dL/dRe + j dL/dIm)
//     grad_W'_t[i, e] = 2 sum_r Phi_t(r, i) Y_te(r),   Phi = exp(+j th), not its conjugate,
// a GEMM over pixels. As a real GEMM with rows [cos th_ri ; sin th_ri] per
// station (M), the columns [Re Y_e, Im Y_e] (N = ncols) and K = pixels:
//     P_c[i, n] = sum_r cos th_ri Y_n(r),  P_s[i, n] = sum_r sin th_ri Y_n(r),
//     grad_W'[i, e] = 2 ((P_c[i, 2e] - P_s[i, 2e+1]) + j (P_c[i, 2e+1] + P_s[i, 2e])).
//
// k_adjoint_tc: one persistent CTA per SM, 18 warps. Per (step t, pass over
// 128 stations) every CTA accumulates P over its 64-pixel chunks:
//   warps 0-15 generate A for the chunk: thread = (station, quarter of the 64
//              pixels); the same 32-bit integer phase and SFU sincos as the
//              forward kernel (header comment of synth_tc.cu), two pixels at a
//              time, split into BF16 hi + lo, written into two M-tiles
//              of 128 rows (64 stations' cos rows, then their sin rows) x 64
//              pixels in the UMMA K-major 128-byte swizzled layout. At the end
//              of each (t, pass) they read the accumulators (tcgen05.ld) and
//              write the CTA's partial P to global memory.
//   warp 16    issues per chunk and M-tile, per 16-pixel K slice,
//              A_hi [Y_hi | Y_lo] (N = 2 ncols) and A_lo Y_hi into TMEM.
//   warp 17    streams the chunk's Y images (hi, lo) with cp.async.bulk.
// The partials are summed over CTAs in a fixed order by k_adj_tc_reduce
// (deterministic), which also forms grad_W'. Every mbarrier wait is bounded
// and sets the abort word on expiry, as in the forward kernel.
#include <math.h>

#include <algorithm>

#include "bipp_internal.cuh"
#include "synth_tc.cuh"
#include "tc_ptx.cuh"

namespace bipp {
namespace {

using namespace tcx;

constexpr int kAProdWarps = 16;
constexpr int kAThreads = (kAProdWarps + 2) * 32;
constexpr int kAMmaWarp = kAProdWarps, kALoadWarp = kAProdWarps + 1;
constexpr int kAPix = 64;                // pixels per stage (K of the MMA: one 128-byte row)
constexpr int kASt = 128;                // stations per pass (2 M-tiles of 64 stations x (cos, sin))
constexpr int kATile = 128 * 128;        // bytes of one M-tile image (128 rows x 128 B)
constexpr int kAImg = 2 * kATile;        // both M-tiles of one image (hi or lo)
constexpr int kAStages = 2;
// Pixel words per stage: word c (0..8: R = round(r 2^29) per component, then r and
// rl = r - R 2^-29 in FP32) of pixel p at c * kAPw + p + 8 (p / 32): the four quarters of a
// warp (pixels 16 q + j) then read four different bank pairs, and the words of pixels
// 2k, 2k + 1 form one aligned 8-byte pair.
constexpr int kAPWords = 9;
constexpr int kAPw = kAPix + 16;
__device__ __forceinline__ int pw_idx(int c, int p) { return c * kAPw + p + 8 * (p >> 5); }

// Dynamic shared memory: kAStages x (A hi, A lo, Y hi, Y lo), 1 KB aligned,
// then the stages' pixel words.
__host__ __device__ constexpr int adj_stage_bytes(int ncols) { return 2 * kAImg + 2 * ncols * 128; }

__global__ void __launch_bounds__(kAThreads, 1)
    k_adjoint_tc(Pixels px, int T, int n_st, int ncols, const uint32_t* __restrict__ qph, int qph_stride,
                 const unsigned char* __restrict__ Y, int nc64, float* __restrict__ part, uint32_t idesc1,
                 uint32_t idesc2, int* status) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t bar_fullA[kAStages], bar_fullB[kAStages], bar_empty[kAStages];
  __shared__ __align__(8) uint64_t bar_accf, bar_acce, bar_drain;
  __shared__ uint32_t s_taddr;
  __shared__ volatile int s_abort;
  const int stage_bytes = adj_stage_bytes(ncols);
  uint32_t* spix = reinterpret_cast<uint32_t*>(smem + kAStages * stage_bytes);  // [stage][kAPWords][kAPw]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t tcols = (uint32_t)max(32, 1 << (32 - __clz(4 * ncols - 1)));  // 2 M-tiles x 2 ncols, power of two
  if (threadIdx.x == 0) {
    for (int s = 0; s < kAStages; ++s) {
      mbar_init(smem_u32(&bar_fullA[s]), kAProdWarps);
      mbar_init(smem_u32(&bar_fullB[s]), 1);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    mbar_init(smem_u32(&bar_accf), 1);
    mbar_init(smem_u32(&bar_acce), kAProdWarps);
    mbar_init(smem_u32(&bar_drain), 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_async_smem();
  }
  if (warp == kAMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_taddr)),
                 "r"(tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = s_taddr;
  const uint32_t smem0 = smem_u32(smem);
  const int npass = (n_st + kASt - 1) / kASt;
  const int n_units = T * npass;

  if (warp < kAProdWarps) {
    // ------------------------------------------------ A producer + epilogue
    const int tid = threadIdx.x;  // 0..511
    const int sl = tid >> 2, quarter = tid & 3;
    const int m = sl >> 6, rc = sl & 63, rs = 64 + (sl & 63);  // M-tile, cos row, sin row
    uint32_t rs_s = 0, rs_rnd = 0;
    bool ok = true;
    // threads 0..63 load their pixel's coordinates one chunk ahead, so that the global
    // loads' latency hides behind the previous chunk's phases
    double pxn[3] = {0.0, 0.0, 0.0};
    auto fetch = [&](int ch) {
      if (tid < kAPix) {
        const int64_t r = (int64_t)ch * kAPix + tid;
#pragma unroll
        for (int c = 0; c < 3; ++c) pxn[c] = (r < px.n) ? px.xyz[(size_t)c * px.n + r] : 0.0;
      }
    };
    if (blockIdx.x < nc64) fetch(blockIdx.x);
    for (int u = 0; u < n_units && ok; ++u) {
      const int t = u / npass, s0 = (u % npass) * kASt;
      const int i = s0 + sl;
      // the station's phase words (k_tc_pack: QH, 2 pi ql, 2 pi q per component), the FP32
      // ones duplicated for the packed operations on two pixels
      uint32_t QH[3] = {0u, 0u, 0u};
      float2 ql2[3], q2[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) ql2[c] = q2[c] = make_float2(0.f, 0.f);
      if (i < n_st) {
        const uint32_t* g = qph + ((size_t)t * qph_stride + (i & ~1)) * 10 + (i & 1);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          QH[c] = g[2 * c];
          const float a = __uint_as_float(g[6 + 2 * c]), b = __uint_as_float(g[12 + 2 * c]);
          ql2[c] = make_float2(a, a);
          q2[c] = make_float2(b, b);
        }
      }
      for (int chunk = blockIdx.x; chunk < nc64; chunk += gridDim.x) {
        const uint32_t s = rs_s, rnd = rs_rnd;
        if (++rs_s == (uint32_t)kAStages) {
          rs_s = 0;
          ++rs_rnd;
        }
        if (!mbar_wait(smem_u32(&bar_empty[s]), (rnd & 1) ^ 1, &s_abort)) {
          ok = false;
          break;
        }
        // the chunk's pixel words: R = round(r 2^29), r and rl = r - R 2^-29 per component
        uint32_t* pw = spix + s * kAPWords * kAPw;
        if (tid < kAPix) {
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const int R = __double2int_rn(pxn[c] * 536870912.0);
            pw[pw_idx(c, tid)] = (uint32_t)R;
            pw[pw_idx(3 + c, tid)] = __float_as_uint((float)pxn[c]);
            pw[pw_idx(6 + c, tid)] = __float_as_uint((float)(pxn[c] - (double)R * 1.862645149230957e-09));
          }
        }
        {
          int nch = chunk + gridDim.x;
          if (nch >= nc64) nch = (u + 1 < n_units) ? (int)blockIdx.x : -1;
          if (nch >= 0) fetch(nch);
        }
        asm volatile("bar.sync 1, %0;" ::"r"(kAProdWarps * 32) : "memory");
        const uint32_t a_hi = smem0 + s * stage_bytes + m * kATile, a_lo = a_hi + kAImg;
        for (int q = 0; q < 2; ++q) {  // 8 pixels per 16-byte piece
          const int pp0 = quarter * 16 + q * 8;
          float cs[8], sn[8];
#pragma unroll
          for (int j = 0; j < 8; j += 2) {  // pixels p, p + 1
            const int p = pp0 + j;
            uint2 R[3];
            float2 rf[3], rl[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              R[c] = *reinterpret_cast<const uint2*>(pw + pw_idx(c, p));
              rf[c] = *reinterpret_cast<const float2*>(pw + pw_idx(3 + c, p));
              rl[c] = *reinterpret_cast<const float2*>(pw + pw_idx(6 + c, p));
            }
            const uint32_t acc0 = R[0].x * QH[0] + R[1].x * QH[1] + R[2].x * QH[2];
            const uint32_t acc1 = R[0].y * QH[0] + R[1].y * QH[1] + R[2].y * QH[2];
            float2 f = __fmul2_rn(rf[0], ql2[0]);
            f = __ffma2_rn(rf[1], ql2[1], f);
            f = __ffma2_rn(rf[2], ql2[2], f);
            f = __ffma2_rn(rl[0], q2[0], f);
            f = __ffma2_rn(rl[1], q2[1], f);
            f = __ffma2_rn(rl[2], q2[2], f);
            constexpr float k2pi32 = 1.4629180792671596e-09f;  // 2 pi 2^-32
            const float2 ph = __ffma2_rn(make_float2((float)(int32_t)acc0, (float)(int32_t)acc1),
                                         make_float2(k2pi32, k2pi32), f);
            __sincosf(ph.x, &sn[j], &cs[j]);
            __sincosf(ph.y, &sn[j + 1], &cs[j + 1]);
          }
          uint32_t ch[4], cl[4], sh[4], sl4[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            split2<false>(cs[2 * j], cs[2 * j + 1], &ch[j], &cl[j]);
            split2<false>(sn[2 * j], sn[2 * j + 1], &sh[j], &sl4[j]);
          }
          const int piece = pp0 >> 3;
          const uint32_t oc = (uint32_t)rc * 128u + (uint32_t)((piece ^ (rc & 7)) << 4);
          const uint32_t os = (uint32_t)rs * 128u + (uint32_t)((piece ^ (rs & 7)) << 4);
          st_shared_v4(a_hi + oc, ch);
          st_shared_v4(a_lo + oc, cl);
          st_shared_v4(a_hi + os, sh);
          st_shared_v4(a_lo + os, sl4);
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bar_fullA[s]));
      }
      if (!ok) break;
      // epilogue of unit u: warp w reads TMEM lanes 32 (w % 4) .. of M-tile (w / 4) % 2,
      // the even (w < 8) or odd (w >= 8) 16-column blocks
      if (!mbar_wait(smem_u32(&bar_accf), (uint32_t)(u & 1), &s_abort)) {
        ok = false;
        break;
      }
      tc_fence_after();
      {
        const int mt = (warp >> 2) & 1, row = (warp & 3) * 32 + lane;
        const int kind = row >> 6, st = s0 + mt * 64 + (row & 63);
        const uint32_t tb = taddr + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(mt * 2 * ncols);
        float* dst = part + ((((size_t)t * gridDim.x + blockIdx.x) * 2 + kind) * n_st + st) * ncols;
        for (int cb = warp >> 3; cb < ncols / 16; cb += 2) {
          float v[16], v2[16];
          tmem_ld16(tb + cb * 16, v);
          tmem_ld16(tb + ncols + cb * 16, v2);
          if (st < n_st) {
#pragma unroll
            for (int k = 0; k < 16; k += 4)
              *reinterpret_cast<float4*>(dst + cb * 16 + k) =
                  make_float4(v[k] + v2[k], v[k + 1] + v2[k + 1], v[k + 2] + v2[k + 2], v[k + 3] + v2[k + 3]);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bar_acce));
    }
    if (!ok) s_abort = 1;
  } else if (warp == kAMmaWarp) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t rs_s = 0, rs_rnd = 0;
      bool ok = true, issued = false;
      for (int u = 0; u < n_units && ok; ++u) {
        if (!mbar_wait(smem_u32(&bar_acce), (uint32_t)((u & 1) ^ 1), &s_abort)) {
          ok = false;
          break;
        }
        tc_fence_after();
        bool first = true;
        for (int chunk = blockIdx.x; chunk < nc64; chunk += gridDim.x) {
          const uint32_t s = rs_s, rnd = rs_rnd;
          if (++rs_s == (uint32_t)kAStages) {
            rs_s = 0;
            ++rs_rnd;
          }
          if (!mbar_wait(smem_u32(&bar_fullA[s]), rnd & 1, &s_abort) ||
              !mbar_wait(smem_u32(&bar_fullB[s]), rnd & 1, &s_abort)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st0 = smem0 + s * stage_bytes;
          const uint32_t y_hi = st0 + 2 * kAImg;
#pragma unroll
          for (int mt = 0; mt < 2; ++mt) {
            const uint32_t d = taddr + (uint32_t)(mt * 2 * ncols);
            const uint32_t a_hi = st0 + mt * kATile, a_lo = a_hi + kAImg;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint32_t ko = kk * 32;
              umma_f16(d, umma_desc(a_hi + ko), umma_desc(y_hi + ko), idesc2, (first && kk == 0) ? 0u : 1u);
              umma_f16(d, umma_desc(a_lo + ko), umma_desc(y_hi + ko), idesc1, 1u);
            }
          }
          first = false;
          issued = true;
          umma_commit(smem_u32(&bar_empty[s]));
        }
        if (!ok) break;
        umma_commit(smem_u32(&bar_accf));
      }
      if (!ok) {
        s_abort = 1;
        if (issued) {
          umma_commit(smem_u32(&bar_drain));
          const long long t0 = clock64();
          while (!mbar_test(smem_u32(&bar_drain), 0) && clock64() - t0 < kWaitCycles) {
          }
        }
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------ Y loader
    if (lane == 0) {
      uint32_t rs_s = 0, rs_rnd = 0;
      bool ok = true;
      uint32_t last_round[kAStages];
      bool used[kAStages] = {false, false};
      const uint32_t bytes = (uint32_t)ncols * 256u;
      for (int u = 0; u < n_units && ok; ++u) {
        const int t = u / npass;
        for (int chunk = blockIdx.x; chunk < nc64; chunk += gridDim.x) {
          const uint32_t s = rs_s, rnd = rs_rnd;
          if (++rs_s == (uint32_t)kAStages) {
            rs_s = 0;
            ++rs_rnd;
          }
          if (!mbar_wait(smem_u32(&bar_empty[s]), (rnd & 1) ^ 1, &s_abort)) {
            ok = false;
            break;
          }
          const uint32_t bar = smem_u32(&bar_fullB[s]);
          mbar_arrive_tx(bar, bytes);
          bulk_g2s(smem0 + s * stage_bytes + 2 * kAImg, Y + ((size_t)t * nc64 + chunk) * bytes, bytes, bar);
          used[s] = true;
          last_round[s] = rnd;
        }
      }
      if (!ok) {
        s_abort = 1;
        for (int s = 0; s < kAStages; ++s) {
          if (!used[s]) continue;
          const long long t0 = clock64();
          while (!mbar_test(smem_u32(&bar_fullB[s]), last_round[s] & 1) && clock64() - t0 < kWaitCycles) {
          }
        }
      }
    }
    __syncwarp();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kAMmaWarp) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(tcols));
  if (threadIdx.x == 0 && s_abort) atomicExch(status, 1);
}

// grad_W'_t[i, e] from the partials of all CTAs, summed in CTA order (FP64).
__global__ void k_adj_tc_reduce(const float* part, int T, int n_cta, int n_st, int K, int ncols, double2* gWp) {
  const int t = blockIdx.y;
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n_st * K) return;
  const int i = w / K, e = w % K;
  double pcr = 0.0, pci = 0.0, psr = 0.0, psi = 0.0;
  for (int c = 0; c < n_cta; ++c) {
    const float* pc = part + ((((size_t)t * n_cta + c) * 2 + 0) * n_st + i) * ncols;
    const float* ps = part + ((((size_t)t * n_cta + c) * 2 + 1) * n_st + i) * ncols;
    pcr += pc[2 * e];
    pci += pc[2 * e + 1];
    psr += ps[2 * e];
    psi += ps[2 * e + 1];
  }
  gWp[((size_t)t * K + e) * n_st + i] = make_double2(2.0 * (pcr - psi), 2.0 * (pci + psr));
}

}  // namespace

int adj_tc_smem_bytes(int ncols) { return kAStages * adj_stage_bytes(ncols) + kAStages * kAPWords * kAPw * 4 + 1024; }

int launch_adjoint_tc(const Pixels& px, int T, int n_st, int K, int ncols, const uint32_t* qph, int qph_stride,
                      const unsigned char* Y, int nc64, float* part, int grid, double2* gWp, int* status,
                      cudaStream_t s) {
  if (K > 64 || ncols > 128 || (ncols & 15)) return -1;
  const uint32_t fmt = 1u;  // BF16 A and B
  auto idesc = [&](int n) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  };
  const int smem = adj_tc_smem_bytes(ncols);
  if (cudaFuncSetAttribute(k_adjoint_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return -2;
  k_adjoint_tc<<<grid, kAThreads, smem, s>>>(px, T, n_st, ncols, qph, qph_stride, Y, nc64, part, idesc(ncols),
                                             idesc(2 * ncols), status);
  k_adj_tc_reduce<<<dim3((n_st * K + 255) / 256, T), 256, 0, s>>>(part, T, grid, n_st, K, ncols, gWp);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace bipp
