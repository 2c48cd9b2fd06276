// synth_tc.cu — fused standard synthesis on the tcgen05 tensor cores.
//
// Per time step the synthesis of Eq. standard_synthesis (Algorithm 2,
// "GEMMEXP") is the real GEMM
//     [z_r | z_i](r, e) = sum_k A(r, k) B(k, n),
//     A(r, 2i) = cos th_ri, A(r, 2i+1) = sin th_ri,  th_ri = 2 pi <r, p_i>/wl,
//     B(2i, 2e) = Re a_ie, B(2i+1, 2e) = Im a_ie, B(2i, 2e+1) = Im a_ie, B(2i+1, 2e+1) = -Re a_ie,
// so that z_e(r) = sum_i exp(-j th_ri) a_ie, followed by the level reduction
// I_l(r) += sum_{e in l} d_e |z_e(r)|^2 (Algorithm 1) and the sum over steps.
//
// Kernel structure (one persistent CTA per SM, 22 warps; 18 for eigenimages):
//   warps 0-15 (4 warpgroups) generate A for a 128-pixel tile on the fly:
//              thread = pixel rows r and r + 64 by stations 4q..4q+3 of the
//              stage; phase reduction by 32-bit integer products (below), SFU
//              sincos, split into hi + lo (BF16 or FP16), written into shared
//              memory in the UMMA K-major 128-byte swizzled layout (one
//              128-byte row per pixel, 32 stations per stage).
//   warps 16-19 run the epilogue (EPW): tcgen05.ld of the FP32 accumulator
//              (pixel row = TMEM lane, every column block), |z|^2, weights and
//              levels in registers, accumulated over all steps and added to
//              the FP64 image once per tile. Without them (eigenimages, and
//              the adjoint's Y stage) the producers run it between units,
//              warpgroup g taking column blocks g, g+4, ...
//   next warp  allocates TMEM (two accumulator buffers) and issues, per
//              16-wide K slice, the split products A_hi*B_hi + A_hi*B_lo +
//              A_lo*B_hi into FP32 accumulators: with FUSE (2 K <= 128
//              columns) as two tcgen05.mma, A_hi*[B_hi | B_lo] (N = 2 ncols:
//              the hi and lo images of B lie side by side) and A_lo*B_hi into
//              the first half, the halves summed in the epilogue; otherwise as
//              three MMAs of N = ncols into one accumulator.
//   last warp  streams the pre-packed, pre-swizzled B chunks of the step with
//              cp.async.bulk into the stage ring.
// Stage handoff uses mbarriers; every wait is bounded (clock64 budget) and on
// expiry sets a device error word, drains its own in-flight work, frees TMEM
// and returns.
//
// Phase. Only frac(<r, q_i>) matters (q_i = p_i/wl in cycles, |<r, q_i>| up to
// ~4e4 at 65 km). Per component, r = R 2^-29 + rl (R = round(r 2^29), a
// 32-bit integer, |rl| <= 2^-30) and q = QH / 8 + ql (QH = round(8 q), a 32-bit
// integer, |ql| <= 1/16), so that
//     r q = R QH 2^-32 + r ql + rl q - rl ql.
// The first term taken mod 1 is the wrapped 32-bit product R QH as a fraction
// of 2^32 (one integer multiply-add per component: the sum over the three
// components wraps exactly), the next two are small (|r ql| <= 1/16,
// |rl q| <= 2^-15) and go to FP32 with ~2^-28 cycles of error, and the last
// (<= 2^-34) is dropped. Per pixel-station pair: three 32-bit IMADs at half
// rate and six FP32 FMAs (packed two stations at a time), against the nine
// IMADs (three of them at quarter rate, mul.hi) of a 64-bit fixed-point sum.
// Error ~2^-25 cycles (the FP32 rounding of the 32-bit fraction); station
// coordinates up to 2^28 wavelengths from the origin (farther ones mark the
// step kStatusRange and the batch commits nothing).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <type_traits>

#include "synth_tc.cuh"
#include "tc_ptx.cuh"

namespace bipp {

namespace {

constexpr int kProdWarps = 16;  // 4 warpgroups
constexpr int kEpiWarps = 4;    // dedicated epilogue warps (EPW): one per quarter of the TMEM lanes
// Threads of a CTA: producers, [epilogue warps,] the MMA issuer and the B loader.
__host__ __device__ constexpr int synth_threads(bool epw) { return (kProdWarps + (epw ? kEpiWarps : 0) + 2) * 32; }
constexpr int kThreads = synth_threads(false);
constexpr int kRows = 128;            // pixels per tile = UMMA M
constexpr int kStations = 32;         // stations per stage (64 K-elements)
constexpr int kABytes = kRows * 128;  // one A operand image per stage (hi or lo)
constexpr int kMaxStages = 4;
constexpr int kQWin = 8;  // chunks of station words staged per window (two windows in shared memory)
constexpr uint32_t kQBytes = 40;  // phase words per station (k_tc_pack: 20 words per pair of stations)
static_assert((kQWin & (kQWin - 1)) == 0, "window of a power-of-two chunk count");

using namespace tcx;

template <int MAXL>
__device__ __forceinline__ void level_add(float (&acc)[MAXL], int lev, float v) {
#pragma unroll
  for (int l = 0; l < MAXL; ++l) acc[l] += (lev == l) ? v : 0.0f;
}

// ---------------------------------------------------------------- the fused kernel

// EPI = 0: level images (above). EPI = 1: the adjoint's first stage: instead
// of |z|^2, write Y_e(r) = d_e R_{l(e)}(r) z_e(r) (R = dL/dI, yo.R) for every
// pixel, step and accumulator column into yo.Y as BF16 hi/lo images in the
// K-major, 128-byte-swizzled layout of a UMMA B operand whose K runs over 64
// pixels (see TcYOut); img is not touched.
template <int MAXL, bool FP16, bool FUSE, int EPI, bool EPW>
__global__ void __launch_bounds__(synth_threads(EPW), 1)
    k_synth_tc(Batch b, Pixels px, int n_level, double* img, TcYOut yo, const TcStep* __restrict__ steps,
               const unsigned char* __restrict__ Bpack, const float* __restrict__ scales,
               const uint32_t* __restrict__ qph, int qph_stride, const int2* __restrict__ lwt, int n_stages,
               int stage_bytes, int ncols_buf, int* status) {
  if (*b.flag) return;  // a step of the batch failed: commit nothing
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t bar_fullA[kMaxStages], bar_fullB[kMaxStages], bar_empty[kMaxStages];
  __shared__ __align__(8) uint64_t bar_accf[2], bar_acce[2], bar_drain, bar_q;
  __shared__ uint32_t s_taddr;
  __shared__ volatile int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int kMmaWarp = kProdWarps + (EPW ? kEpiWarps : 0), kLoadWarp = kMmaWarp + 1;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kMaxStages; ++s) {
      mbar_init(smem_u32(&bar_fullA[s]), kProdWarps);
      mbar_init(smem_u32(&bar_fullB[s]), 1);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(&bar_accf[i]), 1);
      mbar_init(smem_u32(&bar_acce[i]), EPW ? kEpiWarps : kProdWarps);
    }
    mbar_init(smem_u32(&bar_drain), 1);
    mbar_init(smem_u32(&bar_q), kProdWarps);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_async_smem();
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_taddr)),
                 "r"(2 * ncols_buf));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = s_taddr;
  const uint32_t smem0 = smem_u32(smem);
  const int n_tiles = (int)((px.n + kRows - 1) / kRows);
  const int T = b.T;

  if (warp < kMmaWarp) {
    // ------------------------------------------------ A producer + epilogue (EPW: warps past the
    // producers run the epilogue alone, pixel row = their TMEM lane, every column block)
    const bool epi_warp = EPW && warp >= kProdWarps;
    const int row = threadIdx.x & (kRows - 1);
    const int wg = threadIdx.x >> 7;  // warpgroup: column blocks wg + 4j of the epilogue
    // A producer: pixel rows rp and rp + 64 of the tile, stations 4 quad .. 4 quad + 3 of
    // the stage (one 16-byte piece of each row), so that a warp's station words (the
    // same for all its lanes) serve two pixels per load
    const int rp = threadIdx.x & 63, quad = threadIdx.x >> 6;
    uint32_t rs_s = 0, rs_rnd = 0;  // ring slot and round, advanced per chunk
    int unit = 0;
    int pend_tile = -1, pend_t = -1;
    float lacc[MAXL];
#pragma unroll
    for (int l = 0; l < MAXL; ++l) lacc[l] = 0.0f;
    bool ok = true;
    // Station words, staged in shared memory by windows of up to kQWin chunks
    // in two buffers after the stage ring: the window after the current one
    // (in tile, step, chunk order) is copied with cp.async while the current
    // one is produced, so the per-stage reads hit shared memory, not L2.
    constexpr uint32_t kQWinBytes = kQWin * kStations * kQBytes;
    const uint32_t qsm0 = smem0 + (uint32_t)n_stages * (uint32_t)stage_bytes;
    uint32_t qbuf = 0, qphase = 0;
    auto q_prefetch = [&](int tn, int c0, uint32_t buf) {
      const unsigned char* src =
          reinterpret_cast<const unsigned char*>(qph + ((size_t)tn * qph_stride + (size_t)c0 * kStations) * (kQBytes / 4));
      const uint32_t nbytes = (uint32_t)min(kQWin, steps[tn].n_chunks - c0) * kStations * kQBytes;
      for (uint32_t o = threadIdx.x * 16u; o < nbytes; o += kProdWarps * 32u * 16u)
        cp_async16(qsm0 + buf * kQWinBytes + o, src + o);
      cp_async_commit();
    };
    if (!epi_warp && blockIdx.x < n_tiles) q_prefetch(0, 0, 0);

    // cb0, cbs: the column blocks cb0, cb0 + cbs, ... of this thread
    auto epilogue = [&](int tile, int t, int u, int cb0, int cbs) -> bool {
      const int bb = u & 1;
      if (!mbar_wait(smem_u32(&bar_accf[bb]), (uint32_t)((u >> 1) & 1), &s_abort)) return false;
      tc_fence_after();
      const TcStep st = steps[t];
      const int K = b.nkept[t];
      const int2* lw = lwt + (size_t)t * kLwtStride;
      const uint32_t tbase = taddr + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(bb * ncols_buf);
      if constexpr (EPI == 1) {
        // Y = d R z: R of this pixel per level, z = accumulator / scale (the weights hold d / scale^2)
        const int64_t r = (int64_t)tile * kRows + row;
        const bool in = r < px.n;
        float Rl[MAXL];
#pragma unroll
        for (int l = 0; l < MAXL; ++l) Rl[l] = (in && l < n_level) ? (float)yo.R[(size_t)l * px.n + r] : 0.0f;
        const float sc = FP16 ? scales[t] : 1.0f;
        const int64_t chunk = r >> 6;  // the tile's second chunk lies past the image when n_pix % 128 <= 64
        const bool store = chunk < yo.nc64;
        const int p64 = (int)(r & 63);
        unsigned char* yb = yo.Y + ((size_t)t * yo.nc64 + (size_t)chunk) * (size_t)(2 * st.ncols * 128);
        for (int cb = cb0; cb < st.ncols / 16; cb += cbs) {
          float v[16];  // every lane of the warp takes part (tcgen05.ld is warp-wide)
          if constexpr (FUSE) tmem_ld16_sum2(tbase + cb * 16, tbase + st.ncols + cb * 16, v);  // + the A_hi B_lo half
          else tmem_ld16(tbase + cb * 16, v);
#pragma unroll
          for (int p = 0; p < 8; ++p) {
            const int e = cb * 8 + p;
            float f = 0.0f;
            if (e < K) {
              const int2 lv = lw[e];
              float rv = 0.0f;
#pragma unroll
              for (int l = 0; l < MAXL; ++l) rv = (lv.x == l) ? Rl[l] : rv;
              f = __int_as_float(lv.y) * sc * rv;
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              const int n = cb * 16 + 2 * p + q;
              const float y = f * v[2 * p + q];
              const __nv_bfloat16 yh = __float2bfloat16_rn(y);
              const __nv_bfloat16 yl = __float2bfloat16_rn(y - __bfloat162float(yh));
              const size_t off = (size_t)n * 128 + (size_t)((((p64 >> 3) ^ (n & 7)) << 4) + (p64 & 7) * 2);
              if (store) {
                *reinterpret_cast<__nv_bfloat16*>(yb + off) = yh;
                *reinterpret_cast<__nv_bfloat16*>(yb + (size_t)st.ncols * 128 + off) = yl;
              }
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bar_acce[bb]));
        return true;
      }
      for (int cb = cb0; cb < st.ncols / 16; cb += cbs) {
        float v[16];
        if constexpr (FUSE) tmem_ld16_sum2(tbase + cb * 16, tbase + st.ncols + cb * 16, v);  // + the A_hi B_lo half
        else tmem_ld16(tbase + cb * 16, v);
        // a block of 8 pairs in one level (the usual case: levels are eigenvalue
        // intervals of pairs in rank order): one weighted sum, one level add
        const int lb = b.eigen ? -2 : lw[kTcMaxEig + cb].x;
        if (lb >= 0) {
          const int4* w4 = reinterpret_cast<const int4*>(lw + cb * 8);  // (level, weight) x 2; weight 0 if not imaged
          float sacc = 0.0f;
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const int4 q = w4[h];
            sacc = fmaf(__int_as_float(q.y), fmaf(v[4 * h], v[4 * h], v[4 * h + 1] * v[4 * h + 1]), sacc);
            sacc = fmaf(__int_as_float(q.w), fmaf(v[4 * h + 2], v[4 * h + 2], v[4 * h + 3] * v[4 * h + 3]), sacc);
          }
          level_add<MAXL>(lacc, lb, sacc);
        } else if (lb == -2) {
#pragma unroll
          for (int p = 0; p < 8; ++p) {
            const int e = cb * 8 + p;
            if (e < K) {
              const int2 lv = lw[e];
              // eigenimages: slot (cb / 4) * 8 + p of this warpgroup's eigenvectors e = cb * 8 + p
              if (lv.x >= 0)
                level_add<MAXL>(lacc, b.eigen ? (cb >> 2) * 8 + p : lv.x,
                                __int_as_float(lv.y) * fmaf(v[2 * p], v[2 * p], v[2 * p + 1] * v[2 * p + 1]));
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&bar_acce[bb]));
      if (last_of_chan(b, t)) {
        const int64_t r = (int64_t)tile * kRows + row;
        double* im = img + (size_t)step_chan(b, t) * n_level * px.n;
        if (r < px.n) {
          if (b.eigen) {
#pragma unroll
            for (int sl = 0; sl < MAXL; ++sl) {
              const int e = ((sl >> 3) * 4 + wg) * 8 + (sl & 7);
              if (e < n_level && lacc[sl] != 0.0f) atomicAdd(im + (size_t)e * px.n + r, (double)lacc[sl]);
            }
          } else {
#pragma unroll
            for (int l = 0; l < MAXL; ++l)
              if (l < n_level && lacc[l] != 0.0f) atomicAdd(im + (size_t)l * px.n + r, (double)lacc[l]);
          }
        }
#pragma unroll
        for (int l = 0; l < MAXL; ++l) lacc[l] = 0.0f;
      }
      return true;
    };

    if (epi_warp) {  // EPW: the units in the producers' order, each as soon as its accumulator is ready
      int u = 0;
      for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x)
        for (int t = 0; t < T && ok; ++t, ++u) ok = epilogue(tile, t, u, 0, 1);
    } else
    for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
      PhasePix pp[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int64_t rk = (int64_t)tile * kRows + rp + 64 * k;
        double rx[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) rx[c] = (rk < px.n) ? px.xyz[(size_t)c * px.n + rk] : 0.0;
        pp[k] = phase_pix(rx);
      }
      for (int t = 0; t < T && ok; ++t) {
        const int nch = steps[t].n_chunks;
        uint32_t qcur = 0;
        for (int c = 0; c < nch; ++c) {
          if ((c & (kQWin - 1)) == 0) {
            // the window's words have landed in every producer's share, and every
            // producer is done with the previous window: refill its buffer
            cp_async_wait();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&bar_q));
            if (!mbar_wait(smem_u32(&bar_q), qphase, &s_abort)) {
              ok = false;
              break;
            }
            qphase ^= 1;
            if (c + kQWin < nch)
              q_prefetch(t, c + kQWin, qbuf ^ 1);
            else if (t + 1 < T)
              q_prefetch(t + 1, 0, qbuf ^ 1);
            else if (tile + (int)gridDim.x < n_tiles)
              q_prefetch(0, 0, qbuf ^ 1);
            qcur = qsm0 + qbuf * kQWinBytes;
            qbuf ^= 1;
          }
          const uint32_t s = rs_s, rnd = rs_rnd;
          if (++rs_s == (uint32_t)n_stages) {
            rs_s = 0;
            ++rs_rnd;
          }
          if (!mbar_wait(smem_u32(&bar_empty[s]), (rnd & 1) ^ 1, &s_abort)) {
            ok = false;
            break;
          }
          {
            // the thread's eight pairs side by side (phases, sincos, splits), so that their
            // independent dependency chains interleave; padded stations have zero phase
            // words and zero B rows
            const uint32_t qs = qcur + (uint32_t)((c & (kQWin - 1)) * kStations + 4 * quad) * kQBytes;
            float cs[2][4], sn[2][4];
#pragma unroll
            for (int g = 0; g < 2; ++g) {
              const PhaseWords qw = phase_words(qs + 2u * kQBytes * g);
#pragma unroll
              for (int k = 0; k < 2; ++k) {
                const float2 p2 = phase_rad_pair(pp[k], qw);
                __sincosf(p2.x, &sn[k][2 * g], &cs[k][2 * g]);
                __sincosf(p2.y, &sn[k][2 * g + 1], &cs[k][2 * g + 1]);
              }
            }
#pragma unroll
            for (int k = 0; k < 2; ++k) {
              const int rr = rp + 64 * k;
              uint32_t hw[4], lw[4];
#pragma unroll
              for (int j = 0; j < 4; ++j) split2<FP16>(cs[k][j], sn[k][j], &hw[j], &lw[j]);
              const uint32_t a_hi = smem0 + s * stage_bytes + (uint32_t)rr * 128u + (uint32_t)((quad ^ (rr & 7)) << 4);
              st_shared_v4(a_hi, hw);
              st_shared_v4(a_hi + kABytes, lw);
            }
          }
          fence_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&bar_fullA[s]));
        }
        if (!ok) break;
        if (!EPW && pend_tile >= 0 && !epilogue(pend_tile, pend_t, unit - 1, wg, 4)) {
          ok = false;
          break;
        }
        pend_tile = tile;
        pend_t = t;
        ++unit;
      }
    }
    if (!EPW && ok && pend_tile >= 0) ok = epilogue(pend_tile, pend_t, unit - 1, wg, 4);
    cp_async_wait();  // no copy may still be in flight into shared memory at exit
    if (!ok) s_abort = 1;
  } else if (warp == kMmaWarp) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t rs_s = 0, rs_rnd = 0;
      int unit = 0;
      bool ok = true;
      bool issued = false;
      // fault injection (status[1] set by the host): wait for a phase of bar_drain
      // that nothing completes, so that the bounded wait runs out and the abort
      // path below runs
      if (status[1] != 0) ok = mbar_wait(smem_u32(&bar_drain), 0, &s_abort);
      for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
        for (int t = 0; t < T && ok; ++t, ++unit) {
          const TcStep st = steps[t];
          const int bb = unit & 1;
          if (!mbar_wait(smem_u32(&bar_acce[bb]), (uint32_t)(((unit >> 1) & 1) ^ 1), &s_abort)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = taddr + (uint32_t)(bb * ncols_buf);
          for (int c = 0; c < st.n_chunks; ++c) {
            const uint32_t s = rs_s, rnd = rs_rnd;
            if (++rs_s == (uint32_t)n_stages) {
              rs_s = 0;
              ++rs_rnd;
            }
            if (!mbar_wait(smem_u32(&bar_fullA[s]), rnd & 1, &s_abort) ||
                !mbar_wait(smem_u32(&bar_fullB[s]), rnd & 1, &s_abort)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t a_hi = smem0 + s * stage_bytes, a_lo = a_hi + kABytes;
            const uint32_t b_hi = a_hi + 2 * kABytes, b_lo = b_hi + (uint32_t)st.ncols * 128u;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint32_t ko = kk * 32;
              const uint64_t dah = umma_desc(a_hi + ko), dal = umma_desc(a_lo + ko);
              const uint64_t dbh = umma_desc(b_hi + ko), dbl = umma_desc(b_lo + ko);
              if constexpr (FUSE) {
                umma_f16(d, dah, dbh, st.idesc2, (c | kk) != 0);  // [A_hi B_hi | A_hi B_lo]
                umma_f16(d, dal, dbh, st.idesc, 1);               // + A_lo B_hi in the first half
              } else {
                umma_f16(d, dah, dbh, st.idesc, (c | kk) != 0);
                umma_f16(d, dah, dbl, st.idesc, 1);
                umma_f16(d, dal, dbh, st.idesc, 1);
              }
            }
            issued = true;
            umma_commit(smem_u32(&bar_empty[s]));
          }
          if (!ok) break;
          umma_commit(smem_u32(&bar_accf[bb]));
        }
      }
      if (!ok) {
        s_abort = 1;
        if (issued) {  // wait for the MMAs already issued before TMEM is released
          umma_commit(smem_u32(&bar_drain));
          const long long t0 = clock64();
          while (!mbar_test(smem_u32(&bar_drain), 0) && clock64() - t0 < kWaitCycles) {
          }
        }
      }
    }
    __syncwarp();
  } else if (warp == kLoadWarp) {
    // ------------------------------------------------ B loader
    if (lane == 0) {
      uint32_t rs_s = 0, rs_rnd = 0;
      bool ok = true;
      uint32_t last_round[kMaxStages];
      bool used[kMaxStages] = {false, false, false, false};
      for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
        for (int t = 0; t < T && ok; ++t) {
          const TcStep st = steps[t];
          const uint32_t bytes = (uint32_t)st.ncols * 256u;
          for (int c = 0; c < st.n_chunks; ++c) {
            const uint32_t s = rs_s, rnd = rs_rnd;
            if (++rs_s == (uint32_t)n_stages) {
              rs_s = 0;
              ++rs_rnd;
            }
            if (!mbar_wait(smem_u32(&bar_empty[s]), (rnd & 1) ^ 1, &s_abort)) {
              ok = false;
              break;
            }
            const uint32_t bar = smem_u32(&bar_fullB[s]);
            mbar_arrive_tx(bar, bytes);
            bulk_g2s(smem0 + s * stage_bytes + 2 * kABytes, Bpack + st.b_off + (long long)c * bytes, bytes, bar);
            used[s] = true;
            last_round[s] = rnd;
          }
        }
      }
      if (!ok) {
        s_abort = 1;
        for (int s = 0; s < n_stages; ++s) {  // let the copies already issued land
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
  if (warp == kMmaWarp) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(2 * ncols_buf));
  if (threadIdx.x == 0 && s_abort) atomicExch(status, 1);
}

// ---------------------------------------------------------------- operand packing

// FP16 variant: per-step power-of-two scale so that max |W| * scale <= 2^14.
__global__ void k_tc_scale(Batch b, float* scales) {
  const int t = blockIdx.x;
  const int n = b.nst[t], K = b.nkept[t], KM = b.k_max, N = b.n_max;
  __shared__ double red[256];
  double m = 0.0;
  for (int w = threadIdx.x; w < n * K; w += blockDim.x) {
    const int i = w % n, e = w / n;
    const double2 a = b.W64[((size_t)t * KM + e) * N + i];
    m = fmax(m, fmax(fabs(a.x), fabs(a.y)));
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double mx = red[0];
    float s = 1.0f;
    if (mx > 0.0) s = (float)exp2(floor(log2(16384.0 / mx)));
    scales[t] = s;
  }
}

// B chunk c of step t: rows n < ncols (K-major, 128 bytes = 64 K-elements),
// hi image then lo image, 16-byte pieces XOR-swizzled by (row & 7).
// Also the chunk's station phase words: per pair of stations (a, b) 20
// words: QH_x, QH_y, QH_z (QH = round(8 p/wl), 32-bit integers), then 2 pi ql
// and 2 pi q per component in FP32 (ql = p/wl - QH/8), each word for a then b,
// and two zero words (header comment). Padded stations i >= n have zero
// words. A station with |8 p/wl| >= 2^31 marks its step kStatusRange (and the
// batch flag, so that nothing is committed).
template <bool FP16>
__global__ void k_tc_pack(Batch b, const TcStep* steps, unsigned char* Bpack, const float* scales, uint32_t* qph,
                          int qph_stride, int2* lwt) {
  const int t = blockIdx.y, c = blockIdx.x;
  const TcStep st = steps[t];
  if (c >= st.n_chunks) return;
  const int n = b.nst[t], K = b.nkept[t], KM = b.k_max, N = b.n_max;
  if (c == 0) {  // (level, FP32 weight / scale^2) of each accumulator column pair; level -1 = not imaged
    const double inv2 = FP16 ? 1.0 / ((double)scales[t] * (double)scales[t]) : 1.0;
    for (int e = threadIdx.x; e < kTcMaxEig; e += blockDim.x) {
      int2 v = make_int2(-1, 0);
      if (e < K && b.level[(size_t)t * KM + e] >= 0)
        v = make_int2(b.level[(size_t)t * KM + e], __float_as_int((float)(b.wt[(size_t)t * KM + e] * inv2)));
      lwt[(size_t)t * kLwtStride + e] = v;
    }
    for (int q = threadIdx.x; q < kTcMaxEig / 8; q += blockDim.x) {  // the blocks' common levels
      int lv = -1;
      for (int e = 8 * q; e < 8 * q + 8; ++e) {
        const int l = (e < K) ? b.level[(size_t)t * KM + e] : -1;
        if (l >= 0) lv = (lv == -1 || lv == l) ? l : -2;
      }
      lwt[(size_t)t * kLwtStride + kTcMaxEig + q] = make_int2(lv, 0);
    }
  }
  if (threadIdx.x < kStations) {
    const int i = c * kStations + threadIdx.x;
    uint32_t* g = qph + ((size_t)t * qph_stride + (i & ~1)) * (kQBytes / 4);
    const int sl = i & 1;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      int QH = 0;
      float ql = 0.f, qf = 0.f;
      if (i < n) {
        const double q = b.st[((size_t)t * 3 + k) * N + i] / b.wl[t];
        const double q8 = rint(8.0 * q);
        if (fabs(q8) < 2147483647.0) {
          QH = (int)q8;
          ql = (float)(6.283185307179586 * (q - 0.125 * q8));
          qf = (float)(6.283185307179586 * q);
        } else if (q8 == q8) {
          bad = true;  // (a NaN coordinate is left to the Gram matrix's check)
        }
      }
      g[2 * k + sl] = (uint32_t)QH;
      g[6 + 2 * k + sl] = __float_as_uint(ql);
      g[12 + 2 * k + sl] = __float_as_uint(qf);
    }
    g[18 + sl] = 0u;
    if (bad) {
      if (b.status) atomicOr(b.status + t, kStatusRange);
      atomicOr(b.flag, kStatusRange);
    }
  }
  const double scale = FP16 ? (double)scales[t] : 1.0;
  unsigned char* base = Bpack + st.b_off + (size_t)c * st.ncols * 256;
  for (int w = threadIdx.x; w < st.ncols * 8; w += blockDim.x) {
    const int nn = w >> 3, qp = w & 7;
    const int e = nn >> 1, comp = nn & 1;
    uint32_t hw[4], lw[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int i = c * kStations + qp * 4 + j;
      double2 a = make_double2(0.0, 0.0);
      if (i < n && e < K) a = b.W64[((size_t)t * KM + e) * N + i];
      const double wr = a.x * scale, wi = a.y * scale;
      const double v0 = comp ? wi : wr;   // B(2i, n)
      const double v1 = comp ? -wr : wi;  // B(2i+1, n)
      if constexpr (FP16) {
        __half2 h = __floats2half2_rn((float)v0, (float)v1);
        __half2 l = __floats2half2_rn((float)(v0 - (double)__low2float(h)), (float)(v1 - (double)__high2float(h)));
        hw[j] = *reinterpret_cast<uint32_t*>(&h);
        lw[j] = *reinterpret_cast<uint32_t*>(&l);
      } else {
        __nv_bfloat162 h = __floats2bfloat162_rn((float)v0, (float)v1);
        __nv_bfloat162 l =
            __floats2bfloat162_rn((float)(v0 - (double)__low2float(h)), (float)(v1 - (double)__high2float(h)));
        hw[j] = *reinterpret_cast<uint32_t*>(&h);
        lw[j] = *reinterpret_cast<uint32_t*>(&l);
      }
    }
    const size_t off = (size_t)nn * 128 + (size_t)((qp ^ (nn & 7)) << 4);
    *reinterpret_cast<uint4*>(base + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    *reinterpret_cast<uint4*>(base + (size_t)st.ncols * 128 + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
  }
}

inline int ncols_for(int k) { return std::max(16, ((2 * k + 15) / 16) * 16); }
inline int n_chunks_for(int n) { return (n + kStations - 1) / kStations; }

uint32_t make_idesc(int ncols, bool fp16) {
  const uint32_t fmt = fp16 ? 0u : 1u;  // A/B: 0 = F16, 1 = BF16
  return (1u << 4)                      // D = F32
         | (fmt << 7) | (fmt << 10)     // A, B formats; both K-major (bits 15, 16 = 0)
         | ((uint32_t)(ncols >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
}

template <typename F>
void dispatch(int n_level, bool fp16, bool fuse, F&& f) {
  auto lv = [&](auto FPV, auto FU) {
    if (n_level <= 4) f(std::integral_constant<int, 4>{}, FPV, FU);
    else if (n_level <= 8) f(std::integral_constant<int, 8>{}, FPV, FU);
    else f(std::integral_constant<int, 16>{}, FPV, FU);
  };
  auto fu = [&](auto FPV) {
    if (fuse) lv(FPV, std::true_type{});
    else lv(FPV, std::false_type{});
  };
  if (fp16) fu(std::true_type{});
  else fu(std::false_type{});
}

}  // namespace

int tc_alloc(TcWorkspace* w, int T, int N, int K) {
  tc_free(w);
  const int kk = std::min(K, kTcMaxEig);
  const size_t bytes = (size_t)T * n_chunks_for(N) * ncols_for(kk) * 256;
  if (cudaMalloc(&w->B, bytes) != cudaSuccess) return -1;
  w->B_bytes = bytes;
  if (cudaMalloc(&w->steps, sizeof(TcStep) * T) != cudaSuccess) return -1;
  if (cudaMallocHost(&w->h_steps, sizeof(TcStep) * T) != cudaSuccess) return -1;
  if (cudaMalloc(&w->scale, sizeof(float) * T) != cudaSuccess) return -1;
  w->qph_stride = n_chunks_for(N) * kStations;
  if (cudaMalloc(&w->qph, kQBytes * (size_t)T * w->qph_stride) != cudaSuccess) return -1;
  if (cudaMalloc(&w->lwt, sizeof(int2) * (size_t)T * kLwtStride) != cudaSuccess) return -1;
  if (cudaMalloc(&w->status, 2 * sizeof(int)) != cudaSuccess) return -1;
  if (cudaMemset(w->status, 0, 2 * sizeof(int)) != cudaSuccess) return -1;
  w->cap_T = T;
  return 0;
}

void tc_free(TcWorkspace* w) {
  if (w->B) cudaFree(w->B);
  if (w->steps) cudaFree(w->steps);
  if (w->h_steps) cudaFreeHost(w->h_steps);
  if (w->scale) cudaFree(w->scale);
  if (w->qph) cudaFree(w->qph);
  if (w->lwt) cudaFree(w->lwt);
  if (w->status) cudaFree(w->status);
  *w = TcWorkspace{};
}

int tc_set_fail_wait(TcWorkspace* w, int on) {
  if (!w->status) return 0;
  return cudaMemcpy(w->status + 1, &on, sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess ? 0 : -1;
}

int tc_read_status(TcWorkspace* w) {
  int v = 0;
  if (!w->status || cudaMemcpy(&v, w->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
  return v;
}

namespace {

int stage_bytes_for(int ncols_max) { return 2 * kABytes + 2 * ncols_max * 128; }
constexpr int kQStageBytes = 2 * kQWin * kStations * (int)kQBytes;  // the two station-word windows
// Dynamic shared memory: the stage ring, the station-word windows and 1 KB of
// alignment slack, within 227 KB less room for the static barriers.
constexpr int kDynSmemMax = 227 * 1024 - 1024 - 512;
int max_stages_for(int ncols_max) {
  return std::min(kMaxStages, (kDynSmemMax - kQStageBytes) / stage_bytes_for(ncols_max));
}

// Autotuned launch shapes: the stage-ring depth, the MMA shape (fused
// N = 2 ncols, or three MMAs of N = ncols) and, for level images, where the
// epilogue runs (four dedicated warps, or the producers between units; 22 or
// 18 warps per CTA), keyed by (accumulator width,
// station-chunk count rounded up to a power of two, operand type): the tuned
// shape holds for every batch with the same key in this process.
struct TuneKey {
  int ncols, chunks, fp16;
  bool operator<(const TuneKey& o) const {
    return ncols != o.ncols ? ncols < o.ncols : (chunks != o.chunks ? chunks < o.chunks : fp16 < o.fp16);
  }
};
struct TuneVal {
  int n_stages;
  bool fused, epw;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tuned;

TuneKey tune_key(const TcPlan& p) {
  int c = 1;
  while (c < p.max_chunks) c <<= 1;
  return TuneKey{p.ncols_max, c, (int)p.fp16};
}

// TMEM columns per accumulator buffer: a power of two holding the accumulator
// (2 ncols when fused).
void set_shape(TcPlan* p, bool fused) {
  p->fused = fused && 2 * p->ncols_max <= 256;
  p->ncols_buf = 32;
  while (p->ncols_buf < (p->fused ? 2 * p->ncols_max : p->ncols_max)) p->ncols_buf <<= 1;
}

int launch_kernel(const Batch& b, const Pixels& px, int n_level, double* img, const TcPlan& p, int n_stages,
                  TcWorkspace* w, cudaStream_t s) {
  const int stage_bytes = stage_bytes_for(p.ncols_max);
  const size_t smem = (size_t)n_stages * stage_bytes + kQStageBytes + 1024;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int n_tiles = (int)((px.n + kRows - 1) / kRows);
  const int grid = std::min(n_tiles, sms);
  int rc = 0;
  dispatch(n_level, p.fp16, p.fused, [&](auto L, auto FPV, auto FU) {
    constexpr int ML = decltype(L)::value;
    constexpr bool F16 = decltype(FPV)::value;
    constexpr bool FS = decltype(FU)::value;
    // dedicated epilogue warps for energy levels; eigenimages keep the epilogue in the
    // producers (their up to 64 images fit 16 register slots per thread only split four ways)
    auto go = [&](auto kern, int threads) {
      if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        rc = -7;
        return;
      }
      kern<<<grid, threads, smem, s>>>(b, px, n_level, img, TcYOut{}, w->steps, w->B, w->scale, w->qph,
                                       w->qph_stride, w->lwt, n_stages, stage_bytes, p.ncols_buf, w->status);
      if (cudaGetLastError() != cudaSuccess) rc = -11;  // the launch itself failed
    };
    if (b.eigen || !p.epw) go(k_synth_tc<ML, F16, FS, 0, false>, synth_threads(false));
    else go(k_synth_tc<ML, F16, FS, 0, true>, synth_threads(true));
  });
  return rc;
}

}  // namespace

int tc_prepare(const std::vector<int>& nst, const std::vector<int>& neig, bool fp16, TcWorkspace* w, TcPlan* p) {
  const int T = (int)nst.size();
  if (T > w->cap_T) return -2;
  long long off = 0;
  int ncols_max = 16, max_chunks = 1;
  for (int t = 0; t < T; ++t) {
    if (neig[t] > kTcMaxEig) return -3;
    TcStep& st = w->h_steps[t];
    st.b_off = off;
    st.n_chunks = n_chunks_for(nst[t]);
    st.ncols = ncols_for(neig[t]);
    st.idesc = make_idesc(st.ncols, fp16);
    st.idesc2 = make_idesc(std::min(2 * st.ncols, 256), fp16);
    off += (long long)st.n_chunks * st.ncols * 256;
    ncols_max = std::max(ncols_max, st.ncols);
    max_chunks = std::max(max_chunks, st.n_chunks);
  }
  if ((size_t)off > w->B_bytes) return -4;
  p->fp16 = fp16;
  p->ncols_max = ncols_max;
  p->max_chunks = max_chunks;
  const int smax = max_stages_for(ncols_max);
  if (smax < 2) return -6;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tuned.find(tune_key(*p));
  p->tuned = it != g_tuned.end();
  p->n_stages = p->tuned ? it->second.n_stages : smax;
  set_shape(p, p->tuned ? it->second.fused : true);  // untuned: fused where N = 2 ncols <= 256
  p->epw = p->tuned ? it->second.epw : true;
  return 0;
}

void tc_plan_force_fused(TcPlan* p) { set_shape(p, true); }

int tc_enqueue_pack(const Batch& b, const TcPlan& p, TcWorkspace* w, cudaStream_t s) {
  const int T = b.T;
  if (cudaMemcpyAsync(w->steps, w->h_steps, sizeof(TcStep) * T, cudaMemcpyHostToDevice, s) != cudaSuccess) return -5;
  if (cudaMemsetAsync(w->status, 0, sizeof(int), s) != cudaSuccess) return -5;
  if (p.fp16) k_tc_scale<<<T, 256, 0, s>>>(b, w->scale);
  if (p.fp16)
    k_tc_pack<true><<<dim3(p.max_chunks, T), 256, 0, s>>>(b, w->steps, w->B, w->scale, w->qph, w->qph_stride,
                                                          w->lwt);
  else
    k_tc_pack<false><<<dim3(p.max_chunks, T), 256, 0, s>>>(b, w->steps, w->B, w->scale, w->qph, w->qph_stride,
                                                           w->lwt);
  return cudaGetLastError() == cudaSuccess ? 0 : -5;
}

int tc_enqueue_synth(const Batch& b, const Pixels& px, int n_level, double* img, const TcPlan& p, TcWorkspace* w,
                     cudaStream_t s) {
  return launch_kernel(b, px, n_level, img, p, p.n_stages, w, s);
}

int tc_enqueue_yout(const Batch& b, const Pixels& px, int n_level, const TcPlan& p, TcWorkspace* w, TcYOut yo,
                    cudaStream_t s) {
  const int stage_bytes = stage_bytes_for(p.ncols_max);
  const size_t smem = (size_t)p.n_stages * stage_bytes + kQStageBytes + 1024;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int n_tiles = (int)((px.n + kRows - 1) / kRows);
  const int grid = std::min(n_tiles, sms);
  int rc = 0;
  dispatch(n_level, p.fp16, p.fused, [&](auto L, auto FPV, auto FU) {
    constexpr int ML = decltype(L)::value;
    constexpr bool F16 = decltype(FPV)::value;
    constexpr bool FS = decltype(FU)::value;
    if constexpr (ML != 4 || !FS) {  // the adjoint's Y stage is built for <= 4 levels and 2 n_eig <= 128 columns
      rc = -10;
    } else {
      if (cudaFuncSetAttribute(k_synth_tc<ML, F16, FS, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess) {
        rc = -7;
        return;
      }
      k_synth_tc<ML, F16, FS, 1, false><<<grid, kThreads, smem, s>>>(b, px, n_level, nullptr, yo, w->steps, w->B, w->scale,
                                                              w->qph, w->qph_stride, w->lwt, p.n_stages,
                                                              stage_bytes, p.ncols_buf, w->status);
      if (cudaGetLastError() != cudaSuccess) rc = -11;  // the launch itself failed
    }
  });
  return rc;
}

int tc_autotune(const Batch& b, const Pixels& px, int n_level, int n_chan_sub, TcPlan* p, TcWorkspace* w,
                cudaStream_t s) {
  // Time each feasible (MMA shape, stage count) on the first steps of the
  // batch and a pixel subset, into a scratch image (the real images are not
  // touched).
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  Batch bs = b;
  bs.T = std::min(b.T, 4);
  Pixels ps = px;
  ps.n = std::min<int64_t>(px.n, (int64_t)4 * sms * kRows);
  double* scratch = nullptr;
  const size_t bytes = sizeof(double) * (size_t)std::max(1, n_chan_sub) * n_level * ps.n;
  if (cudaMallocAsync(&scratch, bytes, s) != cudaSuccess) return -8;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  TcPlan best = *p;
  float best_ms = 1e30f;
  int rc = 0;
  const int n_shapes = (2 * p->ncols_max <= 256) ? 2 : 1;
  const int n_epw = b.eigen ? 1 : 2;  // eigenimages always run the epilogue in the producers
  for (int f = 0; f < n_shapes * n_epw && rc == 0; ++f) {
    TcPlan q = *p;
    set_shape(&q, f % n_shapes == 0 && n_shapes == 2);
    q.epw = f / n_shapes == 0;
    for (int ns = 2; ns <= max_stages_for(q.ncols_max) && rc == 0; ++ns) {
      rc = launch_kernel(bs, ps, n_level, scratch, q, ns, w, s);  // warm-up
      cudaEventRecord(e0, s);
      if (rc == 0) rc = launch_kernel(bs, ps, n_level, scratch, q, ns, w, s);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rc == 0 && ms < best_ms) {
        best_ms = ms;
        best = q;
        best.n_stages = ns;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(scratch, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return -9;
  if (rc) return rc;
  *p = best;
  p->tuned = true;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tuned[tune_key(*p)] = TuneVal{p->n_stages, p->fused, p->epw};
  return 0;
}

}  // namespace bipp
