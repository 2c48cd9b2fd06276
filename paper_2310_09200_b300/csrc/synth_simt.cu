// synth_simt.cu — CUDA-core standard synthesis (Sec. 2.4, Eq.
// standard_synthesis; Algorithm 2 "GEMMEXP"; Algorithm 1 lines 5-10):
//   z_e(r) = sum_i exp(-j 2 pi <r, p_i>/wl) a_ie,  I_l(r) += sum_{e in l} d_e |z_e(r)|^2
// for every step of a batch, accumulated in registers over the steps and
// added once to the FP64 image.
//
// A CTA owns 64 pixels. Per station chunk it writes the pixel x station
// phasor tile and the station x eigvec chunk of W to shared memory, then each
// thread accumulates 16 eigenvectors of one pixel (a small real GEMM on the
// FP32/FP64 pipes). One exp per (pixel, station) serves every eigenvector,
// as the paper's kernel does.
//
// FP32 variant: the phase t = <r, p_i/wl> (cycles) is reduced exactly mod 1
// from float hi/lo splits of r and p/wl: each hi*hi product is split into its
// rounded value and its exact FMA residual, the rounded value loses its
// integer part exactly (x - rint(x) is exact in FP32), and the remaining
// cross terms are below 2^-8 cycles, so the reduced phase carries an absolute
// error near 2^-24 cycles; sin/cos then run on the SFU.
#include <math.h>

#include <type_traits>

#include "bipp_internal.cuh"
#include "phase.cuh"

namespace bipp {

namespace {

constexpr int kPix = 64;        // pixels per CTA
constexpr int kStChunk = 64;    // stations per shared-memory chunk (FP32)
constexpr int kEigBlk = 64;     // eigenvectors per pass
constexpr int kThreads = 256;   // 64 pixels x 4 eigenvector groups
constexpr int kEigPerThr = kEigBlk / (kThreads / kPix);  // 16

template <int MAXL, typename T>
__device__ __forceinline__ void level_add(T (&acc)[MAXL], int lev, T v) {
#pragma unroll
  for (int l = 0; l < MAXL; ++l) acc[l] += (lev == l) ? v : T(0);
}

// ---------------------------------------------------------------- FP32

template <int MAXL>
__global__ void __launch_bounds__(kThreads) k_synth_f32(Batch b, Pixels px, int n_level, double* img) {
  if (*b.flag) return;  // some step of the batch failed: commit nothing
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sh_c = reinterpret_cast<float*>(smem_raw);                  // [kStChunk][kPix]
  float* sh_s = sh_c + kStChunk * kPix;                              // [kStChunk][kPix]
  float2* sh_w = reinterpret_cast<float2*>(sh_s + kStChunk * kPix);  // [kStChunk][kEigBlk]
  float* sh_red = sh_c;                                              // reused at the end: [4][MAXL][kPix]

  const int pl = threadIdx.x % kPix, eg = threadIdx.x / kPix;
  const int64_t r = (int64_t)blockIdx.x * kPix + pl;
  const bool valid = r < px.n;
  float rr[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) rr[c] = valid ? px.hl[(size_t)c * px.n + r] : 0.0f;

  float lacc[MAXL];
#pragma unroll
  for (int l = 0; l < MAXL; ++l) lacc[l] = 0.0f;

  const int N = b.n_max, KM = b.k_max;
  // reduce the 4 eigenvector groups, then one FP64 read-modify-write per pixel and level
  auto flush = [&](int chan) {
#pragma unroll
    for (int l = 0; l < MAXL; ++l) sh_red[(eg * MAXL + l) * kPix + pl] = lacc[l];
    __syncthreads();
    if (eg == 0 && valid) {
      double* im = img + (size_t)chan * n_level * px.n;
      if (b.eigen) {  // slot s of group g is eigenvector 4 s + g
        for (int l = 0; l < n_level; ++l) im[(size_t)l * px.n + r] += (double)sh_red[((l & 3) * MAXL + (l >> 2)) * kPix + pl];
      } else {
        for (int l = 0; l < n_level; ++l) {
          float s = 0.0f;
          for (int g = 0; g < kThreads / kPix; ++g) s += sh_red[(g * MAXL + l) * kPix + pl];
          im[(size_t)l * px.n + r] += (double)s;
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < MAXL; ++l) lacc[l] = 0.0f;
  };
  for (int t = 0; t < b.T; ++t) {
    const int n = b.nst[t], K = b.nkept[t];
    const float* q = b.q + (size_t)t * 6 * N;
    for (int e0 = 0; e0 < K; e0 += kEigBlk) {
      float zr[kEigPerThr], zi[kEigPerThr];
#pragma unroll
      for (int u = 0; u < kEigPerThr; ++u) zr[u] = zi[u] = 0.0f;
      for (int i0 = 0; i0 < n; i0 += kStChunk) {
        // phasor tile: this thread's pixel, stations eg*16 .. eg*16+15 of the chunk
#pragma unroll 4
        for (int u = 0; u < kStChunk / 4; ++u) {
          const int ii = eg * (kStChunk / 4) + u;
          const int i = i0 + ii;
          float cs = 0.0f, sn = 0.0f;
          if (i < n) {
            float qq[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) qq[c] = q[(size_t)c * N + i];
            sincos_cycles(phase_frac_f32(rr, qq), &sn, &cs);
          }
          sh_c[ii * kPix + pl] = cs;
          sh_s[ii * kPix + pl] = sn;
        }
        for (int w = threadIdx.x; w < kStChunk * kEigBlk; w += kThreads) {
          const int ii = w / kEigBlk, ee = w % kEigBlk;
          const int i = i0 + ii, e = e0 + ee;
          sh_w[w] = (i < n && e < K) ? b.W32[((size_t)t * N + i) * KM + e] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        const int iend = min(kStChunk, n - i0);
        for (int ii = 0; ii < iend; ++ii) {
          const float c = sh_c[ii * kPix + pl], s = sh_s[ii * kPix + pl];
#pragma unroll
          for (int u = 0; u < kEigPerThr; ++u) {
            const float2 w = sh_w[ii * kEigBlk + eg + 4 * u];
            // conj(Phi) * w = (c - j s)(wr + j wi)
            zr[u] = fmaf(c, w.x, fmaf(s, w.y, zr[u]));
            zi[u] = fmaf(c, w.y, fmaf(-s, w.x, zi[u]));
          }
        }
        __syncthreads();
      }
#pragma unroll
      for (int u = 0; u < kEigPerThr; ++u) {
        const int e = e0 + eg + 4 * u;
        if (e < K) {
          const int lev = b.level[(size_t)t * KM + e];
          if (lev >= 0)
            // eigenimages: slot (e - eg) / 4 of this thread's eigenvectors e = eg (mod 4)
            level_add<MAXL, float>(lacc, b.eigen ? e0 / 4 + u : lev, (float)b.wt[(size_t)t * KM + e] * (zr[u] * zr[u] + zi[u] * zi[u]));
        }
      }
    }
    if (last_of_chan(b, t)) flush(step_chan(b, t));
  }
}

// ---------------------------------------------------------------- FP64

constexpr int kStChunk64 = 32;

template <int MAXL>
__global__ void __launch_bounds__(kThreads) k_synth_f64(Batch b, Pixels px, int n_level, double* img) {
  if (*b.flag) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sh_c = reinterpret_cast<double*>(smem_raw);                    // [kStChunk64][kPix]
  double* sh_s = sh_c + kStChunk64 * kPix;                               // [kStChunk64][kPix]
  double2* sh_w = reinterpret_cast<double2*>(sh_s + kStChunk64 * kPix);  // [kStChunk64][kEigBlk]
  double* sh_red = sh_c;  // [4][MAXL][kPix] spans sh_c and sh_s

  const int pl = threadIdx.x % kPix, eg = threadIdx.x / kPix;
  const int64_t r = (int64_t)blockIdx.x * kPix + pl;
  const bool valid = r < px.n;
  const double rx = valid ? px.xyz[r] : 0.0, ry = valid ? px.xyz[px.n + r] : 0.0,
               rz = valid ? px.xyz[2 * px.n + r] : 0.0;

  double lacc[MAXL];
#pragma unroll
  for (int l = 0; l < MAXL; ++l) lacc[l] = 0.0;
  const int N = b.n_max, KM = b.k_max;
  auto flush = [&](int chan) {
#pragma unroll
    for (int l = 0; l < MAXL; ++l) sh_red[(eg * MAXL + l) * kPix + pl] = lacc[l];
    __syncthreads();
    if (eg == 0 && valid) {
      double* im = img + (size_t)chan * n_level * px.n;
      if (b.eigen) {  // slot s of group g is eigenvector 4 s + g
        for (int l = 0; l < n_level; ++l) im[(size_t)l * px.n + r] += sh_red[((l & 3) * MAXL + (l >> 2)) * kPix + pl];
      } else {
        for (int l = 0; l < n_level; ++l) {
          double s = 0.0;
          for (int g = 0; g < kThreads / kPix; ++g) s += sh_red[(g * MAXL + l) * kPix + pl];
          im[(size_t)l * px.n + r] += s;
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < MAXL; ++l) lacc[l] = 0.0;
  };
  for (int t = 0; t < b.T; ++t) {
    const int n = b.nst[t], K = b.nkept[t];
    const double k = 2.0 * M_PI / b.wl[t];
    const double* p = b.st + (size_t)t * 3 * N;
    for (int e0 = 0; e0 < K; e0 += kEigBlk) {
      double zr[kEigPerThr], zi[kEigPerThr];
#pragma unroll
      for (int u = 0; u < kEigPerThr; ++u) zr[u] = zi[u] = 0.0;
      for (int i0 = 0; i0 < n; i0 += kStChunk64) {
        for (int u = 0; u < kStChunk64 / 4; ++u) {
          const int ii = eg * (kStChunk64 / 4) + u;
          const int i = i0 + ii;
          double cs = 0.0, sn = 0.0;
          if (i < n) {
            const double arg = k * (rx * p[i] + ry * p[N + i] + rz * p[2 * N + i]);
            sincos(arg, &sn, &cs);
          }
          sh_c[ii * kPix + pl] = cs;
          sh_s[ii * kPix + pl] = sn;
        }
        for (int w = threadIdx.x; w < kStChunk64 * kEigBlk; w += kThreads) {
          const int ii = w / kEigBlk, ee = w % kEigBlk;
          const int i = i0 + ii, e = e0 + ee;
          sh_w[w] = (i < n && e < K) ? b.W64[((size_t)t * KM + e) * N + i] : make_double2(0.0, 0.0);
        }
        __syncthreads();
        const int iend = min(kStChunk64, n - i0);
        for (int ii = 0; ii < iend; ++ii) {
          const double c = sh_c[ii * kPix + pl], s = sh_s[ii * kPix + pl];
#pragma unroll
          for (int u = 0; u < kEigPerThr; ++u) {
            const double2 w = sh_w[ii * kEigBlk + eg + 4 * u];
            zr[u] = fma(c, w.x, fma(s, w.y, zr[u]));
            zi[u] = fma(c, w.y, fma(-s, w.x, zi[u]));
          }
        }
        __syncthreads();
      }
#pragma unroll
      for (int u = 0; u < kEigPerThr; ++u) {
        const int e = e0 + eg + 4 * u;
        if (e < K) {
          const int lev = b.level[(size_t)t * KM + e];
          if (lev >= 0)
            // eigenimages: slot (e - eg) / 4 of this thread's eigenvectors e = eg (mod 4)
            level_add<MAXL, double>(lacc, b.eigen ? e0 / 4 + u : lev, b.wt[(size_t)t * KM + e] * (zr[u] * zr[u] + zi[u] * zi[u]));
        }
      }
    }
    if (last_of_chan(b, t)) flush(step_chan(b, t));
  }
}

template <typename F>
void dispatch_levels(int n_level, F&& f) {
  if (n_level <= 4) f(std::integral_constant<int, 4>{});
  else if (n_level <= 8) f(std::integral_constant<int, 8>{});
  else f(std::integral_constant<int, 16>{});
}

}  // namespace

void launch_synth_simt_f32(const Batch& b, const Pixels& px, int n_level, double* img, cudaStream_t s) {
  const size_t smem = (size_t)kStChunk * kPix * 4 * 2 + (size_t)kStChunk * kEigBlk * 8;
  const unsigned grid = (unsigned)((px.n + kPix - 1) / kPix);
  dispatch_levels(n_level, [&](auto L) {
    constexpr int ML = decltype(L)::value;
    cudaFuncSetAttribute(k_synth_f32<ML>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_synth_f32<ML><<<grid, kThreads, smem, s>>>(b, px, n_level, img);
  });
}

void launch_synth_simt_f64(const Batch& b, const Pixels& px, int n_level, double* img, cudaStream_t s) {
  const size_t smem = (size_t)kStChunk64 * kPix * 8 * 2 + (size_t)kStChunk64 * kEigBlk * 16;
  const unsigned grid = (unsigned)((px.n + kPix - 1) / kPix);
  dispatch_levels(n_level, [&](auto L) {
    constexpr int ML = decltype(L)::value;
    cudaFuncSetAttribute(k_synth_f64<ML>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_synth_f64<ML><<<grid, kThreads, smem, s>>>(b, px, n_level, img);
  });
}

}  // namespace bipp
