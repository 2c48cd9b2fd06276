// adjoint.cu — differentiable synthesis with station gains (forward and
// hand-written adjoint), device-pointer entry points for the autograd glue.
//
// Model (Sec. 2.1 sampling operator with direction-independent gains g_i,
// Eq. standard_synthesis, Algorithm 1 accumulation over steps):
//   z_te(r) = sum_i conj(g_i exp(j th_tri)) W_t,ie = sum_i conj(Phi_t(r,i)) W'_t,ie,  W' = diag(conj g) W
//   I_l(r)  = sum_t sum_{e: level_te = l} d_te |z_te(r)|^2
// Given R_l(r) = dL/dI_l(r) for a real loss L, with complex gradients in the
// convention grad = dL/dRe + j dL/dIm:
//   Y_te(r)        = d_te R_{l(te)}(r) z_te(r)
//   grad_W'_t[i,e] = 2 sum_r Phi_t(r,i) Y_te(r)        (Phi, not its conjugate)
//   grad_W_t[i,e]  = g_i grad_W'_t[i,e]
//   grad_g[i]      = sum_t sum_e conj(grad_W'_t[i,e]) W_t[i,e]
// Both paths recompute Phi (once for z, once for the pixel contraction)
// instead of storing it, and reduce over pixels in two deterministic stages
// (per-CTA partial sums, then a fixed-order sum over CTAs):
//   - precision BIPP_PREC_SPLIT_FP16 / _BF16 (n_eig <= 64, n_level <= 4 for
//     the adjoint): the forward is the tensor-core synthesis kernel on W'
//     (packed like the eigenvectors of a collect); the adjoint recomputes z
//     with the same kernel, whose epilogue writes Y instead of |z|^2, and runs
//     the pixel contraction Phi^T Y on the tensor cores (adjoint_tc.cu);
//   - BIPP_PREC_FP32: the CUDA-core kernels below (FP32 sums).
#include <math.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "bipp_internal.cuh"
#include "bipp_ss.h"
#include "phase.cuh"
#include "synth_tc.cuh"

namespace bipp {
namespace {

constexpr int kPix = 64;
constexpr int kSt = 64;
constexpr int kThreads = 256;
constexpr int kEb = 64;        // eigenvectors per pass (<= 16 per thread)
constexpr int kAccMax = 12288; // complex accumulators per CTA (96 KB of shared memory)

// W'_t = diag(conj g) W_t into the station-major FP32 layout of the synthesis
// kernels, plus weights, levels and station hi/lo coordinates of each step.
__global__ void k_adj_prep(Batch b, const double2* W, const double* d, const int* level, const double2* g,
                           const double* st, double wl, int* nst, int* nkept) {
  const int t = blockIdx.x;
  const int N = b.n_max, K = b.k_max;
  for (int w = threadIdx.x; w < N * K; w += blockDim.x) {
    const int i = w % N, e = w / N;
    const double2 a = W[((size_t)t * K + e) * N + i];
    const double2 gi = g[i];
    // conj(g) * a
    const double re = gi.x * a.x + gi.y * a.y, im = gi.x * a.y - gi.y * a.x;
    b.W32[((size_t)t * N + i) * K + e] = make_float2((float)re, (float)im);
  }
  for (int e = threadIdx.x; e < K; e += blockDim.x) {
    b.wt[(size_t)t * K + e] = d[(size_t)t * K + e];
    b.level[(size_t)t * K + e] = level[(size_t)t * K + e];
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    for (int c = 0; c < 3; ++c) {
      const double v = st[((size_t)t * 3 + c) * N + i] / wl;
      const float hi = (float)v;
      b.q[((size_t)t * 6 + c) * N + i] = hi;
      b.q[((size_t)t * 6 + c + 3) * N + i] = (float)(v - (double)hi);
    }
  }
  if (threadIdx.x == 0) {
    nst[t] = N;
    nkept[t] = K;
  }
}

// Fused adjoint: one persistent CTA loops over (step, 64-pixel tile); for an
// eigenvector block [e0, e0+eb) it recomputes z (pass 1), forms Y in shared
// memory, recomputes Phi and accumulates Phi^T Y into a per-CTA shared-memory
// partial (pass 2). The partial of step t is written to part[t][cta].
__global__ void __launch_bounds__(kThreads) k_adjoint(Batch b, Pixels px, int n_level, const double* R, int e0,
                                                      int eb, float2* part) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int N = b.n_max, K = b.k_max;
  float2* acc = reinterpret_cast<float2*>(sm);                  // [N][eb]
  float* sh_c = reinterpret_cast<float*>(acc + (size_t)N * eb);  // [kSt][kPix] pass 1 / [kPix][kSt] pass 2
  float* sh_s = sh_c + kSt * kPix;
  float2* sh_w = reinterpret_cast<float2*>(sh_s + kSt * kPix);  // [kSt][kEb] (pass 1)
  float2* sh_y = sh_w + kSt * kEb;                              // [kPix][kEb]
  float* sh_px = reinterpret_cast<float*>(sh_y + kPix * kEb);   // [6][kPix]

  const int tid = threadIdx.x, lo = tid % kPix, eg = tid / kPix;
  const int n_tiles = (int)((px.n + kPix - 1) / kPix);
  for (int t = 0; t < b.T; ++t) {
    const float* q = b.q + (size_t)t * 6 * N;
    for (int w = tid; w < N * eb; w += kThreads) acc[w] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
      const int64_t r0 = (int64_t)tile * kPix;
      for (int w = tid; w < 6 * kPix; w += kThreads) {
        const int c = w / kPix, p = w % kPix;
        sh_px[w] = (r0 + p < px.n) ? px.hl[(size_t)c * px.n + r0 + p] : 0.0f;
      }
      __syncthreads();
      // ---- pass 1: z(r, e) for this thread's pixel lo and eigenvectors e0 + eg + 4u
      float rr[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) rr[c] = sh_px[c * kPix + lo];
      float zr[16], zi[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) zr[u] = zi[u] = 0.f;
      for (int i0 = 0; i0 < N; i0 += kSt) {
        for (int u = 0; u < kSt / 4; ++u) {
          const int ii = eg * (kSt / 4) + u, i = i0 + ii;
          float cs = 0.f, sn = 0.f;
          if (i < N) {
            float qq[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) qq[c] = q[(size_t)c * N + i];
            sincos_cycles(phase_frac_f32(rr, qq), &sn, &cs);
          }
          sh_c[ii * kPix + lo] = cs;
          sh_s[ii * kPix + lo] = sn;
        }
        for (int w = tid; w < kSt * kEb; w += kThreads) {
          const int ii = w / kEb, ee = w % kEb, i = i0 + ii;
          sh_w[w] = (i < N && ee < eb) ? b.W32[((size_t)t * N + i) * K + e0 + ee] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        const int iend = min(kSt, N - i0);
        for (int ii = 0; ii < iend; ++ii) {
          const float c = sh_c[ii * kPix + lo], s = sh_s[ii * kPix + lo];
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const float2 w = sh_w[ii * kEb + eg + 4 * u];
            zr[u] = fmaf(c, w.x, fmaf(s, w.y, zr[u]));
            zi[u] = fmaf(c, w.y, fmaf(-s, w.x, zi[u]));
          }
        }
        __syncthreads();
      }
      // Y(r, e) = d_e R_l(r) z(r, e)
      const int64_t r = r0 + lo;
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int ee = eg + 4 * u;
        float2 y = make_float2(0.f, 0.f);
        if (ee < eb && r < px.n) {
          const int e = e0 + ee;
          const int lev = b.level[(size_t)t * K + e];
          if (lev >= 0 && lev < n_level) {
            const float f = (float)(b.wt[(size_t)t * K + e] * R[(size_t)lev * px.n + r]);
            y = make_float2(f * zr[u], f * zi[u]);
          }
        }
        sh_y[lo * kEb + ee] = y;
      }
      __syncthreads();
      // ---- pass 2: acc[i][e] += sum_r Phi(r,i) Y(r,e); thread = station lo of the chunk, eigvecs eg + 4u
      for (int i0 = 0; i0 < N; i0 += kSt) {
        const int i = i0 + lo;
        float qq[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) qq[c] = (i < N) ? q[(size_t)c * N + i] : 0.f;
        for (int u = 0; u < kPix / 4; ++u) {
          const int p = eg * (kPix / 4) + u;
          float pr[6];
#pragma unroll
          for (int c = 0; c < 6; ++c) pr[c] = sh_px[c * kPix + p];
          float cs = 0.f, sn = 0.f;
          if (i < N) sincos_cycles(phase_frac_f32(pr, qq), &sn, &cs);
          sh_c[p * kSt + lo] = cs;
          sh_s[p * kSt + lo] = sn;
        }
        __syncthreads();
        float ar[16], ai[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) ar[u] = ai[u] = 0.f;
        for (int p = 0; p < kPix; ++p) {
          const float c = sh_c[p * kSt + lo], s = sh_s[p * kSt + lo];
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const float2 y = sh_y[p * kEb + eg + 4 * u];
            // (c + j s)(yr + j yi)
            ar[u] = fmaf(c, y.x, fmaf(-s, y.y, ar[u]));
            ai[u] = fmaf(c, y.y, fmaf(s, y.x, ai[u]));
          }
        }
        if (i < N) {
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const int ee = eg + 4 * u;
            if (ee < eb) {
              float2 a = acc[(size_t)i * eb + ee];
              acc[(size_t)i * eb + ee] = make_float2(a.x + ar[u], a.y + ai[u]);
            }
          }
        }
        __syncthreads();
      }
    }
    // per-CTA partial of step t
    for (int w = tid; w < N * eb; w += kThreads) part[((size_t)t * gridDim.x + blockIdx.x) * N * eb + w] = acc[w];
    __syncthreads();
  }
}

// grad_W'_t[i, e0+ee] = 2 sum_cta part[t][cta][i][ee], summed in CTA order.
__global__ void k_adj_reduce(const float2* part, int T, int n_cta, int N, int K, int e0, int eb, double2* gWp) {
  const int t = blockIdx.y;
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= N * eb) return;
  const int i = w / eb, ee = w % eb;
  double sr = 0.0, si = 0.0;
  for (int c = 0; c < n_cta; ++c) {
    const float2 v = part[((size_t)t * n_cta + c) * N * eb + w];
    sr += v.x;
    si += v.y;
  }
  gWp[((size_t)t * K + e0 + ee) * N + i] = make_double2(2.0 * sr, 2.0 * si);
}

// grad_W = g * grad_W' (in place), grad_g[i] = sum_t sum_e conj(grad_W'_t[i,e]) W_t[i,e].
// Block of 256 threads = 32 stations x 8 slices of the (t, e) pairs; the 8
// partial sums of a station are added in a fixed order (deterministic).
__global__ void __launch_bounds__(256) k_adj_finish(int T, int N, int K, const double2* W, const double2* g,
                                                    double2* gW, double2* gg) {
  const int li = threadIdx.x & 31, sl = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + li;
  __shared__ double2 part[8][32];
  double sr = 0.0, si = 0.0;
  if (i < N) {
    const double2 gi = g[i];
    for (int te = sl; te < T * K; te += 8) {
      const size_t o = (size_t)te * N + i;
      const double2 p = gW[o], w = W[o];
      sr += p.x * w.x + p.y * w.y;  // conj(p) * w
      si += p.x * w.y - p.y * w.x;
      gW[o] = make_double2(gi.x * p.x - gi.y * p.y, gi.x * p.y + gi.y * p.x);
    }
  }
  part[sl][li] = make_double2(sr, si);
  __syncthreads();
  if (sl == 0 && i < N) {
    double2 a = part[0][li];
    for (int k = 1; k < 8; ++k) {
      a.x += part[k][li].x;
      a.y += part[k][li].y;
    }
    gg[i] = a;
  }
}

struct Scratch {
  Batch b{};
  int* nst = nullptr;
  int* nkept = nullptr;
  int* flag = nullptr;
  float* hl = nullptr;
  void* base = nullptr;
};

cudaError_t prep(Scratch* s, int64_t n_pix, const double* d_pix, double wl, int T, int N, int K,
                 const double* d_st, const double* d_W, const double* d_d, const int32_t* d_level,
                 const double* d_g, cudaStream_t st) {
  auto rnd = [](size_t n) { return (n + 255) & ~size_t(255); };
  const size_t bytes = rnd(sizeof(float2) * (size_t)T * N * K) + rnd(sizeof(double) * (size_t)T * K) +
                       rnd(sizeof(int) * (size_t)T * K) + rnd(sizeof(float) * (size_t)T * 6 * N) +
                       2 * rnd(sizeof(int) * (size_t)T) + rnd(sizeof(int)) + rnd(sizeof(float) * 6 * (size_t)n_pix);
  cudaError_t e = cudaMallocAsync(&s->base, bytes, st);
  if (e != cudaSuccess) return e;
  unsigned char* p = static_cast<unsigned char*>(s->base);
  auto take = [&](size_t n) {  // consecutive 256-byte-aligned regions, exactly `bytes` in total
    unsigned char* r = p;
    p += rnd(n);
    return r;
  };
  Batch& b = s->b;
  b.T = T;
  b.n_max = N;
  b.k_max = K;
  b.wl = nullptr;    // the FP32 synthesis reads station coordinates already divided by wl
  b.chan = nullptr;  // one channel
  b.W32 = reinterpret_cast<float2*>(take(sizeof(float2) * (size_t)T * N * K));
  b.wt = reinterpret_cast<double*>(take(sizeof(double) * (size_t)T * K));
  b.level = reinterpret_cast<int*>(take(sizeof(int) * (size_t)T * K));
  b.q = reinterpret_cast<float*>(take(sizeof(float) * (size_t)T * 6 * N));
  s->nst = reinterpret_cast<int*>(take(sizeof(int) * T));
  s->nkept = reinterpret_cast<int*>(take(sizeof(int) * T));
  s->flag = reinterpret_cast<int*>(take(sizeof(int)));
  s->hl = reinterpret_cast<float*>(take(sizeof(float) * 6 * (size_t)n_pix));
  b.nst = s->nst;
  b.nkept = s->nkept;
  b.flag = s->flag;
  if ((e = cudaMemsetAsync(s->flag, 0, sizeof(int), st)) != cudaSuccess) return e;
  k_adj_prep<<<T, 256, 0, st>>>(b, reinterpret_cast<const double2*>(d_W), d_d, d_level,
                                 reinterpret_cast<const double2*>(d_g), d_st, wl, s->nst, s->nkept);
  launch_pixel_split(d_pix, s->hl, n_pix, st);
  return cudaGetLastError();
}

int check(int64_t n_pix, int T, int N, int K, int n_level, const void* a, const void* b2, const void* c,
          const void* d, const void* e, const void* f, const void* g) {
  if (n_pix < 1 || T < 1 || N < 1 || N > kMaxStations || K < 1 || K > N || n_level < 1 || n_level > kMaxLevels)
    return BIPP_ERR_INVALID_ARG;
  if (!a || !b2 || !c || !d || !e || !f || !g) return BIPP_ERR_INVALID_ARG;
  return BIPP_OK;
}

// ---- tensor-core path: W' = diag(conj g) W in the e-major FP64 layout of a
// batch's kept eigenvectors, with its weights, levels, counts and wavelength,
// so that the packing and synthesis kernels of a collect run on it unchanged.
__global__ void k_adj_prep_tc(Batch b, const double2* W, const double* d, const int* level, const double2* g,
                              double wl, int* nst, int* nkept, double* wls) {
  const int t = blockIdx.x;
  const int N = b.n_max, K = b.k_max;
  for (int w = threadIdx.x; w < N * K; w += blockDim.x) {
    const int i = w % N, e = w / N;
    const size_t o = ((size_t)t * K + e) * N + i;
    const double2 a = W[o], gi = g[i];
    b.W64[o] = make_double2(gi.x * a.x + gi.y * a.y, gi.x * a.y - gi.y * a.x);  // conj(g) a
  }
  for (int e = threadIdx.x; e < K; e += blockDim.x) {
    b.wt[(size_t)t * K + e] = d[(size_t)t * K + e];
    b.level[(size_t)t * K + e] = level[(size_t)t * K + e];
  }
  if (threadIdx.x == 0) {
    nst[t] = N;
    nkept[t] = K;
    wls[t] = wl;
  }
}

// One tensor-core workspace per device, and its scratch buffers (the batch
// view of W', the adjoint's Y images and per-CTA partials), grown on demand and
// kept: a call holds the device's lock from packing to its final
// synchronisation.
constexpr int kTcDevs = 64;
std::mutex g_tc_mu[kTcDevs];
TcWorkspace g_tc_ws[kTcDevs];
int g_tc_cap[kTcDevs][3];
struct DevBuf {
  void* p = nullptr;
  size_t n = 0;
};
DevBuf g_tc_buf[kTcDevs][3];

// Buffer `slot` of the device, at least `bytes` long; the caller holds g_tc_mu[dev].
void* tc_buf(int dev, int slot, size_t bytes) {
  DevBuf& b = g_tc_buf[dev][slot];
  if (b.p && b.n >= bytes) return b.p;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.n = 0;
  if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
    (void)cudaGetLastError();
    b.p = nullptr;
    return nullptr;
  }
  b.n = bytes;
  return b.p;
}

struct TcScratch {
  Batch b{};
  void* base = nullptr;
};

size_t rnd256(size_t n) { return (n + 255) & ~size_t(255); }
size_t prep_tc_bytes(int T, int N, int K) {
  return rnd256(sizeof(double2) * (size_t)T * N * K) + rnd256(sizeof(double) * (size_t)T * K) +
         rnd256(sizeof(int) * (size_t)T * K) + 2 * rnd256(sizeof(int) * (size_t)T) + rnd256(sizeof(double) * (size_t)T) +
         rnd256(sizeof(int));
}

// base: prep_tc_bytes(T, N, K) bytes of device scratch.
cudaError_t prep_tc(TcScratch* s, void* base, int T, int N, int K, const double* d_st, const double* d_W,
                    const double* d_d, const int32_t* d_level, const double* d_g, double wl, cudaStream_t st) {
  auto rnd = rnd256;
  cudaError_t e = cudaSuccess;
  s->base = base;
  unsigned char* p = static_cast<unsigned char*>(base);
  auto take = [&](size_t n) {
    unsigned char* r = p;
    p += rnd(n);
    return r;
  };
  Batch& b = s->b;
  b.T = T;
  b.n_max = N;
  b.k_max = K;
  b.st = d_st;
  b.chan = nullptr;
  b.eigen = 0;
  b.W64 = reinterpret_cast<double2*>(take(sizeof(double2) * (size_t)T * N * K));
  b.wt = reinterpret_cast<double*>(take(sizeof(double) * (size_t)T * K));
  b.level = reinterpret_cast<int*>(take(sizeof(int) * (size_t)T * K));
  int* nst = reinterpret_cast<int*>(take(sizeof(int) * T));
  int* nkept = reinterpret_cast<int*>(take(sizeof(int) * T));
  double* wls = reinterpret_cast<double*>(take(sizeof(double) * T));
  int* flag = reinterpret_cast<int*>(take(sizeof(int)));
  b.nst = nst;
  b.neig = nkept;
  b.nkept = nkept;
  b.wl = wls;
  b.flag = flag;
  if ((e = cudaMemsetAsync(flag, 0, sizeof(int), st)) != cudaSuccess) return e;
  k_adj_prep_tc<<<T, 256, 0, st>>>(b, reinterpret_cast<const double2*>(d_W), d_d, d_level,
                                   reinterpret_cast<const double2*>(d_g), wl, nst, nkept, wls);
  return cudaGetLastError();
}

// The device's workspace, sized for (T, N, K); the caller holds g_tc_mu[dev].
TcWorkspace* tc_ws(int dev, int T, int N, int K) {
  int* c = g_tc_cap[dev];
  if (g_tc_ws[dev].B && T <= c[0] && N <= c[1] && K <= c[2]) return &g_tc_ws[dev];
  T = std::max(T, c[0]);
  N = std::max(N, c[1]);
  K = std::max(K, c[2]);
  if (tc_alloc(&g_tc_ws[dev], T, N, K)) {
    tc_free(&g_tc_ws[dev]);
    c[0] = c[1] = c[2] = 0;
    return nullptr;
  }
  c[0] = T;
  c[1] = N;
  c[2] = K;
  return &g_tc_ws[dev];
}

int err_of(cudaError_t e) {
  return e == cudaSuccess ? BIPP_OK : (e == cudaErrorMemoryAllocation ? BIPP_ERR_OUT_OF_MEMORY : BIPP_ERR_CUDA);
}

// Forward or adjoint on the tensor cores; R == nullptr: forward into img.
int run_tc(int64_t n_pix, const double* d_pix, double wl, int T, int N, int K, int n_level, const double* d_st,
           const double* d_W, const double* d_d, const int32_t* d_level, const double* d_g, bool fp16, double* img,
           const double* R, double* gW, double* gg, cudaStream_t s) {
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kTcDevs) return BIPP_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  std::lock_guard<std::mutex> lock(g_tc_mu[dev]);
  TcWorkspace* w = tc_ws(dev, T, N, K);
  if (!w) return BIPP_ERR_OUT_OF_MEMORY;
  TcScratch sc;
  unsigned char* Y = nullptr;
  float* part = nullptr;
  int rc = BIPP_OK;
  void* pbase = tc_buf(dev, 0, prep_tc_bytes(T, N, K));
  if (!pbase) return BIPP_ERR_OUT_OF_MEMORY;
  cudaError_t e = prep_tc(&sc, pbase, T, N, K, d_st, d_W, d_d, d_level, d_g, wl, s);
  TcPlan plan;
  if (e == cudaSuccess) {
    const std::vector<int> nst(T, N), neig(T, K);
    if (tc_prepare(nst, neig, fp16, w, &plan)) rc = BIPP_ERR_UNSUPPORTED;
    else if (R) tc_plan_force_fused(&plan);  // the Y stage is built for the fused shape
  }
  if (e == cudaSuccess && rc == BIPP_OK && tc_enqueue_pack(sc.b, plan, w, s)) e = cudaErrorLaunchFailure;
  if (e == cudaSuccess && rc == BIPP_OK) {
    Pixels px{n_pix, d_pix, nullptr};  // the tensor-core kernels form their integer phase words from FP64
    if (!R) {
      e = cudaMemsetAsync(img, 0, sizeof(double) * n_pix * n_level, s);
      if (e == cudaSuccess && tc_enqueue_synth(sc.b, px, n_level, img, plan, w, s)) e = cudaErrorLaunchFailure;
    } else {
      const int nc64 = (int)((n_pix + 63) / 64);
      const int ncols = plan.ncols_max;
      const int grid = std::max(1, std::min(nc64, sms));
      Y = static_cast<unsigned char*>(tc_buf(dev, 1, (size_t)T * nc64 * 2 * ncols * 128));
      part = static_cast<float*>(tc_buf(dev, 2, sizeof(float) * (size_t)T * grid * 2 * N * ncols));
      if (!Y || !part) e = cudaErrorMemoryAllocation;
      if (e == cudaSuccess) {
        TcYOut yo;
        yo.R = R;
        yo.Y = Y;
        yo.nc64 = nc64;
        const int yr = tc_enqueue_yout(sc.b, px, n_level, plan, w, yo, s);
        if (yr) rc = (yr == -11) ? BIPP_ERR_CUDA : BIPP_ERR_UNSUPPORTED;  // -11: the launch failed
      }
      if (e == cudaSuccess && rc == BIPP_OK &&
          launch_adjoint_tc(px, T, N, K, ncols, w->qph, w->qph_stride, Y, nc64, part, grid,
                            reinterpret_cast<double2*>(gW), w->status, s))
        e = cudaErrorLaunchFailure;
      if (e == cudaSuccess && rc == BIPP_OK) {
        k_adj_finish<<<(N + 31) / 32, 256, 0, s>>>(T, N, K, reinterpret_cast<const double2*>(d_W),
                                                     reinterpret_cast<const double2*>(d_g),
                                                     reinterpret_cast<double2*>(gW), reinterpret_cast<double2*>(gg));
        e = cudaGetLastError();
      }
    }
  }
  const cudaError_t es = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = es;
  if (rc == BIPP_OK) rc = err_of(e);
  if (rc == BIPP_OK && tc_read_status(w) != 0) rc = BIPP_ERR_DEVICE_TIMEOUT;
  if (rc == BIPP_OK && sc.b.flag) {  // a station beyond the phase's range (k_tc_pack): nothing was computed
    int fl = 0;
    if (cudaMemcpy(&fl, sc.b.flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) rc = BIPP_ERR_CUDA;
    else if (fl & kStatusRange) rc = BIPP_ERR_UNSUPPORTED;
  }
  return rc;
}

}  // namespace
}  // namespace bipp

using namespace bipp;

extern "C" int bipp_ss_synth_levels_device(int64_t n_pix, const double* d_pix, double wl, int32_t n_t,
                                           int32_t n_st, int32_t n_eig, int32_t n_level, const double* d_st_xyz,
                                           const double* d_W, const double* d_d, const int32_t* d_level,
                                           const double* d_gains, double* d_img, int32_t precision, void* stream) {
  int rc = check(n_pix, n_t, n_st, n_eig, n_level, d_pix, d_st_xyz, d_W, d_d, d_level, d_gains, d_img);
  if (rc || !(wl > 0.0)) return BIPP_ERR_INVALID_ARG;
  if (precision != BIPP_PREC_FP32 && precision != BIPP_PREC_SPLIT_BF16 && precision != BIPP_PREC_SPLIT_FP16)
    return BIPP_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision != BIPP_PREC_FP32) {
    (void)cudaGetLastError();
    if (n_eig > kTcMaxEig) return BIPP_ERR_UNSUPPORTED;
    return run_tc(n_pix, d_pix, wl, n_t, n_st, n_eig, n_level, d_st_xyz, d_W, d_d, d_level, d_gains,
                  precision == BIPP_PREC_SPLIT_FP16, d_img, nullptr, nullptr, nullptr, s);
  }
  Scratch sc;
  cudaError_t e = prep(&sc, n_pix, d_pix, wl, n_t, n_st, n_eig, d_st_xyz, d_W, d_d, d_level, d_gains, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_img, 0, sizeof(double) * n_pix * n_level, s);
  if (e == cudaSuccess) {
    Pixels px{n_pix, d_pix, sc.hl};
    launch_synth_simt_f32(sc.b, px, n_level, d_img, s);
    e = cudaGetLastError();
  }
  if (sc.base) cudaFreeAsync(sc.base, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? BIPP_OK : (e == cudaErrorMemoryAllocation ? BIPP_ERR_OUT_OF_MEMORY : BIPP_ERR_CUDA);
}

extern "C" int bipp_ss_synth_adjoint_device(int64_t n_pix, const double* d_pix, double wl, int32_t n_t,
                                            int32_t n_st, int32_t n_eig, int32_t n_level, const double* d_st_xyz,
                                            const double* d_W, const double* d_d, const int32_t* d_level,
                                            const double* d_gains, const double* d_grad_img, double* d_grad_W,
                                            double* d_grad_g, int32_t precision, void* stream) {
  int rc = check(n_pix, n_t, n_st, n_eig, n_level, d_pix, d_st_xyz, d_W, d_d, d_level, d_gains, d_grad_img);
  if (rc || !d_grad_W || !d_grad_g || !(wl > 0.0)) return BIPP_ERR_INVALID_ARG;
  if (precision != BIPP_PREC_FP32 && precision != BIPP_PREC_SPLIT_BF16 && precision != BIPP_PREC_SPLIT_FP16)
    return BIPP_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision != BIPP_PREC_FP32) {
    (void)cudaGetLastError();
    if (n_eig > 64 || n_level > 4) return BIPP_ERR_UNSUPPORTED;
    return run_tc(n_pix, d_pix, wl, n_t, n_st, n_eig, n_level, d_st_xyz, d_W, d_d, d_level, d_gains,
                  precision == BIPP_PREC_SPLIT_FP16, nullptr, d_grad_img, d_grad_W, d_grad_g, s);
  }
  Scratch sc;
  cudaError_t e = prep(&sc, n_pix, d_pix, wl, n_t, n_st, n_eig, d_st_xyz, d_W, d_d, d_level, d_gains, s);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int n_tiles = (int)((n_pix + kPix - 1) / kPix);
  const int grid = std::max(1, std::min(n_tiles, sms));
  // eigenvector block so that the per-CTA accumulator (n_st x eb complex) fits 128 KB
  const int eb = std::max(1, std::min(std::min(n_eig, kEb), kAccMax / n_st));
  float2* part = nullptr;
  if (e == cudaSuccess) e = cudaMallocAsync(&part, sizeof(float2) * (size_t)n_t * grid * n_st * eb, s);
  const size_t smem = sizeof(float2) * (size_t)n_st * eb + sizeof(float) * 2 * kSt * kPix +
                      sizeof(float2) * kSt * kEb + sizeof(float2) * kPix * kEb + sizeof(float) * 6 * kPix;
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_adjoint, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  Pixels px{n_pix, d_pix, sc.hl};
  for (int e0 = 0; e == cudaSuccess && e0 < n_eig; e0 += eb) {
    const int ebb = std::min(eb, n_eig - e0);
    k_adjoint<<<grid, kThreads, smem, s>>>(sc.b, px, n_level, d_grad_img, e0, ebb, part);
    k_adj_reduce<<<dim3((n_st * ebb + 255) / 256, n_t), 256, 0, s>>>(part, n_t, grid, n_st, n_eig, e0, ebb,
                                                                     reinterpret_cast<double2*>(d_grad_W));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_adj_finish<<<(n_st + 31) / 32, 256, 0, s>>>(n_t, n_st, n_eig, reinterpret_cast<const double2*>(d_W),
                                                     reinterpret_cast<const double2*>(d_gains),
                                                     reinterpret_cast<double2*>(d_grad_W),
                                                     reinterpret_cast<double2*>(d_grad_g));
    e = cudaGetLastError();
  }
  if (part) cudaFreeAsync(part, s);
  if (sc.base) cudaFreeAsync(sc.base, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? BIPP_OK : (e == cudaErrorMemoryAllocation ? BIPP_ERR_OUT_OF_MEMORY : BIPP_ERR_CUDA);
}
