// tridiag32.cuh — FP32 Householder reduction of a Hermitian matrix to real
// tridiagonal form (the first stage of the mixed-precision eigensolver).
//
// For each problem (one CTA per problem; n x n Hermitian C, column-major):
// T = H^H C H, H = H_0 H_1 ... H_{n-2}, H_k = I - tau_k v_k v_k^H acting on
// indices k+1..n-1 with v_k[k+1] = 1 and beta_k = (H_k^H C[k+1:, k])[0] real,
// so that T is real symmetric tridiagonal (diagonal d, off-diagonal e = beta).
// The rank-2 update of step k is fused with the matrix-vector product of step
// k+1: the trailing matrix is read and written once per step. The reflectors
// v_k[k+2:] overwrite C below its subdiagonal; d, e and tau go to the scratch.
// The leading eigenpairs of T and their back-transformation are in
// tridiag_sel.cuh.
#pragma once

#include <math.h>

#include "bipp_internal.cuh"

namespace bipp {

constexpr int kTdThreads = 512;

struct TridiagArgs {
  float2* C;          // [T] n x n Hermitian (ld, stride): overwritten by the reflectors v_k[k+2:]
  float* scratch;     // [T] per problem: Z (ld x ld floats, the eigenvectors of T), d, e (ld floats each), tau (ld float2)
  size_t sstride;     // floats between the scratch regions of consecutive problems
  int* status;        // [T] problems with a status bit are skipped
  const int* n;       // [T]
  int ld;
  size_t stride;      // float2 elements between consecutive problems of C
  const int* order = nullptr;  // [T] problem of each block (Batch::order), or nullptr
};

// Per-problem scratch layout (in floats): Z at 0, d at ld^2, e at ld^2 + ld,
// tau (float2, 8-byte aligned) after them.
__host__ __device__ __forceinline__ size_t td_off_d(int ld) { return (size_t)ld * ld; }
__host__ __device__ __forceinline__ size_t td_off_e(int ld) { return (size_t)ld * ld + ld; }
__host__ __device__ __forceinline__ size_t td_off_tau(int ld) { return ((size_t)ld * ld + 2 * (size_t)ld + 1) & ~(size_t)1; }
__host__ __device__ __forceinline__ size_t td_scratch_floats(int ld) { return td_off_tau(ld) + 2 * (size_t)ld; }

namespace td {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}

// Sum over the block of kTdThreads threads (all threads get the result).
template <typename V>
__device__ __forceinline__ float2 block_sum2(float2 v, V* red) {
  const int tid = threadIdx.x;
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  float2 s = make_float2(0.f, 0.f);
#pragma unroll
  for (int w = 0; w < kTdThreads / 32; ++w) {
    s.x += red[w].x;
    s.y += red[w].y;
  }
  __syncthreads();
  return s;
}

}  // namespace td

// ---- 1. Householder reduction to real tridiagonal form
// Dynamic shared memory: 5 * ld float2 (v_prev, w_prev, v, w, p).
__global__ void __launch_bounds__(kTdThreads, 1) k_tridiag32(TridiagArgs a) {
  using namespace td;
  const int t = prob_of(a.order, blockIdx.x);
  if (a.status[t]) return;
  const int n = a.n[t], N = a.ld, tid = threadIdx.x;
  float2* A = a.C + (size_t)t * a.stride;
  float* S = a.scratch + (size_t)t * a.sstride;
  float* d = S + td_off_d(N);
  float* e = S + td_off_e(N);
  float2* tau = reinterpret_cast<float2*>(S + td_off_tau(N));
  extern __shared__ __align__(16) unsigned char tdsm[];
  float2* vp = reinterpret_cast<float2*>(tdsm);  // v_{k-1} (global row index)
  float2* wp = vp + N;                            // w_{k-1}
  float2* v = wp + N;                             // v_k
  float2* w = v + N;                              // w_k
  float2* p = w + N;                              // p_k = A v_k
  __shared__ float2 red[kTdThreads / 32];
  __shared__ float2 s_tau, s_scale;
  __shared__ float s_beta;
  __shared__ int s_trivial;
  for (int i = tid; i < N; i += kTdThreads) {
    vp[i] = make_float2(0.f, 0.f);
    wp[i] = make_float2(0.f, 0.f);
  }
  if (n == 1 && tid == 0) d[0] = A[0].x;
  __syncthreads();
  for (int k = 0; k + 1 < n; ++k) {
    const int m = n - k - 1;  // rows k+1..n-1
    // (a) reflector from column k (already up to date)
    float2 sg = make_float2(0.f, 0.f);
    for (int r = tid; r < m; r += kTdThreads) {
      const float2 x = A[(size_t)(k + 1 + r) + (size_t)k * N];
      if (r > 0) sg.x += x.x * x.x + x.y * x.y;
    }
    const float sigma = block_sum2(sg, red).x;
    if (tid == 0) {
      const float2 al = A[(size_t)(k + 1) + (size_t)k * N];
      d[k] = A[(size_t)k + (size_t)k * N].x;
      if (sigma == 0.f && al.y == 0.f) {
        s_trivial = 1;
        s_tau = make_float2(0.f, 0.f);
        s_beta = al.x;
        s_scale = make_float2(0.f, 0.f);
      } else {
        const float beta = -copysignf(sqrtf(al.x * al.x + al.y * al.y + sigma), al.x);
        s_trivial = 0;
        s_tau = make_float2((beta - al.x) / beta, -al.y / beta);
        s_beta = beta;
        const float2 dn = make_float2(al.x - beta, al.y);  // 1 / (alpha - beta)
        const float inv = 1.f / (dn.x * dn.x + dn.y * dn.y);
        s_scale = make_float2(dn.x * inv, -dn.y * inv);
      }
      e[k] = s_beta;
      tau[k] = s_tau;
    }
    __syncthreads();
    const float2 tk = s_tau, sc = s_scale;
    const bool triv = s_trivial != 0;
    for (int r = tid; r < m; r += kTdThreads) {
      float2 vv;
      if (r == 0) {
        vv = make_float2(1.f, 0.f);
      } else if (triv) {
        vv = make_float2(0.f, 0.f);
      } else {
        vv = cmul(A[(size_t)(k + 1 + r) + (size_t)k * N], sc);
        A[(size_t)(k + 1 + r) + (size_t)k * N] = vv;  // reflector storage
      }
      v[k + 1 + r] = vv;
    }
    __syncthreads();
    // (b) fused pass over A[k+1:, k+1:]: pending rank-2 update of step k-1, then p = A v_k
    for (int r = tid; r < m; r += kTdThreads) {
      const int i = k + 1 + r;
      const float2 vpi = vp[i], wpi = wp[i];
      float2 acc = make_float2(0.f, 0.f);
      float2* Ai = A + i;
      // 8 columns per group, the next group's loads issued before this group is stored
      constexpr int G = 8;
      int j = k + 1;
      float2 cur[G], nxt[G];
      if (j + G <= n) {
#pragma unroll
        for (int u = 0; u < G; ++u) cur[u] = Ai[(size_t)(j + u) * N];
      }
      for (; j + G <= n; j += G) {
        const bool more = j + 2 * G <= n;
        if (more) {
#pragma unroll
          for (int u = 0; u < G; ++u) nxt[u] = Ai[(size_t)(j + G + u) * N];
        }
#pragma unroll
        for (int u = 0; u < G; ++u) {
          // a -= w_i conj(v_j) + v_i conj(w_j)
          float2 x = cur[u];
          const float2 t1 = cmulc(wpi, vp[j + u]), t2 = cmulc(vpi, wp[j + u]);
          x.x -= t1.x + t2.x;
          x.y -= t1.y + t2.y;
          Ai[(size_t)(j + u) * N] = x;
          const float2 pv = cmul(x, v[j + u]);
          acc.x += pv.x;
          acc.y += pv.y;
        }
        if (more) {
#pragma unroll
          for (int u = 0; u < G; ++u) cur[u] = nxt[u];
        }
      }
      for (; j < n; ++j) {
        float2 x = Ai[(size_t)j * N];
        const float2 t1 = cmulc(wpi, vp[j]), t2 = cmulc(vpi, wp[j]);
        x.x -= t1.x + t2.x;
        x.y -= t1.y + t2.y;
        Ai[(size_t)j * N] = x;
        const float2 pv = cmul(x, v[j]);
        acc.x += pv.x;
        acc.y += pv.y;
      }
      p[i] = acc;
    }
    __syncthreads();
    // (c) gamma = v^H p (real), w = tau p - |tau|^2 gamma / 2 v
    float2 gp = make_float2(0.f, 0.f);
    for (int r = tid; r < m; r += kTdThreads) {
      const int i = k + 1 + r;
      const float2 vi = v[i], pi = p[i];
      gp.x += vi.x * pi.x + vi.y * pi.y;
    }
    const float gamma = block_sum2(gp, red).x;
    const float hg = 0.5f * (tk.x * tk.x + tk.y * tk.y) * gamma;
    for (int r = tid; r < m; r += kTdThreads) {
      const int i = k + 1 + r;
      const float2 tp = cmul(tk, p[i]), vi = v[i];
      w[i] = make_float2(tp.x - hg * vi.x, tp.y - hg * vi.y);
    }
    __syncthreads();
    // (d) column k+1 gets the update of step k now (v_k[k+1] = 1); the rest is pending
    const float2 wk1 = w[k + 1];
    for (int r = tid; r < m; r += kTdThreads) {
      const int i = k + 1 + r;
      float2 x = A[(size_t)i + (size_t)(k + 1) * N];
      const float2 t2 = cmulc(v[i], wk1);
      x.x -= w[i].x + t2.x;
      x.y -= w[i].y + t2.y;
      A[(size_t)i + (size_t)(k + 1) * N] = x;
      vp[i] = v[i];
      wp[i] = w[i];
    }
    if (tid == 0) vp[k] = wp[k] = make_float2(0.f, 0.f);
    __syncthreads();
    if (k + 2 == n && tid == 0) d[n - 1] = A[(size_t)(n - 1) + (size_t)(n - 1) * N].x;
  }
}

// ---- 1'. the same reduction on the lower triangle only (ld <= 512): the
// fused pass runs over 32 x 32 tiles of the trailing lower triangle, one warp
// per tile with lane = row and 16 of the tile's columns at a time in registers
// (16 loads in flight per lane); an element a_ij (i >= j) contributes a_ij v_j to p_i and,
// off the diagonal, conj(a_ij) v_i to p_j. Each tile writes its row sums and
// its column sums into fixed slots (rowp[tile column][i], colp[tile row][j]),
// summed in a fixed order afterwards, so the result is deterministic.
// Dynamic shared memory: 5 * ld + 2 * 16 * ld float2.
constexpr int kTdLoMax = 512;

__global__ void __launch_bounds__(kTdThreads, 1) k_tridiag32_lo(TridiagArgs a) {
  using namespace td;
  const int t = prob_of(a.order, blockIdx.x);
  if (a.status[t]) return;
  const int n = a.n[t], N = a.ld, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  float2* A = a.C + (size_t)t * a.stride;
  float* S = a.scratch + (size_t)t * a.sstride;
  float* d = S + td_off_d(N);
  float* e = S + td_off_e(N);
  float2* tau = reinterpret_cast<float2*>(S + td_off_tau(N));
  extern __shared__ __align__(16) unsigned char tdlsm[];
  float2* vp = reinterpret_cast<float2*>(tdlsm);
  float2* wp = vp + N;
  float2* v = wp + N;
  float2* w = v + N;
  float2* p = w + N;
  float2* rowp = p + N;                       // [16][N]
  float2* colp = rowp + (size_t)(kTdLoMax / 32) * N;  // [16][N]
  __shared__ float2 red[kTdThreads / 32];
  __shared__ float2 s_tau, s_scale;
  __shared__ float s_beta;
  __shared__ int s_trivial;
  for (int i = tid; i < N; i += kTdThreads) {
    vp[i] = make_float2(0.f, 0.f);
    wp[i] = make_float2(0.f, 0.f);
  }
  if (n == 1 && tid == 0) d[0] = A[0].x;
  __syncthreads();
  for (int k = 0; k + 1 < n; ++k) {
    const int m = n - k - 1;
    // (a) reflector from column k
    float2 sg = make_float2(0.f, 0.f);
    for (int r = tid; r < m; r += kTdThreads) {
      const float2 x = A[(size_t)(k + 1 + r) + (size_t)k * N];
      if (r > 0) sg.x += x.x * x.x + x.y * x.y;
    }
    const float sigma = block_sum2(sg, red).x;
    if (tid == 0) {
      const float2 al = A[(size_t)(k + 1) + (size_t)k * N];
      d[k] = A[(size_t)k + (size_t)k * N].x;
      if (sigma == 0.f && al.y == 0.f) {
        s_trivial = 1;
        s_tau = make_float2(0.f, 0.f);
        s_beta = al.x;
        s_scale = make_float2(0.f, 0.f);
      } else {
        const float beta = -copysignf(sqrtf(al.x * al.x + al.y * al.y + sigma), al.x);
        s_trivial = 0;
        s_tau = make_float2((beta - al.x) / beta, -al.y / beta);
        s_beta = beta;
        const float2 dn = make_float2(al.x - beta, al.y);
        const float inv = 1.f / (dn.x * dn.x + dn.y * dn.y);
        s_scale = make_float2(dn.x * inv, -dn.y * inv);
      }
      e[k] = s_beta;
      tau[k] = s_tau;
    }
    __syncthreads();
    const float2 tk = s_tau, sc = s_scale;
    const bool triv = s_trivial != 0;
    const int nt = (m + 31) / 32;  // tile rows = tile columns of the trailing block
    for (int r = tid; r < m; r += kTdThreads) {
      float2 vv;
      if (r == 0) {
        vv = make_float2(1.f, 0.f);
      } else if (triv) {
        vv = make_float2(0.f, 0.f);
      } else {
        vv = cmul(A[(size_t)(k + 1 + r) + (size_t)k * N], sc);
        A[(size_t)(k + 1 + r) + (size_t)k * N] = vv;
      }
      v[k + 1 + r] = vv;
    }
    for (int e0 = tid; e0 < nt * N; e0 += kTdThreads) {
      rowp[e0] = make_float2(0.f, 0.f);
      colp[e0] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    // (b) tiles (ti >= tj) of the lower triangle of A[k+1:, k+1:]
    {
      int tile = 0;
      for (int ti = 0; ti < nt; ++ti) {
        for (int tj = 0; tj <= ti; ++tj, ++tile) {
          if (tile % (kTdThreads / 32) != wid) continue;
          const int i = k + 1 + ti * 32 + lane, j0 = k + 1 + tj * 32;
          const bool rv = i < n;
          const float2 zero = make_float2(0.f, 0.f);
          const float2 vpi = rv ? vp[i] : zero, wpi = rv ? wp[i] : zero, vi = rv ? v[i] : zero;
          float2* Ai = A + (rv ? i : k + 1);
          float2 acc = zero;
#pragma unroll
          for (int h = 0; h < 2; ++h) {  // two halves of 16 columns
            float2 x[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
              const int j = j0 + 16 * h + u;
              x[u] = (rv && j <= i) ? Ai[(size_t)j * N] : zero;
            }
            float2 cv[16];  // this row's contributions conj(a_ij) v_i to the 16 column sums
#pragma unroll
            for (int u = 0; u < 16; ++u) {
              const int j = j0 + 16 * h + u;
              const bool ok = rv && j <= i;
              cv[u] = zero;
              if (ok) {
                const float2 t1 = cmulc(wpi, vp[j]), t2 = cmulc(vpi, wp[j]);
                x[u].x -= t1.x + t2.x;
                x[u].y -= t1.y + t2.y;
                Ai[(size_t)j * N] = x[u];
                const float2 pv = cmul(x[u], v[j]);
                acc.x += pv.x;
                acc.y += pv.y;
                if (j < i) cv[u] = cmulc(vi, x[u]);
              }
            }
            // column sums over the 32 rows by a reduce-scatter butterfly: at each level a
            // lane keeps half of its partial sums and adds its partner's other half, so
            // the 16 sums take 16 shuffles per component instead of 80; lane l ends with
            // the sum of column 8 b4 + 4 b3 + 2 b2 + b1 (bits of l), as does lane l ^ 1
#pragma unroll
            for (int lv = 0; lv < 4; ++lv) {
              const int half = 8 >> lv, bit = 16 >> lv;
              const bool up = (lane & bit) != 0;
#pragma unroll
              for (int k = 0; k < half; ++k) {
                const float2 send = up ? cv[k] : cv[k + half];
                const float2 keep = up ? cv[k + half] : cv[k];
                cv[k].x = keep.x + __shfl_xor_sync(0xffffffffu, send.x, bit);
                cv[k].y = keep.y + __shfl_xor_sync(0xffffffffu, send.y, bit);
              }
            }
            cv[0].x += __shfl_xor_sync(0xffffffffu, cv[0].x, 1);
            cv[0].y += __shfl_xor_sync(0xffffffffu, cv[0].y, 1);
            {
              const int cu = 8 * ((lane >> 4) & 1) + 4 * ((lane >> 3) & 1) + 2 * ((lane >> 2) & 1) + ((lane >> 1) & 1);
              const int j = j0 + 16 * h + cu;
              if ((lane & 1) == 0 && j < n) colp[(size_t)ti * N + j] = cv[0];
            }
          }
          if (rv) rowp[(size_t)tj * N + i] = acc;
        }
      }
    }
    __syncthreads();
    for (int r = tid; r < m; r += kTdThreads) {
      const int i = k + 1 + r;
      float2 sum = make_float2(0.f, 0.f);
      for (int q = 0; q < nt; ++q) {
        sum.x += rowp[(size_t)q * N + i].x + colp[(size_t)q * N + i].x;
        sum.y += rowp[(size_t)q * N + i].y + colp[(size_t)q * N + i].y;
      }
      p[i] = sum;
    }
    __syncthreads();
    // (c) gamma = v^H p, w = tau p - |tau|^2 gamma / 2 v
    float2 gp = make_float2(0.f, 0.f);
    for (int r = tid; r < m; r += kTdThreads) {
      const int i = k + 1 + r;
      const float2 vi = v[i], pi = p[i];
      gp.x += vi.x * pi.x + vi.y * pi.y;
    }
    const float gamma = block_sum2(gp, red).x;
    const float hg = 0.5f * (tk.x * tk.x + tk.y * tk.y) * gamma;
    for (int r = tid; r < m; r += kTdThreads) {
      const int i = k + 1 + r;
      const float2 tp = cmul(tk, p[i]), vi = v[i];
      w[i] = make_float2(tp.x - hg * vi.x, tp.y - hg * vi.y);
    }
    __syncthreads();
    // (d) column k+1 (rows k+1..n-1) gets the update of step k now
    const float2 wk1 = w[k + 1];
    for (int r = tid; r < m; r += kTdThreads) {
      const int i = k + 1 + r;
      float2 x = A[(size_t)i + (size_t)(k + 1) * N];
      const float2 t2 = cmulc(v[i], wk1);
      x.x -= w[i].x + t2.x;
      x.y -= w[i].y + t2.y;
      A[(size_t)i + (size_t)(k + 1) * N] = x;
      vp[i] = v[i];
      wp[i] = w[i];
    }
    if (tid == 0) vp[k] = wp[k] = make_float2(0.f, 0.f);
    __syncthreads();
    if (k + 2 == n && tid == 0) d[n - 1] = A[(size_t)(n - 1) + (size_t)(n - 1) * N].x;
  }
}

// Householder reduction only (1 launch): reflectors, d, e and tau.
inline void launch_tridiag32_reduce(const TridiagArgs& a, int T, cudaStream_t s) {
  const int N = a.ld;
  if (N <= kTdLoMax) {
    const int smem1l = (5 + 2 * (kTdLoMax / 32)) * N * (int)sizeof(float2);
    cudaFuncSetAttribute(k_tridiag32_lo, cudaFuncAttributeMaxDynamicSharedMemorySize, smem1l);
    k_tridiag32_lo<<<T, kTdThreads, smem1l, s>>>(a);
  } else {
    const int smem1 = 5 * N * (int)sizeof(float2);
    cudaFuncSetAttribute(k_tridiag32, cudaFuncAttributeMaxDynamicSharedMemorySize, smem1);
    k_tridiag32<<<T, kTdThreads, smem1, s>>>(a);
  }
}

}  // namespace bipp
