// tridiag32.cuh — FP32 Hermitian eigendecomposition through a real tridiagonal
// form (the preconditioning stage of the mixed-precision eigensolver).
//
// For each problem (one CTA per problem; n x n Hermitian C, column-major):
//   1. k_tridiag32: Householder reduction T = H^H C H, H = H_0 H_1 ... H_{n-2},
//      H_k = I - tau_k v_k v_k^H acting on indices k+1..n-1 with v_k[k+1] = 1
//      and beta_k = (H_k^H C[k+1:, k])[0] real, so that T is real symmetric
//      tridiagonal (diagonal d, off-diagonal e = beta). The rank-2 update of
//      step k is fused with the matrix-vector product of step k+1: the
//      trailing matrix is read and written once per step.
//   2. k_tridiag_qr32: implicit symmetric QR with the Wilkinson shift on (d, e);
//      one thread chases the bulge and records the Givens rotations of each
//      QR step while the other warps apply those of the previous step to
//      their rows of Z (Z starts as I), so that T = Z diag(d) Z^T at
//      convergence.
//   3. k_tridiag_back32_blk: Q = H Z, applying H_{n-2} first, in blocks of
//      reflectors with each column of Q in a warp's registers (the one-reflector
//      -at-a-time k_tridiag_back32 serves n_max > 1024).
// Result: C ~ Q diag(d) Q^H with Q unitary to FP32 rounding; the eigenvalues
// are left unsorted in mu.
#pragma once

#include <math.h>

#include "bipp_internal.cuh"

namespace bipp {

constexpr int kTdThreads = 512;

struct TridiagArgs {
  float2* C;          // [T] n x n Hermitian (ld, stride): overwritten by the reflectors v_k[k+2:]
  float2* Q;          // [T] eigenvectors (ld, stride)
  float* scratch;     // [T] per problem: Z (ld x ld floats), d, e (ld floats each), tau (ld float2)
  size_t sstride;     // floats between the scratch regions of consecutive problems
  double* mu;         // [T][ld] eigenvalues (unsorted)
  int* status;        // [T] problems with a status bit are skipped; QR failure sets kStatusNotConverged
  int* steps;         // [T] QR steps used
  const int* n;       // [T]
  int ld;
  size_t stride;      // float2 elements between consecutive problems of C and Q
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
  const int t = blockIdx.x;
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
  const int t = blockIdx.x;
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

// ---- 2. implicit symmetric QR on (d, e) with the Wilkinson shift, rotations applied to Z
// One driver thread (lane 0 of warp 0) runs the QR iteration on the
// tridiagonal (scaled to unit Frobenius norm) and records the Givens rotations
// of step s+1 while the applier warps apply those of step s to their rows of Z
// (double-buffered rotation lists, one barrier per step). The driver's chain
// of dependent operations is the critical path, so the warps that share its
// SM sub-partition (warp index = 0 mod 4) stay idle and the appliers are the
// other 18 of 24 warps (one row of Z each up to n = 576).
// Dynamic shared memory: 6 * ld floats (d, e, two (c, s) lists).
constexpr int kQrThreads = 768;
constexpr int kQrApply = kQrThreads / 4 * 3;

__global__ void __launch_bounds__(kQrThreads, 1) k_tridiag_qr32(TridiagArgs a, int max_steps) {
  const int t = blockIdx.x;
  if (a.status[t]) return;
  const int n = a.n[t], N = a.ld, tid = threadIdx.x;
  float* Z = a.scratch + (size_t)t * a.sstride;
  const float* dg = Z + td_off_d(N);
  const float* eg = Z + td_off_e(N);
  extern __shared__ __align__(16) unsigned char qrsm[];
  float* d = reinterpret_cast<float*>(qrsm);
  float* e = d + N;
  float* rc0 = e + N;  // [2][N] cosines
  float* rs0 = rc0 + 2 * N;  // [2][N] sines
  __shared__ int s_p[2], s_q[2], s_state[2];  // state: 0 apply, 1 done, 2 step cap hit
  __shared__ float s_norm;
  for (int i = tid; i < n; i += kQrThreads) {
    d[i] = dg[i];
    e[i] = (i + 1 < n) ? eg[i] : 0.f;
  }
  for (int e0 = tid; e0 < n * n; e0 += kQrThreads) {
    const int r = e0 % n, c = e0 / n;
    Z[(size_t)r + (size_t)c * N] = (r == c) ? 1.f : 0.f;
  }
  __syncthreads();
  const int wid = tid >> 5, lane = tid & 31;
  const bool driver = tid == 0;
  const int ai = (wid & 3) ? (wid - 1 - (wid >> 2)) * 32 + (tid & 31) : -1;  // applier index
  const float eps = 5.96e-8f, tiny = 1e-8f;  // deflation: relative to the neighbours, or to ||T||_F = 1
  int q = n - 1, plo = n, steps = 0, fin = 0;  // driver state (plo >= q: find the block start again)
  auto small = [&](float ev, float d0, float d1) { return ev <= eps * (fabsf(d0) + fabsf(d1)) || ev <= tiny; };
  auto drive = [&](int slot) {
    int state = 1;
    while (q > 0) {
      if (small(fabsf(e[q - 1]), d[q - 1], d[q])) {
        e[q - 1] = 0.f;
        --q;
        continue;
      }
      if (steps >= max_steps) {
        state = 2;
        break;
      }
      if (plo >= q) {  // start of the unreduced block ending at q
        plo = q - 1;
        while (plo > 0 && !small(fabsf(e[plo - 1]), d[plo - 1], d[plo])) --plo;
        if (plo > 0) e[plo - 1] = 0.f;
      }
      const int p = plo;
      // Wilkinson shift from the trailing 2 x 2 block
      const float dl = 0.5f * (d[q - 1] - d[q]), ee = e[q - 1];
      const float den = dl + copysignf(sqrtf(dl * dl + ee * ee), dl);
      const float mu = d[q] - ((den != 0.f) ? ee * ee / den : 0.f);
      // Givens rotation zeroing z against x (scaled T: |x|, |z| <= ~1); rsqrtf's error is
      // biased, and a bias in c^2 + s^2 would build up linearly over the ~n^2 rotations
      // applied to Z, so one Newton-Raphson step on c^2 + s^2 = 1 with the residual
      // formed by FMAs (exact far below an ulp) leaves only unbiased rounding.
      auto givens = [](float x, float z, float& c, float& s, float& r) {
        const float r2 = fmaf(x, x, z * z);
        const float ri = rsqrtf(r2);
        c = x * ri;
        s = z * ri;
        const float hh = 0.5f * fmaf(-c, c, fmaf(-s, s, 1.f));
        c = fmaf(hh, c, c);
        s = fmaf(hh, s, s);
        const bool deg = !(r2 > 0.f);  // x = z = 0: identity (replaces the NaNs of 0 * inf)
        c = deg ? 1.f : c;
        s = deg ? 0.f : s;
        r = fmaf(x, c, z * s);
      };
      float* rc = rc0 + slot * N;
      float* rs = rs0 + slot * N;
      // e[q] = 0 at the bottom of an unreduced block, so the bulge leaves it without a test
      float ak = d[p], bk = e[p];
      float x = ak - mu, z = bk;
      float dk1 = d[p + 1], ek1 = e[p + 1];
      int k = p;
      {  // first rotation: creates the bulge, no off-diagonal to its left
        float c, s, r;
        givens(x, z, c, s, r);
        const float cc = c * c, ss = s * s, cs = c * s;
        d[p] = cc * ak + 2.f * cs * bk + ss * dk1;
        const float ndk1 = ss * ak - 2.f * cs * bk + cc * dk1;
        x = cs * (dk1 - ak) + (cc - ss) * bk;
        z = s * ek1;
        bk = c * ek1;
        ak = ndk1;
        rc[0] = c;
        rs[0] = s;
        ++k;
      }
      float dn = d[k + 1], en = e[k + 1];
      for (; k < q; ++k) {  // chase: rotation k removes the bulge at (k + 1, k - 1)
        dk1 = dn;
        ek1 = en;
        dn = d[k + 2];  // one ahead; past the block the values are read but unused
        en = e[k + 2];
        float c, s, r;
        givens(x, z, c, s, r);
        const float cc = c * c, ss = s * s, cs = c * s;
        d[k] = cc * ak + 2.f * cs * bk + ss * dk1;
        const float ndk1 = ss * ak - 2.f * cs * bk + cc * dk1;
        e[k - 1] = r;
        x = cs * (dk1 - ak) + (cc - ss) * bk;
        z = s * ek1;
        bk = c * ek1;
        ak = ndk1;
        rc[k - p] = c;
        rs[k - p] = s;
      }
      e[q - 1] = x;
      d[q] = ak;
      ++steps;
      s_p[slot] = p;
      s_q[slot] = q;
      state = 0;
      break;
    }
    s_state[slot] = state;
    fin = state;
  };
  // After a QR step the driver warp scans the block's off-diagonals for new
  // negligible ones (a split: the next steps start below the last one).
  auto scan_splits = [&](int slot) {
    __syncwarp();
    if (s_state[slot] != 0) return;
    const int p = s_p[slot], qq = s_q[slot];
    int best = -1;
    for (int k = p + 1 + lane; k < qq; k += 32) {
      if (small(fabsf(e[k - 1]), d[k - 1], d[k])) {
        e[k - 1] = 0.f;
        best = k;
      }
    }
    best = __reduce_max_sync(0xffffffffu, best);
    if (driver && best > plo) plo = best;
    __syncwarp();
  };
  if (driver) {
    float tn2 = 0.f;
    for (int i = 0; i < n; ++i) tn2 += d[i] * d[i] + 2.f * e[i] * e[i];
    const float tn = sqrtf(tn2), sc = tn > 0.f ? 1.f / tn : 1.f;
    for (int i = 0; i < n; ++i) {
      d[i] *= sc;
      e[i] *= sc;
    }
    s_norm = tn > 0.f ? tn : 1.f;
    drive(0);
  }
  if (wid == 0) scan_splits(0);
  __syncthreads();
  for (int it = 0;; ++it) {
    const int cur = it & 1;
    if (s_state[cur] != 0) break;
    if (wid == 0) {
      if (driver) drive(cur ^ 1);
      scan_splits(cur ^ 1);
    } else if (ai >= 0) {
      const int p = s_p[cur], qq = s_q[cur];
      const float* rc = rc0 + cur * N;
      const float* rs = rs0 + cur * N;
      const size_t sN = (size_t)N;
      for (int r = ai; r < n; r += kQrApply) {
        float* wr = Z + r + (size_t)p * N;  // column k of row r
        const float* rd = wr + sN;         // next column to load
        float zc = *wr;
        // groups of 8 columns; the next group's loads are issued before this group is rotated
        constexpr int G = 8;
        int k = p;
        float cur[G], nxt[G];
        if (k + G <= qq) {
#pragma unroll
          for (int u = 0; u < G; ++u) {
            cur[u] = *rd;
            rd += sN;
          }
        }
        for (; k + G <= qq; k += G) {
          const bool more = k + 2 * G <= qq;
          if (more) {
#pragma unroll
            for (int u = 0; u < G; ++u) {
              nxt[u] = *rd;
              rd += sN;
            }
          }
#pragma unroll
          for (int u = 0; u < G; ++u) {
            const float c = rc[k + u - p], s = rs[k + u - p];
            *wr = fmaf(c, zc, s * cur[u]);
            wr += sN;
            zc = fmaf(c, cur[u], -s * zc);
          }
          if (more) {
#pragma unroll
            for (int u = 0; u < G; ++u) cur[u] = nxt[u];
          }
        }
        for (; k < qq; ++k) {
          const float zn = wr[sN];
          const float c = rc[k - p], s = rs[k - p];
          *wr = fmaf(c, zc, s * zn);
          wr += sN;
          zc = fmaf(c, zn, -s * zc);
        }
        *wr = zc;
      }
    }
    __syncthreads();
  }
  const float tn = s_norm;
  for (int i = tid; i < n; i += kQrThreads) a.mu[(size_t)t * N + i] = (double)(d[i] * tn);
  if (driver) {
    a.steps[t] = steps;
    if (fin == 2) a.status[t] |= kStatusNotConverged;
  }
}

// ---- 3. back-transformation Q = H_0 ... H_{n-2} Z, one warp per column
// Grid (column groups, T); dynamic shared memory: ld float2 (the current v_k).
__global__ void __launch_bounds__(kTdThreads) k_tridiag_back32(TridiagArgs a, int cols_per_cta) {
  using namespace td;
  const int t = blockIdx.y;
  if (a.status[t]) return;
  const int n = a.n[t], N = a.ld, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int c0 = blockIdx.x * cols_per_cta;
  if (c0 >= n) return;
  const int c1 = min(n, c0 + cols_per_cta);
  const float2* A = a.C + (size_t)t * a.stride;
  float2* Q = a.Q + (size_t)t * a.stride;
  const float* Z = a.scratch + (size_t)t * a.sstride;
  const float2* tau = reinterpret_cast<const float2*>(Z + td_off_tau(N));
  extern __shared__ __align__(16) unsigned char bksm[];
  float2* v = reinterpret_cast<float2*>(bksm);
  for (int e0 = tid; e0 < n * (c1 - c0); e0 += kTdThreads) {
    const int r = e0 % n, c = c0 + e0 / n;
    Q[(size_t)r + (size_t)c * N] = make_float2(Z[(size_t)r + (size_t)c * N], 0.f);
  }
  for (int k = n - 2; k >= 0; --k) {
    const int m = n - k - 1;
    __syncthreads();
    for (int r = tid; r < m; r += kTdThreads)
      v[r] = (r == 0) ? make_float2(1.f, 0.f) : A[(size_t)(k + 1 + r) + (size_t)k * N];
    __syncthreads();
    const float2 tk = tau[k];
    if (tk.x == 0.f && tk.y == 0.f) continue;
    for (int c = c0 + wid; c < c1; c += kTdThreads / 32) {
      float2* Qc = Q + (size_t)(k + 1) + (size_t)c * N;
      float2 u = make_float2(0.f, 0.f);  // v^H Q[k+1:, c]
      for (int r = lane; r < m; r += 32) {
        const float2 x = Qc[r], vr = v[r];
        u.x += vr.x * x.x + vr.y * x.y;
        u.y += vr.x * x.y - vr.y * x.x;
      }
      for (int o = 16; o > 0; o >>= 1) {
        u.x += __shfl_xor_sync(0xffffffffu, u.x, o);
        u.y += __shfl_xor_sync(0xffffffffu, u.y, o);
      }
      const float2 tu = cmul(tk, u);
      for (int r = lane; r < m; r += 32) {
        const float2 vr = v[r], y = cmul(vr, tu);
        float2 x = Qc[r];
        x.x -= y.x;
        x.y -= y.y;
        Qc[r] = x;
      }
    }
  }
}

// ---- 3'. the same back-transformation, reflectors applied in blocks of RB
// with each column of Q held in a warp's registers for a whole block (lane l
// holds rows l, l + 32, ...): per block the reflectors' vectors are staged in
// shared memory, every column is read and written once, and the dot product
// of each reflector is a warp reduction. Columns of up to 32 * RPL rows.
// Grid (column groups, T); dynamic shared memory: ld x (RB + 1) float2.
template <int RB, int RPL>
__global__ void __launch_bounds__(kTdThreads) k_tridiag_back32_blk(TridiagArgs a, int cols_per_cta) {
  using namespace td;
  const int t = blockIdx.y;
  if (a.status[t]) return;
  const int n = a.n[t], N = a.ld, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int c0 = blockIdx.x * cols_per_cta;
  if (c0 >= n) return;
  const int c1 = min(n, c0 + cols_per_cta);
  const float2* A = a.C + (size_t)t * a.stride;
  float2* Q = a.Q + (size_t)t * a.stride;
  const float* Z = a.scratch + (size_t)t * a.sstride;
  const float2* tau = reinterpret_cast<const float2*>(Z + td_off_tau(N));
  extern __shared__ __align__(16) unsigned char bbsm[];
  float2* V = reinterpret_cast<float2*>(bbsm);  // [row - (k0 + 1)][j], leading dimension RB + 1
  __shared__ float2 stau[RB];
  for (int e0 = tid; e0 < n * (c1 - c0); e0 += kTdThreads) {
    const int r = e0 % n, c = c0 + e0 / n;
    Q[(size_t)r + (size_t)c * N] = make_float2(Z[(size_t)r + (size_t)c * N], 0.f);
  }
  const int nref = n - 1;  // reflectors 0 .. n-2
  for (int k0 = ((nref - 1) / RB) * RB; k0 >= 0 && nref > 0; k0 -= RB) {
    const int nb = min(RB, nref - k0), mb = n - k0 - 1;  // reflectors k0..k0+nb-1 act on rows k0+1..n-1
    __syncthreads();
    for (int e0 = tid; e0 < mb * nb; e0 += kTdThreads) {
      const int r = e0 % mb, j = e0 / mb;  // v_{k0+j}: 1 at local row j, stored below it
      float2 v = make_float2(0.f, 0.f);
      if (r == j) v = make_float2(1.f, 0.f);
      else if (r > j) v = A[(size_t)(k0 + 1 + r) + (size_t)(k0 + j) * N];
      V[(size_t)r * (RB + 1) + j] = v;
    }
    if (tid < nb) stau[tid] = tau[k0 + tid];
    __syncthreads();
    for (int c = c0 + wid; c < c1; c += kTdThreads / 32) {
      float2* Qc = Q + (size_t)(k0 + 1) + (size_t)c * N;
      float2 q[RPL];
#pragma unroll
      for (int i = 0; i < RPL; ++i) {
        const int r = lane + 32 * i;
        q[i] = (r < mb) ? Qc[r] : make_float2(0.f, 0.f);
      }
      for (int j = nb - 1; j >= 0; --j) {
        const float2 tj = stau[j];
        float2 u = make_float2(0.f, 0.f);  // v^H q
#pragma unroll
        for (int i = 0; i < RPL; ++i) {
          const int r = lane + 32 * i;
          if (r < mb) {
            const float2 vr = V[(size_t)r * (RB + 1) + j];
            u.x += vr.x * q[i].x + vr.y * q[i].y;
            u.y += vr.x * q[i].y - vr.y * q[i].x;
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          u.x += __shfl_xor_sync(0xffffffffu, u.x, o);
          u.y += __shfl_xor_sync(0xffffffffu, u.y, o);
        }
        const float2 tu = cmul(tj, u);
#pragma unroll
        for (int i = 0; i < RPL; ++i) {
          const int r = lane + 32 * i;
          if (r < mb) {
            const float2 y = cmul(V[(size_t)r * (RB + 1) + j], tu);
            q[i].x -= y.x;
            q[i].y -= y.y;
          }
        }
      }
#pragma unroll
      for (int i = 0; i < RPL; ++i) {
        const int r = lane + 32 * i;
        if (r < mb) Qc[r] = q[i];
      }
    }
  }
}

// Launches the three stages on stream s; 3 kernel launches.
inline void launch_tridiag32(const TridiagArgs& a, int T, cudaStream_t s) {
  const int N = a.ld;
  const int smem1 = 5 * N * (int)sizeof(float2), smem2 = 6 * N * (int)sizeof(float), smem3 = N * (int)sizeof(float2);
  cudaFuncSetAttribute(k_tridiag32, cudaFuncAttributeMaxDynamicSharedMemorySize, smem1);
  const int smem1l = (5 + 2 * (kTdLoMax / 32)) * N * (int)sizeof(float2);
  cudaFuncSetAttribute(k_tridiag_qr32, cudaFuncAttributeMaxDynamicSharedMemorySize, smem2);
  cudaFuncSetAttribute(k_tridiag_back32, cudaFuncAttributeMaxDynamicSharedMemorySize, smem3);
  if (N <= kTdLoMax) {
    cudaFuncSetAttribute(k_tridiag32_lo, cudaFuncAttributeMaxDynamicSharedMemorySize, smem1l);
    k_tridiag32_lo<<<T, kTdThreads, smem1l, s>>>(a);
  } else {
    k_tridiag32<<<T, kTdThreads, smem1, s>>>(a);
  }
  k_tridiag_qr32<<<T, kQrThreads, smem2, s>>>(a, 30 * N + 30);
  constexpr int kCols = 64;
  if (N <= 512) {
    const int smb = N * (32 + 1) * (int)sizeof(float2);
    cudaFuncSetAttribute(k_tridiag_back32_blk<32, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb);
    k_tridiag_back32_blk<32, 16><<<dim3((N + kCols - 1) / kCols, T), kTdThreads, smb, s>>>(a, kCols);
  } else if (N <= 1024) {
    const int smb = N * (16 + 1) * (int)sizeof(float2);
    cudaFuncSetAttribute(k_tridiag_back32_blk<16, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb);
    k_tridiag_back32_blk<16, 32><<<dim3((N + kCols - 1) / kCols, T), kTdThreads, smb, s>>>(a, kCols);
  } else {
    k_tridiag_back32<<<dim3((N + kCols - 1) / kCols, T), kTdThreads, smem3, s>>>(a, kCols);
  }
}

}  // namespace bipp
