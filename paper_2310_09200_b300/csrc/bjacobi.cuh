// bjacobi.cuh — FP32 block Jacobi for batched Hermitian matrices (the
// preconditioning stage of the mixed-precision eigensolver).
//
// The n indices are split into contiguous blocks of 32; a block round pairs
// the blocks by the round-robin ("circle") schedule, and for each block pair
// P = I u J (<= 64 indices) one CTA
//   1. loads the 64 x 64 pivot block S = C[P, P] into shared memory and
//      diagonalises it with a parallel-order scalar Jacobi (the same rotation
//      as the scalar kernel), accumulating the 64 x 64 unitary U;
//   2. applies U to the whole matrix: R = U^H C[P, :] column chunk by chunk
//      (rows P get R, columns P get R^H; the pivot block gets U^H S U, the
//      inner result), and Q[:, P] <- Q[:, P] U row chunk by row chunk.
// Every global access touches contiguous 32-index runs, unlike the scalar
// round-robin sweep whose 2x2 blocks are scattered across the matrix, and a
// block sweep (nb - 1 block rounds) replaces n - 1 scalar rounds.
#pragma once

#include "jacobi.cuh"

namespace bipp {

constexpr int kBJ = 32;          // block size
constexpr int kBJ2 = 2 * kBJ;    // pivot block size
constexpr int kBJThreads = 512;
constexpr int kBJLd = kBJ2 + 1;  // shared-memory leading dimension (bank spread)

struct BJacobiArgs {
  float2* C;          // [T] n x n (ld, stride), overwritten
  float2* Q;          // [T] rotations (ld, stride)
  double* mu;         // [T][ld] final diagonal
  const int* status;  // [T] skip problems with a status bit
  int* sweeps;        // [T] block sweeps used
  const int* n;
  int ld;
  size_t stride;
};

namespace bj {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) { return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x)); }

// Global index of local pivot index l (0..63) for blocks (bi, bj); -1 if beyond n.
__device__ __forceinline__ int gidx(int l, int bi, int bj, int n) {
  const int g = (l < kBJ) ? bi * kBJ + l : bj * kBJ + (l - kBJ);
  return g < n ? g : -1;
}

}  // namespace bj

__global__ void __launch_bounds__(kBJThreads, 1) k_bjacobi32(BJacobiArgs a, double tol, int max_sweeps,
                                                             int inner_sweeps) {
  using namespace bj;
  const int t = blockIdx.x;
  if (a.status[t]) return;
  const int n = a.n[t];
  const int N = a.ld;
  float2* C = a.C + (size_t)t * a.stride;
  float2* Q = a.Q + (size_t)t * a.stride;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* S = reinterpret_cast<float2*>(smraw);  // [64][kBJLd] column-major pivot block
  float2* U = S + kBJ2 * kBJLd;                  // [64][kBJLd] accumulated rotations
  float2* T1 = U + kBJ2 * kBJLd;                 // [64][kBJLd] chunk buffer
  __shared__ int sp[kBJ], sq[kBJ];
  __shared__ float sc[kBJ];
  __shared__ float2 ssig[kBJ];
  __shared__ float sdp[kBJ], sdq[kBJ];
  __shared__ double red[kBJThreads / 32];
  __shared__ double s_fro, s_off;
  const int tid = threadIdx.x;

  auto block_sum = [&](double v) -> double {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (tid < 32) {
      s = (tid < kBJThreads / 32) ? red[tid] : 0.0;
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    __syncthreads();
    return s;
  };

  // Q = I, ||C||_F
  double fro = 0.0;
  for (int e = tid; e < n * n; e += kBJThreads) {
    const int i = e % n, j = e / n;
    Q[(size_t)i + (size_t)j * N] = make_float2(i == j ? 1.f : 0.f, 0.f);
    const float2 v = C[(size_t)i + (size_t)j * N];
    fro += (double)v.x * v.x + (double)v.y * v.y;
  }
  fro = block_sum(fro);
  if (tid == 0) s_fro = sqrt(fro);
  __syncthreads();
  const double thresh = tol * s_fro;

  const int nb0 = (n + kBJ - 1) / kBJ;
  const int nb = nb0 + (nb0 & 1);  // phantom block when odd
  int sweep = 0;
  for (;;) {
    double off = 0.0;
    for (int e = tid; e < n * n; e += kBJThreads) {
      const int i = e % n, j = e / n;
      if (i != j) {
        const float2 v = C[(size_t)i + (size_t)j * N];
        off += (double)v.x * v.x + (double)v.y * v.y;
      }
    }
    off = block_sum(off);
    if (tid == 0) s_off = sqrt(off);
    __syncthreads();
    if (s_off <= thresh || s_fro == 0.0 || sweep >= max_sweeps || nb0 < 1) break;
    ++sweep;
    for (int r = 0; r < nb - 1; ++r) {
      for (int k = 0; k < nb / 2; ++k) {
        int bi, bjj;
        jac::rr_pair(r, k, nb, &bi, &bjj);
        if (bi >= nb0 && bjj >= nb0) continue;
        // ---- 1. pivot block into shared memory (invalid indices: identity rows)
        for (int e = tid; e < kBJ2 * kBJ2; e += kBJThreads) {
          const int li = e % kBJ2, lj = e / kBJ2;
          const int gi = gidx(li, bi, bjj, n), gj = gidx(lj, bi, bjj, n);
          float2 v = make_float2(0.f, 0.f);
          if (gi >= 0 && gj >= 0) v = C[(size_t)gi + (size_t)gj * N];
          S[li + lj * kBJLd] = v;
          U[li + lj * kBJLd] = make_float2(li == lj ? 1.f : 0.f, 0.f);
        }
        __syncthreads();
        // ---- inner parallel-order Jacobi on the 64 x 64 block (phantom rows stay zero)
        for (int is = 0; is < inner_sweeps; ++is) {
          for (int rr = 0; rr < kBJ2 - 1; ++rr) {
            if (tid < kBJ) {
              int p, q;
              jac::rr_pair(rr, tid, kBJ2, &p, &q);
              sp[tid] = p;
              sq[tid] = q;
              float c = 1.f, dp = S[p + p * kBJLd].x, dq = S[q + q * kBJLd].x;
              float2 sig = make_float2(0.f, 0.f);
              const float2 x = S[p + q * kBJLd];
              const float rx = hypotf(x.x, x.y);
              if (rx > 0.f) {
                const float tau = (dq - dp) / (2.f * rx);
                const float tt = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + hypotf(1.f, tau));
                c = 1.f / sqrtf(1.f + tt * tt);
                const float s = tt * c;
                sig = make_float2(s * x.x / rx, s * x.y / rx);
                const float a0 = dp, b0 = dq;
                dp = a0 - tt * rx;
                dq = b0 + tt * rx;
              }
              sc[tid] = c;
              ssig[tid] = sig;
              sdp[tid] = dp;
              sdq[tid] = dq;
            }
            __syncthreads();
            // 2x2 blocks (k1 <= k2) of S, mirrored below the diagonal. A plain
            // 32 x 32 item grid (half of it idle): a triangular decode with a
            // data-dependent loop here produced wrong rotations at ptxas -O3.
            for (int e = tid; e < kBJ * kBJ; e += kBJThreads) {
              const int k1 = e / kBJ, k2 = e % kBJ;
              if (k2 < k1) continue;
              const int p1 = sp[k1], q1 = sq[k1], p2 = sp[k2], q2 = sq[k2];
              if (k1 == k2) {
                S[p1 + p1 * kBJLd] = make_float2(sdp[k1], 0.f);
                S[q1 + q1 * kBJLd] = make_float2(sdq[k1], 0.f);
                S[p1 + q1 * kBJLd] = make_float2(0.f, 0.f);
                S[q1 + p1 * kBJLd] = make_float2(0.f, 0.f);
                continue;
              }
              const float c1 = sc[k1], c2 = sc[k2];
              const float2 g1 = ssig[k1], g2 = ssig[k2];
              const float2 x11 = S[p1 + p2 * kBJLd], x12 = S[p1 + q2 * kBJLd];
              const float2 x21 = S[q1 + p2 * kBJLd], x22 = S[q1 + q2 * kBJLd];
              const float2 g2c = make_float2(g2.x, -g2.y);
              const float2 t12 = cmul(x12, g2c), t22 = cmul(x22, g2c);
              const float2 y11 = make_float2(c2 * x11.x - t12.x, c2 * x11.y - t12.y);
              const float2 u11 = cmul(x11, g2);
              const float2 y12 = make_float2(u11.x + c2 * x12.x, u11.y + c2 * x12.y);
              const float2 y21 = make_float2(c2 * x21.x - t22.x, c2 * x21.y - t22.y);
              const float2 u21 = cmul(x21, g2);
              const float2 y22 = make_float2(u21.x + c2 * x22.x, u21.y + c2 * x22.y);
              const float2 m21 = cmul(g1, y21), m22 = cmul(g1, y22);
              const float2 z11 = make_float2(c1 * y11.x - m21.x, c1 * y11.y - m21.y);
              const float2 z12 = make_float2(c1 * y12.x - m22.x, c1 * y12.y - m22.y);
              const float2 g1c = make_float2(g1.x, -g1.y);
              const float2 n11 = cmul(g1c, y11), n12 = cmul(g1c, y12);
              const float2 z21 = make_float2(n11.x + c1 * y21.x, n11.y + c1 * y21.y);
              const float2 z22 = make_float2(n12.x + c1 * y22.x, n12.y + c1 * y22.y);
              S[p1 + p2 * kBJLd] = z11;
              S[p2 + p1 * kBJLd] = make_float2(z11.x, -z11.y);
              S[p1 + q2 * kBJLd] = z12;
              S[q2 + p1 * kBJLd] = make_float2(z12.x, -z12.y);
              S[q1 + p2 * kBJLd] = z21;
              S[p2 + q1 * kBJLd] = make_float2(z21.x, -z21.y);
              S[q1 + q2 * kBJLd] = z22;
              S[q2 + q1 * kBJLd] = make_float2(z22.x, -z22.y);
            }
            // U <- U J
            for (int e = tid; e < kBJ2 * kBJ; e += kBJThreads) {
              const int i = e % kBJ2, k = e / kBJ2;
              const int p = sp[k], q = sq[k];
              const float c = sc[k];
              const float2 g = ssig[k];
              const float2 up = U[i + p * kBJLd], uq = U[i + q * kBJLd];
              const float2 gc = make_float2(g.x, -g.y);
              const float2 t1 = cmul(uq, gc), t2 = cmul(up, g);
              U[i + p * kBJLd] = make_float2(c * up.x - t1.x, c * up.y - t1.y);
              U[i + q * kBJLd] = make_float2(t2.x + c * uq.x, t2.y + c * uq.y);
            }
            __syncthreads();
          }
        }
        // ---- 2a. rows/columns P of C: R = U^H C[P, chunk] for 64-column chunks
        for (int j0 = 0; j0 < n; j0 += kBJ2) {
          for (int e = tid; e < kBJ2 * kBJ2; e += kBJThreads) {
            const int li = e % kBJ2, lj = e / kBJ2;
            const int gi = gidx(li, bi, bjj, n), gj = j0 + lj;
            T1[li + lj * kBJLd] = (gi >= 0 && gj < n) ? C[(size_t)gi + (size_t)gj * N] : make_float2(0.f, 0.f);
          }
          __syncthreads();
          // each thread: 8 outputs (row li, columns lj..)
          float2 acc[8];
          const int li = tid % kBJ2, lg = tid / kBJ2;  // lg 0..7
#pragma unroll
          for (int u = 0; u < 8; ++u) acc[u] = make_float2(0.f, 0.f);
          for (int k = 0; k < kBJ2; ++k) {
            const float2 uh = U[k + li * kBJLd];  // conj(U[k, li])
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const float2 x = T1[k + (lg + 8 * u) * kBJLd];
              // conj(uh) * x
              acc[u].x = fmaf(uh.x, x.x, fmaf(uh.y, x.y, acc[u].x));
              acc[u].y = fmaf(uh.x, x.y, fmaf(-uh.y, x.x, acc[u].y));
            }
          }
          __syncthreads();
          const int gi = gidx(li, bi, bjj, n);
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int gj = j0 + lg + 8 * u;
            if (gi < 0 || gj >= n) continue;
            const bool in_p = (gj / kBJ == bi) || (gj / kBJ == bjj);
            if (in_p) continue;  // the pivot block is written from S below
            C[(size_t)gi + (size_t)gj * N] = acc[u];
            C[(size_t)gj + (size_t)gi * N] = make_float2(acc[u].x, -acc[u].y);
          }
          __syncthreads();
        }
        // pivot block = diagonalised S
        for (int e = tid; e < kBJ2 * kBJ2; e += kBJThreads) {
          const int li = e % kBJ2, lj = e / kBJ2;
          const int gi = gidx(li, bi, bjj, n), gj = gidx(lj, bi, bjj, n);
          if (gi >= 0 && gj >= 0) C[(size_t)gi + (size_t)gj * N] = S[li + lj * kBJLd];
        }
        // ---- 2b. Q[:, P] <- Q[:, P] U for 64-row chunks
        for (int i0 = 0; i0 < n; i0 += kBJ2) {
          for (int e = tid; e < kBJ2 * kBJ2; e += kBJThreads) {
            const int ri = e % kBJ2, lj = e / kBJ2;
            const int gi = i0 + ri, gj = gidx(lj, bi, bjj, n);
            T1[ri + lj * kBJLd] = (gi < n && gj >= 0) ? Q[(size_t)gi + (size_t)gj * N] : make_float2(0.f, 0.f);
          }
          __syncthreads();
          float2 acc[8];
          const int ri = tid % kBJ2, lg = tid / kBJ2;
#pragma unroll
          for (int u = 0; u < 8; ++u) acc[u] = make_float2(0.f, 0.f);
          for (int k = 0; k < kBJ2; ++k) {
            const float2 x = T1[ri + k * kBJLd];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const float2 uu = U[k + (lg + 8 * u) * kBJLd];
              acc[u].x = fmaf(x.x, uu.x, fmaf(-x.y, uu.y, acc[u].x));
              acc[u].y = fmaf(x.x, uu.y, fmaf(x.y, uu.x, acc[u].y));
            }
          }
          __syncthreads();
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int gi = i0 + ri, gj = gidx(lg + 8 * u, bi, bjj, n);
            if (gi < n && gj >= 0) Q[(size_t)gi + (size_t)gj * N] = acc[u];
          }
          __syncthreads();
        }
      }
    }
  }
  for (int i = tid; i < n; i += kBJThreads) a.mu[(size_t)t * N + i] = (double)C[(size_t)i + (size_t)i * N].x;
  if (tid == 0) a.sweeps[t] = sweep;
}

inline size_t bjacobi_smem() { return sizeof(float2) * 3 * kBJ2 * kBJLd; }

}  // namespace bipp
