// eig.cu — FP64 stages 1-3 of standard synthesis, batched over time steps
// (and over channels): Gram matrix (Sec. 2.2, Eq. gram), reduction of the
// generalised problem V a = mu G a to standard form (Sec. 2.3, Eq.
// eigenvaleq), parallel-order complex Jacobi, and selection of the n_eig
// leading eigenpairs with their filter weights and levels (Sec. 2.6,
// Algorithm 1 lines 3-9).
//
// One CTA owns one step's eigenproblem for the sequential factorisations
// (Cholesky, Jacobi); the dense products of the reduction are tiled over the
// whole GPU. Matrices live in global memory (L2-resident at N <= 1024).
#include <math.h>

#include <algorithm>

#include "bipp_internal.cuh"
#include "dfloat.cuh"
#include "jacobi.cuh"

namespace bipp {

namespace {

__device__ __forceinline__ size_t mat_off(int t, int n_max) { return (size_t)t * n_max * n_max; }

// ---------------------------------------------------------------- Gram

// G_ij = sinc(2 ||p_i - p_j|| / wl) with sinc(x) = sin(pi x)/(pi x) (Eq. gram, App. A).
__global__ void k_gram(Batch b, int gram_identity) {
  const int t = prob_of(b.order, blockIdx.z);
  const int n = b.nst[t];
  const double wl = b.wl[t];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= n || j >= n || i > j) return;  // G is symmetric: the upper triangle, mirrored
  double g;
  if (gram_identity) {
    g = (i == j) ? 1.0 : 0.0;
  } else {
    const double* p = b.st + (size_t)t * 3 * b.n_max;
    double dx = p[i] - p[j];
    double dy = p[b.n_max + i] - p[b.n_max + j];
    double dz = p[2 * b.n_max + i] - p[2 * b.n_max + j];
    double x = 2.0 * sqrt(dx * dx + dy * dy + dz * dz) / wl;
    g = (x == 0.0) ? 1.0 : sinpi(x) / (M_PI * x);  // NaN positions propagate to G
  }
  b.G[mat_off(t, b.n_max) + (size_t)i + (size_t)j * b.n_max] = g;
  if (i != j) b.G[mat_off(t, b.n_max) + (size_t)j + (size_t)i * b.n_max] = g;
}

// ---------------------------------------------------------------- Cholesky

// Right-looking Cholesky G = L L^T in place (lower triangle), one CTA per step.
__global__ void k_cholesky(Batch b) {
  const int t = prob_of(b.order, blockIdx.x);
  const int n = b.nst[t];
  const int N = b.n_max;
  double* A = b.G + mat_off(t, N);
  __shared__ int bad;
  __shared__ double inv;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      double s = A[j + (size_t)j * N];
      if (!(s > 0.0)) {
        bad = 1;
      } else {
        double l = sqrt(s);
        A[j + (size_t)j * N] = l;
        inv = 1.0 / l;
      }
    }
    __syncthreads();
    if (bad) break;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[i + (size_t)j * N] *= inv;
    __syncthreads();
    for (int c = j + 1 + warp; c < n; c += nwarp) {
      const double lcj = A[c + (size_t)j * N];
      for (int r = c + lane; r < n; r += 32) A[r + (size_t)c * N] -= A[r + (size_t)j * N] * lcj;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && bad) b.status[t] |= kStatusNotPD;
}

// Blocked right-looking Cholesky G = L L^T in place (lower triangle), one CTA
// per step: for each 32-column panel, factor its diagonal block (one warp),
// solve the rows below against it (one thread per row) and subtract the
// panel's outer product from the trailing lower triangle (one warp per 32 x 32
// tile, K = 32 from shared memory). Global traffic is one read and write of
// the trailing triangle per panel instead of per column.
// Dynamic shared memory: (n_max + 32) x (kChB + 1) doubles: the panel,
// row-major, plus 32 rows that the last partial tile reads and never stores.
constexpr int kChB = 32;
constexpr int kChThreads = 512;
constexpr int kChLd = kChB + 1;

__global__ void __launch_bounds__(kChThreads, 1) k_cholesky_blk(Batch b) {
  const int t = prob_of(b.order, blockIdx.x);
  const int n = b.nst[t];
  const int N = b.n_max;
  double* A = b.G + mat_off(t, N);
  extern __shared__ double sP[];
  __shared__ int bad;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int k0 = 0; k0 < n; k0 += kChB) {
    const int bw = min(kChB, n - k0), m = n - k0;
    for (int e = tid; e < m * bw; e += kChThreads) {
      const int r = e % m, c = e / m;
      sP[r * kChLd + c] = A[(size_t)(k0 + r) + (size_t)(k0 + c) * N];
    }
    __syncthreads();
    if (warp == 0) {  // diagonal block, lane = row
      for (int j = 0; j < bw; ++j) {
        double d = 1.0;
        if (lane == j) {
          const double sjj = sP[j * kChLd + j];
          if (!(sjj > 0.0)) bad = 1;
          d = sqrt(fmax(sjj, 1e-300));
          sP[j * kChLd + j] = d;
        }
        d = __shfl_sync(0xffffffffu, d, j);
        if (lane > j && lane < bw) sP[lane * kChLd + j] /= d;
        __syncwarp();
        if (lane > j && lane < bw) {
          const double lij = sP[lane * kChLd + j];
          for (int c = j + 1; c <= lane; ++c) sP[lane * kChLd + c] -= lij * sP[c * kChLd + j];
        }
        __syncwarp();
      }
    }
    __syncthreads();
    if (bad) break;
    for (int r = bw + tid; r < m; r += kChThreads) {  // x L_dd^T = p, forward substitution
      double* x = sP + r * kChLd;
      for (int j = 0; j < bw; ++j) {
        double sj = x[j];
        for (int k = 0; k < j; ++k) sj -= x[k] * sP[j * kChLd + k];
        x[j] = sj / sP[j * kChLd + j];
      }
    }
    __syncthreads();
    for (int e = tid; e < m * bw; e += kChThreads) {
      const int r = e % m, c = e / m;
      if (r >= c) A[(size_t)(k0 + r) + (size_t)(k0 + c) * N] = sP[r * kChLd + c];
    }
    __syncthreads();
    // the panel's trailing rows become double-float pairs (hi, lo) in place, so the
    // trailing update runs on the FP32 pipe (dfloat.cuh)
    for (int e = tid; e < (m - bw) * bw; e += kChThreads) {
      double* slot = sP + (bw + e / bw) * kChLd + e % bw;
      float hi, lo;
      df::split(*slot, hi, lo);
      *reinterpret_cast<float2*>(slot) = make_float2(hi, lo);
    }
    __syncthreads();
    // trailing lower triangle: A(i, j) -= sum_k P(i, k) P(j, k) for k0 + bw <= j <= i < n
    const int m2 = m - bw, nt = (m2 + 31) / 32;
    const float2* P2 = reinterpret_cast<const float2*>(sP);
    int tile = 0;
    for (int ti = 0; ti < nt; ++ti) {
      for (int tj = 0; tj <= ti; ++tj, ++tile) {
        if (tile % (kChThreads / 32) != warp) continue;
        const int i = ti * 32 + lane;
        if (i >= m2) continue;
        const float2* pi = P2 + (bw + i) * kChLd;
        double* Ai = A + (size_t)(k0 + bw + i);
        for (int h = 0; h < 2; ++h) {  // 16 columns at a time
          float ah[16], al[16];
#pragma unroll
          for (int c = 0; c < 16; ++c) ah[c] = al[c] = 0.f;
          const float2* pj = P2 + (bw + tj * 32 + 16 * h) * kChLd;  // rows past the panel hold stale values, unused
          for (int k = 0; k < bw; ++k) {
            const float2 a = pi[k];
#pragma unroll
            for (int c = 0; c < 16; ++c) {
              const float2 q = pj[c * kChLd + k];
              df::mac(ah[c], al[c], a.x, a.y, q.x, q.y);
            }
            if ((k & 15) == 15) {
#pragma unroll
              for (int c = 0; c < 16; ++c) df::renorm(ah[c], al[c]);
            }
          }
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            const int j = tj * 32 + 16 * h + c;
            if (j <= i && j < m2) Ai[(size_t)(k0 + bw + j) * N] -= df::to_double(ah[c], al[c]);
          }
        }
      }
    }
    __syncthreads();
  }
  if (tid == 0 && bad) b.status[t] |= kStatusNotPD;
}

// L^{-1} column block by column block: one CTA per (32-column block cb, step)
// solves L Y = E[:, cb] by block forward substitution, Y_i = L_ii^{-1}
// (E_i - sum_{cb <= j < i} L_ij Y_j) over 32-row blocks i >= cb (Y_i = 0 for
// i < cb). The products are 32 x 32 x 32 tiles staged in shared memory; the
// diagonal solves run one thread per column. Stored row-major (Linv[i*N + j]).
constexpr int kTiThreads = 256;

__global__ void __launch_bounds__(kTiThreads) k_trinv_blk(Batch b, int gram_identity) {
  const int t = prob_of(b.order, blockIdx.y), cb = blockIdx.x;
  const int n = b.nst[t];
  const int N = b.n_max;
  const int c0 = cb * 32;
  if (c0 >= n || b.status[t]) return;
  const double* L = b.G + mat_off(t, N);
  double* R = b.Linv + mat_off(t, N);
  const int cw = min(32, n - c0);
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;  // 8 rows of 4 outputs per thread
  __shared__ double sL[32][33], sAcc[32][33];
  __shared__ float2 fL[32][33], fY[32][33];  // tiles of the products as double-float pairs (dfloat.cuh)
  // rows above the block are zero
  for (int e = tid; e < c0 * cw; e += kTiThreads) {
    const int i = e / cw, j = e % cw;
    R[(size_t)i * N + c0 + j] = 0.0;
  }
  for (int i0 = c0; i0 < n; i0 += 32) {
    const int rh = min(32, n - i0);
    float ah[4] = {0.f, 0.f, 0.f, 0.f}, al[4] = {0.f, 0.f, 0.f, 0.f};  // rows ty + 8u, column tx
    if (!gram_identity) {
      for (int j0 = c0; j0 < i0; j0 += 32) {
        __syncthreads();
        for (int e = tid; e < 32 * 32; e += kTiThreads) {
          float h, l;
          const int r = e % 32, k = e / 32;  // L tile: column-major reads
          df::split((i0 + r < n) ? L[(size_t)(i0 + r) + (size_t)(j0 + k) * N] : 0.0, h, l);
          fL[r][k] = make_float2(h, l);
          const int kr = e / 32, c = e % 32;  // Y tile: row-major reads
          df::split((c < cw && j0 + kr < n) ? R[(size_t)(j0 + kr) * N + c0 + c] : 0.0, h, l);
          fY[kr][c] = make_float2(h, l);
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < 32; ++k) {
          const float2 y = fY[k][tx];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float2 a = fL[ty + 8 * u][k];
            df::mac(ah[u], al[u], a.x, a.y, y.x, y.y);
          }
          if ((k & 15) == 15) {
#pragma unroll
            for (int u = 0; u < 4; ++u) df::renorm(ah[u], al[u]);
          }
        }
      }
    }
    double acc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] = df::to_double(ah[u], al[u]);
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = ty + 8 * u;
      sAcc[r][tx] = ((i0 + r == c0 + tx) ? 1.0 : 0.0) - acc[u];  // E_i - sum
    }
    for (int e = tid; e < 32 * 32; e += kTiThreads) {  // diagonal block of L
      const int r = e % 32, k = e / 32;
      sL[r][k] = (r < rh && k < rh) ? L[(size_t)(i0 + r) + (size_t)(i0 + k) * N] : (r == k ? 1.0 : 0.0);
    }
    __syncthreads();
    if (tid < 32) {  // column tid: forward substitution with L_ii
      for (int r = 0; r < rh; ++r) {
        double sr = sAcc[r][tid];
        if (gram_identity) {
          sAcc[r][tid] = sr;
          continue;
        }
        for (int k = 0; k < r; ++k) sr -= sL[r][k] * sAcc[k][tid];
        sAcc[r][tid] = sr / sL[r][r];
      }
    }
    __syncthreads();
    for (int e = tid; e < rh * cw; e += kTiThreads) {
      const int r = e / cw, c = e % cw;
      R[(size_t)(i0 + r) * N + c0 + c] = sAcc[r][c];
    }
    // the next block row reads these rows of Y back through global memory
    __threadfence_block();
  }
}

// ---------------------------------------------------------------- reduction C = L^{-1} V L^{-T}

constexpr int GT = 32;  // output tile
constexpr int GK = 16;  // k tile

// mode 0: X = Linv V           X(i,j) = sum_{k <= i} Linv(i,k) V(k,j)
// mode 1: C = X Linv^T         C(i,j) = sum_{k <= j} X(i,k) Linv(j,k); C is
//         Hermitian, so only tiles with i0 <= j0 are formed and mirrored.
// Both products in double-float arithmetic (dfloat.cuh): FP64-class results
// (~1e-13 relative at N = 512) on the FP32 pipe, which issues 64 FMAs per
// FP64 one on B300. Operands are split into hi/lo floats once per tile.
template <int MODE>
__global__ void k_reduce_gemm_df(Batch b) {
  const int t = prob_of(b.order, blockIdx.z);
  const int n = b.nst[t];
  const int N = b.n_max;
  if (b.status[t]) return;
  const int i0 = blockIdx.x * GT, j0 = blockIdx.y * GT;
  if (i0 >= n || j0 >= n) return;
  if (MODE == 1 && i0 > j0) return;
  const double* Linv = b.Linv + mat_off(t, N);
  const double2* Z = (MODE == 0) ? (b.vis + mat_off(t, N)) : (b.X + mat_off(t, N));
  double2* out = (MODE == 0) ? (b.X + mat_off(t, N)) : (b.C + mat_off(t, N));
  __shared__ float2 sR[GK][GT + 1];  // (hi, lo)
  __shared__ float4 sZ[GK][GT + 1];  // (re hi, re lo, im hi, im lo)
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[u][c] = 0.f;
  const int kend = min(n, (MODE == 0 ? i0 : j0) + GT);
  for (int k0 = 0; k0 < kend; k0 += GK) {
    for (int e = threadIdx.x; e < GK * GT; e += blockDim.x) {
      const int kk = e / GT, ii = e % GT, k = k0 + kk;
      double r;
      double2 z;
      if (MODE == 0) {
        const int i = i0 + ii, j = j0 + ii;
        r = (k < n && i < n) ? Linv[(size_t)i * N + k] : 0.0;
        z = (k < n && j < n) ? Z[(size_t)k + (size_t)j * N] : make_double2(0.0, 0.0);
      } else {
        const int i = i0 + ii, j = j0 + ii;
        z = (k < n && i < n) ? Z[(size_t)i + (size_t)k * N] : make_double2(0.0, 0.0);
        r = (k < n && j < n) ? Linv[(size_t)j * N + k] : 0.0;
      }
      float2 fr;
      float4 fz;
      df::split(r, fr.x, fr.y);
      df::split(z.x, fz.x, fz.y);
      df::split(z.y, fz.z, fz.w);
      sR[kk][ii] = fr;
      sZ[kk][ii] = fz;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < GK; ++kk) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int ii = tx, jj = ty + 8 * u;
        const float2 r = (MODE == 0) ? sR[kk][ii] : sR[kk][jj];
        const float4 z = (MODE == 0) ? sZ[kk][jj] : sZ[kk][ii];
        df::mac(acc[u][0], acc[u][1], r.x, r.y, z.x, z.y);
        df::mac(acc[u][2], acc[u][3], r.x, r.y, z.z, z.w);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      df::renorm(acc[u][0], acc[u][1]);
      df::renorm(acc[u][2], acc[u][3]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + tx, j = j0 + ty + 8 * u;
    if (i < n && j < n) {
      const double2 v = make_double2(df::to_double(acc[u][0], acc[u][1]), df::to_double(acc[u][2], acc[u][3]));
      out[(size_t)i + (size_t)j * N] = v;
      if (MODE == 1 && i0 != j0) out[(size_t)j + (size_t)i * N] = make_double2(v.x, -v.y);
    }
  }
}

// The same reduction in FP32 for the mixed-precision eigensolver, whose FP32
// stage needs C only to FP32 accuracy and whose refinement applies
// L^{-1} V L^{-T} in factored form (eig_mixed.cu):
// mode 0: X32 = Linv V into the C buffer (float2, 2 N^2 per problem);
// mode 1: C32 = X32 Linv^T (upper tiles, mirrored) into the first half of the X buffer.
template <int MODE>
__global__ void k_reduce32(Batch b) {
  const int t = prob_of(b.order, blockIdx.z);
  const int n = b.nst[t];
  const int N = b.n_max;
  if (b.status[t]) return;
  const int i0 = blockIdx.x * GT, j0 = blockIdx.y * GT;
  if (i0 >= n || j0 >= n) return;
  if (MODE == 1 && i0 > j0) return;
  const double* Linv = b.Linv + mat_off(t, N);
  const size_t NN = (size_t)N * N;
  const float2* Z32 = reinterpret_cast<const float2*>(b.C) + (size_t)t * 2 * NN;
  const double2* V = b.vis + mat_off(t, N);
  float2* out = (MODE == 0) ? reinterpret_cast<float2*>(b.C) + (size_t)t * 2 * NN
                            : reinterpret_cast<float2*>(b.X) + (size_t)t * 2 * NN;
  __shared__ float sR[GK][GT + 1];
  __shared__ float2 sZ[GK][GT + 1];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float2 acc[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) acc[u] = make_float2(0.f, 0.f);
  const int kend = min(n, (MODE == 0 ? i0 : j0) + GT);
  for (int k0 = 0; k0 < kend; k0 += GK) {
    for (int e = threadIdx.x; e < GK * GT; e += blockDim.x) {
      const int kk = e / GT, ii = e % GT, k = k0 + kk;
      const int i = i0 + ii, j = j0 + ii;
      if (MODE == 0) {
        sR[kk][ii] = (k < n && i < n) ? (float)Linv[(size_t)i * N + k] : 0.f;
        const double2 z = (k < n && j < n) ? V[(size_t)k + (size_t)j * N] : make_double2(0.0, 0.0);
        sZ[kk][ii] = make_float2((float)z.x, (float)z.y);
      } else {
        sZ[kk][ii] = (k < n && i < n) ? Z32[(size_t)i + (size_t)k * N] : make_float2(0.f, 0.f);
        sR[kk][ii] = (k < n && j < n) ? (float)Linv[(size_t)j * N + k] : 0.f;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int ii = tx, jj = ty + 8 * u;
        const float r = (MODE == 0) ? sR[kk][ii] : sR[kk][jj];
        const float2 z = (MODE == 0) ? sZ[kk][jj] : sZ[kk][ii];
        acc[u].x = fmaf(r, z.x, acc[u].x);
        acc[u].y = fmaf(r, z.y, acc[u].y);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + tx, j = j0 + ty + 8 * u;
    if (i < n && j < n) {
      out[(size_t)i + (size_t)j * N] = acc[u];
      if (MODE == 1 && i0 != j0) out[(size_t)j + (size_t)i * N] = make_float2(acc[u].x, -acc[u].y);
    }
  }
}

// G = I in the mixed eigensolver: C32 = the Hermitian part of V, in FP32,
// into the first half of the X buffer.
__global__ void k_herm32(Batch b) {
  const int t = prob_of(b.order, blockIdx.z);
  const int n = b.nst[t];
  const int N = b.n_max;
  if (b.status[t]) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= n || j >= n) return;
  const double2* V = b.vis + mat_off(t, N);
  const double2 a = V[(size_t)i + (size_t)j * N], c = V[(size_t)j + (size_t)i * N];
  float2* C32 = reinterpret_cast<float2*>(b.X) + (size_t)t * 2 * (size_t)N * N;
  C32[(size_t)i + (size_t)j * N] = make_float2((float)(0.5 * (a.x + c.x)), i == j ? 0.f : (float)(0.5 * (a.y - c.y)));
}

// C <- (C + C^H)/2 (or C <- Hermitian part of V when G = I): removes
// rounding-level asymmetry before the Jacobi sweeps.
__global__ void k_hermitize(Batch b, int from_vis) {
  const int t = prob_of(b.order, blockIdx.z);
  const int n = b.nst[t];
  const int N = b.n_max;
  if (b.status[t]) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= n || j >= n || i > j) return;
  const double2* S = from_vis ? (b.vis + mat_off(t, N)) : (b.C + mat_off(t, N));
  double2 a = S[(size_t)i + (size_t)j * N];
  double2 c = S[(size_t)j + (size_t)i * N];
  double2 h = make_double2(0.5 * (a.x + c.x), 0.5 * (a.y - c.y));
  if (i == j) h.y = 0.0;
  double2* C = b.C + mat_off(t, N);
  C[(size_t)i + (size_t)j * N] = h;
  C[(size_t)j + (size_t)i * N] = make_double2(h.x, -h.y);
}

// ---------------------------------------------------------------- select + pack

// Keep the n_eig algebraically largest eigenvalues (descending, ties by lower
// Jacobi index), assign filter weights and levels, back-transform the kept
// eigenvectors a = L^{-T} q, and pack them for the synthesis kernels.
// Grid (T, eigenvector groups of kSelE): every CTA ranks the step's
// eigenvalues; group 0 also writes levels, weights and station coordinates;
// each group back-transforms its kSelE kept eigenvectors (double-float).
constexpr int kSelE = 8;

__global__ void k_select(Batch b, int n_level, const double* all_bounds, int filter) {
  const int t = prob_of(b.order, blockIdx.x), eg = blockIdx.y;
  const int n = b.nst[t];
  const int N = b.n_max;
  const int K = b.neig[t];
  const int KM = b.k_max;
  const double wl = b.wl[t];
  const double* bounds = all_bounds + (size_t)step_chan(b, t) * 2 * n_level;
  __shared__ int idx[kMaxEig];
  const int st = b.status[t];
  if (st) {
    if (eg != 0) return;
    for (int e = threadIdx.x; e < KM; e += blockDim.x) b.level[(size_t)t * KM + e] = -1;
    if (threadIdx.x == 0) {
      b.nkept[t] = 0;
      atomicOr(b.flag, st);
    }
    return;
  }
  const double* mu = b.mu + (size_t)t * N;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double mi = mu[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double mj = mu[j];
      rank += (mj > mi) || (mj == mi && j < i);
    }
    if (rank < K) idx[rank] = i;
  }
  __syncthreads();
  for (int e = threadIdx.x; eg == 0 && e < KM; e += blockDim.x) {
    int lev = -1;
    double m = 0.0, w = 0.0;
    if (e < K) {
      m = mu[idx[e]];
      w = (filter == 0) ? m : 1.0;
      if (b.eigen) {  // eigenimages: the level is the rank
        lev = e;
      } else {
        for (int l = 0; l < n_level; ++l) {
          if (bounds[l] <= m && m < bounds[n_level + l]) {
            lev = l;
            break;
          }
        }
      }
    }
    b.sel_mu[(size_t)t * KM + e] = m;
    b.wt[(size_t)t * KM + e] = w;
    b.level[(size_t)t * KM + e] = lev;
  }
  // a_e[i] = sum_{k >= i} Linv(k, i) q_{idx[e]}[k] for this group's eigenvectors, in double-float:
  // the group's columns of Q staged in shared memory as hi/lo pairs, one row i per thread
  const int e0 = eg * kSelE, ne = min(kSelE, K - e0);
  if (ne > 0) {
    extern __shared__ __align__(16) unsigned char selsm[];
    float4* sq = reinterpret_cast<float4*>(selsm);  // [kSelE][N]
    const double* Linv = b.Linv + mat_off(t, N);
    const double2* Qm = b.Q + mat_off(t, N);
    for (int w = threadIdx.x; w < ne * n; w += blockDim.x) {
      const int k = w % n, e = w / n;
      const double2 qk = Qm[(size_t)idx[e0 + e] * N + k];
      float4 f;
      df::split(qk.x, f.x, f.y);
      df::split(qk.y, f.z, f.w);
      sq[(size_t)e * N + k] = f;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      float acc[kSelE][4];
#pragma unroll
      for (int e = 0; e < kSelE; ++e) acc[e][0] = acc[e][1] = acc[e][2] = acc[e][3] = 0.f;
      for (int k = i; k < n; ++k) {
        float rh, rl;
        df::split(Linv[(size_t)k * N + i], rh, rl);
#pragma unroll
        for (int e = 0; e < kSelE; ++e) {
          if (e < ne) {
            const float4 q = sq[(size_t)e * N + k];
            df::mac(acc[e][0], acc[e][1], rh, rl, q.x, q.y);
            df::mac(acc[e][2], acc[e][3], rh, rl, q.z, q.w);
          }
        }
        if (((k - i) & 15) == 15) {
#pragma unroll
          for (int e = 0; e < kSelE; ++e) {
            df::renorm(acc[e][0], acc[e][1]);
            df::renorm(acc[e][2], acc[e][3]);
          }
        }
      }
#pragma unroll
      for (int e = 0; e < kSelE; ++e) {
        if (e < ne) {
          const double2 a = make_double2(df::to_double(acc[e][0], acc[e][1]), df::to_double(acc[e][2], acc[e][3]));
          b.W64[((size_t)t * KM + e0 + e) * N + i] = a;
          b.W32[((size_t)t * N + i) * KM + e0 + e] = make_float2((float)a.x, (float)a.y);
        }
      }
    }
  }
  if (eg != 0) return;
  // station coordinates in cycles per unit direction cosine, float hi/lo
  const double* p = b.st + (size_t)t * 3 * N;
  float* q = b.q + (size_t)t * 6 * N;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    for (int c = 0; c < 3; ++c) {
      const double v = p[(size_t)c * N + i] / wl;
      const float hi = (float)v;
      q[(size_t)c * N + i] = hi;
      q[(size_t)(c + 3) * N + i] = (float)(v - (double)hi);
    }
  }
  if (threadIdx.x == 0) b.nkept[t] = K;
}

__global__ void k_pixel_split(const double* xyz, float* hl, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int c = 0; c < 3; ++c) {
    double v = xyz[(size_t)c * n + i];
    float hi = (float)v;
    hl[(size_t)c * n + i] = hi;
    hl[(size_t)(c + 3) * n + i] = (float)(v - (double)hi);
  }
}

// Complex64 visibilities widened to complex128 (exact), grid-stride.
__global__ void k_vis_widen(const float2* __restrict__ in, double2* __restrict__ out, size_t n) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const float2 v = in[i];
    out[i] = make_double2((double)v.x, (double)v.y);
  }
}

}  // namespace

void launch_gram(const Batch& b, int gram_identity, cudaStream_t s) {
  dim3 blk(16, 16), grd((b.n_max + 15) / 16, (b.n_max + 15) / 16, b.T);
  k_gram<<<grd, blk, 0, s>>>(b, gram_identity);
}

void launch_cholesky(const Batch& b, int gram_identity, cudaStream_t s) {
  const size_t smem = sizeof(double) * (size_t)(b.n_max + 32) * kChLd;
  if (!gram_identity) {
    if (smem <= 200 * 1024) {
      cudaFuncSetAttribute(k_cholesky_blk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_cholesky_blk<<<b.T, kChThreads, smem, s>>>(b);
    } else {
      k_cholesky<<<b.T, 256, 0, s>>>(b);
    }
  }
  k_trinv_blk<<<dim3((b.n_max + 31) / 32, b.T), kTiThreads, 0, s>>>(b, gram_identity);
}

void launch_reduce(const Batch& b, int gram_identity, cudaStream_t s) {
  dim3 hb(16, 16), hg((b.n_max + 15) / 16, (b.n_max + 15) / 16, b.T);
  if (gram_identity) {
    k_hermitize<<<hg, hb, 0, s>>>(b, 1);
    return;
  }
  dim3 grd((b.n_max + GT - 1) / GT, (b.n_max + GT - 1) / GT, b.T);
  k_reduce_gemm_df<0><<<grd, 256, 0, s>>>(b);
  k_reduce_gemm_df<1><<<grd, 256, 0, s>>>(b);
  k_hermitize<<<hg, hb, 0, s>>>(b, 0);
}

void launch_reduce32(const Batch& b, int gram_identity, cudaStream_t s) {
  if (gram_identity) {
    dim3 hb(16, 16), hg((b.n_max + 15) / 16, (b.n_max + 15) / 16, b.T);
    k_herm32<<<hg, hb, 0, s>>>(b);
    return;
  }
  dim3 grd((b.n_max + GT - 1) / GT, (b.n_max + GT - 1) / GT, b.T);
  k_reduce32<0><<<grd, 256, 0, s>>>(b);
  k_reduce32<1><<<grd, 256, 0, s>>>(b);
}

void launch_jacobi(const Batch& b, double tol, int max_sweeps, cudaStream_t s) {
  JacobiArgs a;
  a.C = b.C;
  a.Q = b.Q;
  a.mu = b.mu;
  a.status = b.status;
  a.sweeps = b.sweeps;
  a.n = b.nst;
  a.ld = b.n_max;
  a.stride = (size_t)b.n_max * b.n_max;
  a.report_nonconv = 1;
  a.order = b.order;
  launch_jacobi_args(a, b.T, false, tol, max_sweeps, s);
}

void launch_select(const Batch& b, int n_level, const double* d_bounds, int filter, cudaStream_t s) {
  const int smem = (int)(sizeof(float4) * kSelE * (size_t)b.n_max);
  cudaFuncSetAttribute(k_select, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  k_select<<<dim3(b.T, std::max(1, (b.k_max + kSelE - 1) / kSelE)), 256, smem, s>>>(b, n_level, d_bounds, filter);
}

void launch_pixel_split(const double* d_xyz, float* d_hl, int64_t n, cudaStream_t s) {
  k_pixel_split<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d_xyz, d_hl, n);
}

void launch_vis_widen(const float2* d_in, double2* d_out, size_t n, cudaStream_t s) {
  if (n == 0) return;
  const size_t blocks = std::min<size_t>((n + 255) / 256, (size_t)148 * 16);
  k_vis_widen<<<(unsigned)blocks, 256, 0, s>>>(d_in, d_out, n);
}

}  // namespace bipp
