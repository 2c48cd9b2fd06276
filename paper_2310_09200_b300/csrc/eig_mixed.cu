// eig_mixed.cu — mixed-precision generalised eigensolve (BIPP_EIG_MIXED).
//
// Same result as the FP64 Jacobi of Sec. 2.3 (Eq. eigenvaleq) for the pairs
// that are kept, at a fraction of the FP64 work, which matters on B300 where
// the FP64 pipe runs at 1/58 of the FP32 rate. Only the kp = min(n, n_eig + 16)
// leading pairs are computed (Sec. 2.6 keeps the n_eig largest):
//   1. the reduced matrix C = L^{-1} V L^{-T} (formed in FP64) is rounded to
//      FP32 and reduced to real tridiagonal form, C32 = H T H^H (tridiag32.cuh);
//      the kp largest eigenvalues of T come from multisection, their
//      eigenvectors from inverse iteration, and only those kp columns are
//      back-transformed, X = H Z_k (tridiag_sel.cuh);
//   2. X is refined in FP64-class arithmetic with the operator C itself:
//        orthonormalise X (Cholesky QR), Y = C X, H = X^H Y,
//        H = U diag(theta) U^H (FP64 Jacobi on kp x kp), X <- X U, Y <- Y U,
//        R = Y - X diag(theta) (residuals),
//        X <- X - H P (T - theta_j I)^{-1} P H^H R, P = I - Z_k Z_k^T,
//      i.e. the FP32 shift-and-invert of C on the complement of the kept
//      directions (the same correction as Q32 (M32 - theta)^{-1} Q32^H over the
//      complement of a full FP32 eigendecomposition, without computing it);
//      the correction runs in FP32, as it carries no more accuracy than the
//      FP32 decomposition, while the residual it corrects is formed in FP64;
//      each pass contracts the error by the FP32 stage's relative accuracy over
//      the spectral gap (about 5e-6 per pass here); a problem whose kept
//      residuals fall below 100 * jacobi_tol * ||C||_F stops early (after one
//      correction, typically), the rest run at most kPasses passes.
//   3. theta and X replace the Jacobi eigenvalues and eigenvectors; the
//      residual of the last pass is checked against 1e3 * jacobi_tol * ||C||_F.
// FP64-class cost per pass is O(n^2 kp) (one n x n by n x kp product) instead
// of the O(n^3) of every FP64 Jacobi sweep, and the FP32 stage is O(n^3) for
// the reduction plus O(n^2 kp) for the kp vectors.
#include <math.h>

#include <algorithm>

#include "bipp_internal.cuh"
#include "dfloat.cuh"
#include "jacobi.cuh"
#include "tridiag32.cuh"
#include "tridiag_sel.cuh"

namespace bipp {
namespace {

constexpr int kPad = 16;       // extra leading pairs refined beyond n_eig
constexpr int kPasses = 4;     // refinement passes at most
constexpr int kMxDone = kMxDoneBit;  // st2 bit: residual met the early-exit bound, later passes skip the step
constexpr int GT = 32, GK = 16;
static_assert(6 + 2 + 19 * (kPasses - 1) + 12 == kMixedLaunches, "launch count of the mixed eigensolver");

// Shape codes of the batched complex products: dimension = n_st or kp of the problem.
enum Dim { DN = 0, DKP = 1 };

__device__ __forceinline__ int dim_of(int code, int n, int kp) { return code == DN ? n : kp; }


// Problem t takes no further part in the refinement: an error status, or its
// residual already met the early-exit bound.
__device__ __forceinline__ bool mx_skip(const int* status, const int* st2, int t) {
  return status[t] || (st2[t] & kMxDone);
}

// The FP64-class products of the refinement in double-float arithmetic
// (dfloat.cuh): out[i, j] = sum_k op(A)[i, k] B[k, j], op = identity or
// conjugate transpose, all operands column-major with per-problem strides,
// with ~2^-48 relative rounding per operation instead of FP64's 2^-53, at
// several times the FP64 pipe's rate. Operands are split into hi/lo floats
// once per tile. The real and imaginary accumulations of an output run side
// by side on the packed FP32 operations (df::mac2): re += ar br, im += ar bi
// as one packed step and re += (-ai) bi, im += ai br as the next, so the
// operands are staged in shared memory already paired (and negated where
// mac2 needs it). Column blocks of 8 that lie wholly past the problem's
// width are skipped (a warp-uniform test), so kp = 80 columns cost 80, not
// the 96 of three 32-wide tiles. With CONJ_T the product is one of the
// refinement's Hermitian kp x kp matrices (X^H X, X1^H C X1): only the tiles
// on and above the diagonal are computed, and each tile above it is also
// written, conjugated, to its mirror below.
struct DfA2 {  // one element a of op(A), paired for the two packed steps
  float2 h1, nh1, nl1;  // (ar, ar) hi, and -(ar, ar) hi / lo
  float2 h2, nh2, nl2;  // (-ai, ai) hi, and -(-ai, ai) hi / lo
};
struct DfB2 {  // one element b of B
  float2 h1, l1;  // (br, bi) hi / lo
  float2 h2, l2;  // (bi, br) hi / lo
};
template <bool CONJ_T>
__global__ void k_zgemm_df(const int* nst, const int* kp, int mc, int nc, int kc, const double2* A, size_t sa,
                           int lda, const double2* B, size_t sb, int ldb, double2* out, size_t so, int ldo,
                           const int* status, const int* st2) {
  const int t = blockIdx.z;
  if (mx_skip(status, st2, t)) return;
  const int n = nst[t], k_p = kp[t];
  const int M = dim_of(mc, n, k_p), NN = dim_of(nc, n, k_p), K = dim_of(kc, n, k_p);
  const int i0 = blockIdx.x * GT, j0 = blockIdx.y * GT;
  if (i0 >= M || j0 >= NN || (CONJ_T && blockIdx.x > blockIdx.y)) return;
  A += (size_t)t * sa;
  B += (size_t)t * sb;
  out += (size_t)t * so;
  __shared__ DfA2 sA[GK][GT + 1];
  __shared__ DfB2 sB[GK][GT + 1];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int nu = min(4, max(0, (NN - j0 - ty + 7) >> 3));  // column blocks u < nu hold columns < NN
  float2 ah[4], al[4];  // [u] (re, im) hi and lo accumulators
#pragma unroll
  for (int u = 0; u < 4; ++u) ah[u] = al[u] = make_float2(0.f, 0.f);
  for (int k0 = 0; k0 < K; k0 += GK) {
    for (int e = threadIdx.x; e < GK * GT; e += blockDim.x) {
      const int kk = e / GT, ii = e % GT, k = k0 + kk;
      const int i = i0 + ii, j = j0 + ii;
      double2 a = make_double2(0.0, 0.0), bv = make_double2(0.0, 0.0);
      if (k < K && i < M) {
        if (CONJ_T) {
          a = A[(size_t)k + (size_t)i * lda];
          a.y = -a.y;
        } else {
          a = A[(size_t)i + (size_t)k * lda];
        }
      }
      if (k < K && j < NN) bv = B[(size_t)k + (size_t)j * ldb];
      float arh, arl, aih, ail, brh, brl, bih, bil;
      df::split(a.x, arh, arl);
      df::split(a.y, aih, ail);
      df::split(bv.x, brh, brl);
      df::split(bv.y, bih, bil);
      DfA2 pa;
      pa.h1 = make_float2(arh, arh);
      pa.nh1 = make_float2(-arh, -arh);
      pa.nl1 = make_float2(-arl, -arl);
      pa.h2 = make_float2(-aih, aih);
      pa.nh2 = make_float2(aih, -aih);
      pa.nl2 = make_float2(ail, -ail);
      DfB2 pb;
      pb.h1 = make_float2(brh, bih);
      pb.l1 = make_float2(brl, bil);
      pb.h2 = make_float2(bih, brh);
      pb.l2 = make_float2(bil, brl);
      sA[kk][ii] = pa;
      sB[kk][ii] = pb;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < GK; ++kk) {
      const DfA2 a = sA[kk][tx];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (u >= nu) break;
        const DfB2 bv = sB[kk][ty + 8 * u];
        df::mac2(ah[u], al[u], a.h1, a.nh1, a.nl1, bv.h1, bv.l1);  // (re, im) += ar (br, bi)
        df::mac2(ah[u], al[u], a.h2, a.nh2, a.nl2, bv.h2, bv.l2);  //          + (-ai, ai) (bi, br)
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) df::renorm2(ah[u], al[u]);
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + tx, j = j0 + ty + 8 * u;
    if (i < M && j < NN) {
      const double2 v = make_double2(df::to_double(ah[u].x, al[u].x), df::to_double(ah[u].y, al[u].y));
      out[(size_t)i + (size_t)j * ldo] = v;
      if (CONJ_T && blockIdx.x < blockIdx.y) out[(size_t)j + (size_t)i * ldo] = make_double2(v.x, -v.y);
    }
  }
}

// The same products in plain FP32 arithmetic (FP64 operands and results): for
// the first pass, whose orthonormalisation and Rayleigh-Ritz matrix only need
// the FP32 stage's accuracy (the products that form the residual stay in
// double-float).
template <bool CONJ_T>
__global__ void k_zgemm_f32(const int* nst, const int* kp, int mc, int nc, int kc, const double2* A, size_t sa,
                            int lda, const double2* B, size_t sb, int ldb, double2* out, size_t so, int ldo,
                            const int* status, const int* st2) {
  const int t = blockIdx.z;
  if (mx_skip(status, st2, t)) return;
  const int n = nst[t], k_p = kp[t];
  const int M = dim_of(mc, n, k_p), NN = dim_of(nc, n, k_p), K = dim_of(kc, n, k_p);
  const int i0 = blockIdx.x * GT, j0 = blockIdx.y * GT;
  if (i0 >= M || j0 >= NN || (CONJ_T && blockIdx.x > blockIdx.y)) return;
  A += (size_t)t * sa;
  B += (size_t)t * sb;
  out += (size_t)t * so;
  __shared__ float2 sA[GK][GT + 1];
  __shared__ float2 sB[GK][GT + 1];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int nu = min(4, max(0, (NN - j0 - ty + 7) >> 3));
  float2 acc[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) acc[u] = make_float2(0.f, 0.f);
  for (int k0 = 0; k0 < K; k0 += GK) {
    for (int e = threadIdx.x; e < GK * GT; e += blockDim.x) {
      const int kk = e / GT, ii = e % GT, k = k0 + kk;
      const int i = i0 + ii, j = j0 + ii;
      double2 a = make_double2(0.0, 0.0), bv = make_double2(0.0, 0.0);
      if (k < K && i < M) {
        if (CONJ_T) {
          a = A[(size_t)k + (size_t)i * lda];
          a.y = -a.y;
        } else {
          a = A[(size_t)i + (size_t)k * lda];
        }
      }
      if (k < K && j < NN) bv = B[(size_t)k + (size_t)j * ldb];
      sA[kk][ii] = make_float2((float)a.x, (float)a.y);
      sB[kk][ii] = make_float2((float)bv.x, (float)bv.y);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      const float2 a = sA[kk][tx];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (u >= nu) break;
        const float2 bv = sB[kk][ty + 8 * u];
        acc[u].x = fmaf(a.x, bv.x, fmaf(-a.y, bv.y, acc[u].x));
        acc[u].y = fmaf(a.x, bv.y, fmaf(a.y, bv.x, acc[u].y));
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + tx, j = j0 + ty + 8 * u;
    if (i < M && j < NN) {
      out[(size_t)i + (size_t)j * ldo] = make_double2(acc[u].x, acc[u].y);
      if (CONJ_T && blockIdx.x < blockIdx.y) out[(size_t)j + (size_t)i * ldo] = make_double2(acc[u].x, -acc[u].y);
    }
  }
}

// The factored operator of the refinement, C = L^{-1} V L^{-T}, applied as
// three products: out = op(Linv) B with Linv the row-major FP64 inverse
// Cholesky factor (real), B an n x kp complex block (column-major, ld N,
// NN apart), op = transpose (UPPER: (L^{-T})_ik = Linv[k][i], k >= i) or
// identity (L^{-1}, k <= i); double-float arithmetic as k_zgemm_df, the zero
// triangle skipped.
template <bool UPPER>
__global__ void k_rgemm_df(const Batch b, const MixedWs w, const double2* B0, double2* out0) {
  const int t = blockIdx.z;
  if (mx_skip(b.status, w.st2, t)) return;
  const int n = b.nst[t], k_p = w.kp[t], N = b.n_max;
  const size_t NN = (size_t)N * N;
  const int i0 = blockIdx.x * GT, j0 = blockIdx.y * GT;
  if (i0 >= n || j0 >= k_p) return;
  const double* Linv = b.Linv + (size_t)t * NN;
  const double2* B = B0 + (size_t)t * NN;
  double2* out = out0 + (size_t)t * NN;
  struct RA {
    float2 h, nh, nl;  // (a, a) hi, -(a, a) hi / lo
  };
  __shared__ RA sA[GK][GT + 1];
  __shared__ float4 sB[GK][GT + 1];  // (re hi, im hi, re lo, im lo)
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int nu = min(4, max(0, (k_p - j0 - ty + 7) >> 3));
  float2 ah[4], al[4];  // [u] (re, im) hi and lo accumulators
#pragma unroll
  for (int u = 0; u < 4; ++u) ah[u] = al[u] = make_float2(0.f, 0.f);
  const int kbeg = UPPER ? (i0 / GK) * GK : 0, kend = UPPER ? n : min(n, i0 + GT);
  for (int k0 = kbeg; k0 < kend; k0 += GK) {
    for (int e = threadIdx.x; e < GK * GT; e += blockDim.x) {
      const int kk = e / GT, ii = e % GT, k = k0 + kk;
      const int i = i0 + ii, j = j0 + ii;
      double a = 0.0;
      if (k < n && i < n) a = UPPER ? (k >= i ? Linv[(size_t)k * N + i] : 0.0) : (k <= i ? Linv[(size_t)i * N + k] : 0.0);
      const double2 bv = (k < n && j < k_p) ? B[(size_t)k + (size_t)j * N] : make_double2(0.0, 0.0);
      float ahi, alo, brh, brl, bih, bil;
      df::split(a, ahi, alo);
      df::split(bv.x, brh, brl);
      df::split(bv.y, bih, bil);
      RA pa;
      pa.h = make_float2(ahi, ahi);
      pa.nh = make_float2(-ahi, -ahi);
      pa.nl = make_float2(-alo, -alo);
      sA[kk][ii] = pa;
      sB[kk][ii] = make_float4(brh, bih, brl, bil);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < GK; ++kk) {
      const RA a = sA[kk][tx];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (u >= nu) break;
        const float4 bv = sB[kk][ty + 8 * u];
        df::mac2(ah[u], al[u], a.h, a.nh, a.nl, make_float2(bv.x, bv.y), make_float2(bv.z, bv.w));
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) df::renorm2(ah[u], al[u]);
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + tx, j = j0 + ty + 8 * u;
    if (i < n && j < k_p)
      out[(size_t)i + (size_t)j * N] = make_double2(df::to_double(ah[u].x, al[u].x), df::to_double(ah[u].y, al[u].y));
  }
}


// The kp back-transformed FP32 eigenvectors (rank order) become the FP64
// start X of the refinement; ||C||_F = ||T||_F.
__global__ void k_mx_pick(Batch b, MixedWs w, const float2* Q32, size_t qstride) {
  const int t = blockIdx.x;
  if (b.status[t]) return;
  const int n = b.nst[t], N = b.n_max, kp = w.kp[t];
  const float2* Qt = Q32 + (size_t)t * qstride;
  double2* X = b.Q + (size_t)t * N * N;
  if (threadIdx.x == 0) {
    w.cnorm[t] = (double)w.tnorm[t];
    b.sweeps[t] = 0;
  }
  for (int e = threadIdx.x; e < n * kp; e += blockDim.x) {
    const int i = e % n, j = e / n;
    const float2 v = Qt[(size_t)i + (size_t)j * N];
    X[(size_t)i + (size_t)j * N] = make_double2(v.x, v.y);
  }
}

// W such that X W has orthonormal columns, from the kp x kp Gram matrix S of
// X. One CTA (256 threads) per step. Usually S^{-1/2} by its series (below);
// otherwise S = R^H R (upper Cholesky) and W = R^{-1}, in one
// kp x kp shared-memory buffer: R in the upper triangle, W transposed into
// the strict lower triangle (W(i, c) at (c, i)) with its diagonal beside it.
// The factorisation is right-looking (row j of R, then the trailing update in
// parallel); W is solved one thread per column.
// Dynamic shared memory: (kp_max^2 + kp_max) complex doubles.
__global__ void k_mx_cholinv(Batch b, MixedWs w, const double2* S0, double2* W0, size_t stride, int ld) {
  const int t = blockIdx.x;
  if (mx_skip(b.status, w.st2, t)) return;
  const int kp = w.kp[t];
  const double2* S = S0 + (size_t)t * stride;
  double2* W = W0 + (size_t)t * stride;
  extern __shared__ __align__(16) unsigned char cism[];
  double2* B = reinterpret_cast<double2*>(cism);  // column-major, leading dimension kp
  double2* wd = B + (size_t)kp * kp;              // diagonal of W
  __shared__ int bad;
  __shared__ double s_inv;
  __shared__ double red[256];
  if (threadIdx.x == 0) bad = 0;
  // Nearly orthonormal columns (max |S - I| < 0.05, the usual case): W = S^{-1/2} by its series
  // I - E/2 + 3/8 E^2 - 5/16 E^3 (E = S - I; truncation 35/128 |E|^4 <= 2e-6, and 1e-28 once the
  // columns are orthonormal to FP32 accuracy), the linear term in FP64 and the small E^2, E^3
  // terms in FP32, instead of the FP64 Cholesky below (FP64 runs at 1/64 of FP32 here).
  double emax = 0.0;
  for (int e = threadIdx.x; e < kp * kp; e += blockDim.x) {
    const int i = e % kp, c = e / kp;
    const double2 v = S[(size_t)i + (size_t)c * ld];
    emax = fmax(emax, fmax(fabs(v.x - (i == c ? 1.0 : 0.0)), fabs(v.y)));
  }
  red[threadIdx.x] = emax;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (red[0] < 0.05) {
    float2* E = reinterpret_cast<float2*>(cism);  // E, then E^2, kp x kp each
    float2* E2 = E + (size_t)kp * kp;
    for (int e = threadIdx.x; e < kp * kp; e += blockDim.x) {
      const int i = e % kp, c = e / kp;
      const double2 v = S[(size_t)i + (size_t)c * ld];
      E[e] = make_float2((float)(v.x - (i == c ? 1.0 : 0.0)), (float)v.y);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kp * kp; e += blockDim.x) {
      const int i = e % kp, c = e / kp;
      float2 a = make_float2(0.f, 0.f);
      for (int k = 0; k < kp; ++k) {
        const float2 x = E[i + (size_t)k * kp], y = E[k + (size_t)c * kp];
        a.x = fmaf(x.x, y.x, fmaf(-x.y, y.y, a.x));
        a.y = fmaf(x.x, y.y, fmaf(x.y, y.x, a.y));
      }
      E2[e] = a;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kp * kp; e += blockDim.x) {
      const int i = e % kp, c = e / kp;
      float2 a = make_float2(0.f, 0.f);  // (E E^2)(i, c)
      for (int k = 0; k < kp; ++k) {
        const float2 x = E[i + (size_t)k * kp], y = E2[k + (size_t)c * kp];
        a.x = fmaf(x.x, y.x, fmaf(-x.y, y.y, a.x));
        a.y = fmaf(x.x, y.y, fmaf(x.y, y.x, a.y));
      }
      const double2 sv = S[(size_t)i + (size_t)c * ld];
      const float2 e2 = E2[e];
      W[(size_t)i + (size_t)c * ld] =
          make_double2((i == c ? 1.5 : 0.0) - 0.5 * sv.x + (double)(0.375f * e2.x - 0.3125f * a.x),
                       -0.5 * sv.y + (double)(0.375f * e2.y - 0.3125f * a.y));
    }
    return;
  }
  for (int e = threadIdx.x; e < kp * kp; e += blockDim.x) {
    const int i = e % kp, c = e / kp;
    if (i <= c) B[e] = S[(size_t)i + (size_t)c * ld];
  }
  __syncthreads();
  for (int j = 0; j < kp; ++j) {
    if (threadIdx.x == 0) {
      const double d = B[j + (size_t)j * kp].x;
      if (!(d > 0.0)) bad = 1;
      const double r = sqrt(fmax(d, 1e-300));
      B[j + (size_t)j * kp] = make_double2(r, 0.0);
      s_inv = 1.0 / r;
    }
    __syncthreads();
    const double inv = s_inv;
    for (int c = j + 1 + threadIdx.x; c < kp; c += blockDim.x) {
      const double2 v = B[j + (size_t)c * kp];
      B[j + (size_t)c * kp] = make_double2(v.x * inv, v.y * inv);
    }
    __syncthreads();
    const int m = kp - j - 1;  // S(c1, c2) -= conj(R(j, c1)) R(j, c2), j < c1 <= c2
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int c1 = j + 1 + e % m, c2 = j + 1 + e / m;
      if (c1 > c2) continue;
      const double2 a1 = B[j + (size_t)c1 * kp], a2 = B[j + (size_t)c2 * kp];
      double2 v = B[c1 + (size_t)c2 * kp];
      v.x -= a1.x * a2.x + a1.y * a2.y;
      v.y -= a1.x * a2.y - a1.y * a2.x;
      B[c1 + (size_t)c2 * kp] = v;
    }
    __syncthreads();
  }
  // W = R^{-1}: column c solves R w = e_c from the bottom up
  for (int c = threadIdx.x; c < kp; c += blockDim.x) {
    for (int i = c; i >= 0; --i) {
      double2 sm = make_double2(i == c ? 1.0 : 0.0, 0.0);
      for (int k = i + 1; k <= c; ++k) {
        const double2 r = B[i + (size_t)k * kp];
        const double2 x = (k == c) ? wd[c] : B[c + (size_t)k * kp];
        sm.x -= r.x * x.x - r.y * x.y;
        sm.y -= r.x * x.y + r.y * x.x;
      }
      const double rii = B[i + (size_t)i * kp].x;
      const double2 v = make_double2(sm.x / rii, sm.y / rii);
      if (i == c) wd[c] = v;
      else B[c + (size_t)i * kp] = v;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kp * kp; e += blockDim.x) {
    const int i = e % kp, c = e / kp;
    W[(size_t)i + (size_t)c * ld] = (i < c) ? B[c + (size_t)i * kp] : (i == c ? wd[c] : make_double2(0.0, 0.0));
  }
  if (threadIdx.x == 0 && bad) b.status[t] |= kStatusNotConverged;
}
__global__ void k_mx_herm(Batch b, MixedWs w, double2* H0, size_t stride, int ld) {
  const int t = blockIdx.x;
  if (mx_skip(b.status, w.st2, t)) return;
  const int kp = w.kp[t];
  double2* H = H0 + (size_t)t * stride;
  for (int e = threadIdx.x; e < kp * kp; e += blockDim.x) {
    const int i = e % kp, j = e / kp;
    if (i > j) continue;
    const double2 a = H[i + (size_t)j * ld], c = H[j + (size_t)i * ld];
    double2 h = make_double2(0.5 * (a.x + c.x), 0.5 * (a.y - c.y));
    if (i == j) h.y = 0.0;
    H[i + (size_t)j * ld] = h;
    H[j + (size_t)i * ld] = make_double2(h.x, -h.y);
  }
}

// TO32: H32 = fp32(H) (kp x kp, ld KP); else U = fp64(U32). The FP32 views
// lie 2 N^2 float2 apart per problem, the FP64 blocks N^2 double2 apart.
template <bool TO32>
__global__ void k_mx_cvt(Batch b, MixedWs w, double2* D0, float2* F0, size_t stride, int ld) {
  const int t = blockIdx.x;
  if (mx_skip(b.status, w.st2, t)) return;
  const int kp = w.kp[t];
  double2* D = D0 + (size_t)t * stride;
  float2* F = F0 + (size_t)t * 2 * stride;
  for (int e = threadIdx.x; e < kp * kp; e += blockDim.x) {
    const size_t o = (size_t)(e % kp) + (size_t)(e / kp) * ld;
    if (TO32) F[o] = make_float2((float)D[o].x, (float)D[o].y);
    else D[o] = make_double2((double)F[o].x, (double)F[o].y);
  }
}

// R = Y - X diag(theta) in place of Y; rnorm[j] = ||R[:, j]||.
__global__ void k_mx_resid(Batch b, MixedWs w, const double2* X0, double2* Y0, float2* R32, size_t stride) {
  const int t = blockIdx.y, j = blockIdx.x;
  if (mx_skip(b.status, w.st2, t)) return;
  const int n = b.nst[t], N = b.n_max, kp = w.kp[t];
  if (j >= kp) return;
  const double th = w.theta[(size_t)t * w.KP + j];
  const double2* X = X0 + (size_t)t * stride + (size_t)j * N;
  double2* Y = Y0 + (size_t)t * stride + (size_t)j * N;
  float2* Rf = R32 + (size_t)t * stride * 2 + (size_t)j * N;  // stride counts double2 elements
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double2 x = X[i], y = Y[i];
    const double2 r = make_double2(y.x - th * x.x, y.y - th * x.y);
    Y[i] = r;
    Rf[i] = make_float2((float)r.x, (float)r.y);
    s += r.x * r.x + r.y * r.y;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) w.rnorm[(size_t)t * w.KP + j] = sqrt(red[0]);
}

// X <- X - D on the n x kp block.
__global__ void k_mx_sub(Batch b, MixedWs w, double2* X0, const float2* D0, size_t stride_x, size_t stride_d) {
  const int t = blockIdx.y;
  if (mx_skip(b.status, w.st2, t)) return;
  const int n = b.nst[t], N = b.n_max, kp = w.kp[t];
  double2* X = X0 + (size_t)t * stride_x;
  const float2* D = D0 + (size_t)t * stride_d;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * kp; e += gridDim.x * blockDim.x) {
    const int i = e % n, j = e / n;
    const double2 x = X[(size_t)i + (size_t)j * N];
    const float2 d = D[(size_t)i + (size_t)j * N];
    X[(size_t)i + (size_t)j * N] = make_double2(x.x - d.x, x.y - d.y);
  }
}

// Largest residual norm among the pairs that can be kept (the n_eig largest
// theta of problem t), over the whole block (every thread gets it).
__device__ double mx_worst_kept(const Batch& b, const MixedWs& w, int t, double* red) {
  const int kp = w.kp[t], K = b.neig[t];
  const double* th = w.theta + (size_t)t * w.KP;
  double worst = 0.0;
  for (int j = threadIdx.x; j < kp; j += blockDim.x) {
    const double tj = th[j];
    int rank = 0;
    for (int i = 0; i < kp; ++i) rank += (th[i] > tj) || (th[i] == tj && i < j);
    if (rank < K) worst = fmax(worst, w.rnorm[(size_t)t * w.KP + j]);
  }
  red[threadIdx.x] = worst;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}
// Early exit: a problem whose kept residuals are already below rtol ||C||_F
// skips the remaining passes (its X, theta and residuals stay as they are).
// One block of 128 threads per problem.
__global__ void k_mx_check(Batch b, MixedWs w, double rtol) {
  const int t = blockIdx.x;
  if (mx_skip(b.status, w.st2, t)) return;
  __shared__ double red[128];
  const double worst = mx_worst_kept(b, w, t, red);
  if (threadIdx.x == 0 && worst <= rtol * w.cnorm[t]) w.st2[t] |= kMxDone;
}
// Hand theta / X to the selection stage (which ranks b.mu and reads the
// columns of b.Q): mu[j] = theta[j] for j < kp, -inf beyond; check the last
// residuals of the n_eig leading pairs. One block of 128 threads per problem.
__global__ void k_mx_final(Batch b, MixedWs w, double rtol) {
  const int t = blockIdx.x;
  if (b.status[t]) return;
  const int n = b.nst[t], N = b.n_max, kp = w.kp[t];
  double* mu = b.mu + (size_t)t * N;
  for (int j = threadIdx.x; j < n; j += blockDim.x) mu[j] = (j < kp) ? w.theta[(size_t)t * w.KP + j] : -INFINITY;
  __shared__ double red[128];
  const double worst = mx_worst_kept(b, w, t, red);
  if (threadIdx.x == 0 && (!(worst <= rtol * w.cnorm[t]) || (w.st2[t] & ~kMxDone))) b.status[t] |= kStatusNotConverged;
}

template <bool CT>
void zgemm_df(const Batch& b, const MixedWs& w, int mc, int nc, int kc, int mmax, int nmax, const double2* A,
              size_t sa, int lda, const double2* B, size_t sb, int ldb, double2* out, size_t so, int ldo,
              cudaStream_t s, bool fp32 = false) {
  dim3 grd((mmax + GT - 1) / GT, (nmax + GT - 1) / GT, b.T);
  if (fp32)
    k_zgemm_f32<CT><<<grd, 256, 0, s>>>(b.nst, w.kp, mc, nc, kc, A, sa, lda, B, sb, ldb, out, so, ldo, b.status,
                                        w.st2);
  else
    k_zgemm_df<CT><<<grd, 256, 0, s>>>(b.nst, w.kp, mc, nc, kc, A, sa, lda, B, sb, ldb, out, so, ldo, b.status,
                                       w.st2);
}

}  // namespace

// The refinement's blocks must fit the Q buffer, and the kp x kp Cholesky of
// k_mx_cholinv its shared memory (kp <= 110: 195 KB).
// The FP32 stage keeps its reflectors, kp vectors and tridiagonal scratch in
// the X buffer (2 N^2 + 2 N kp + N^2 + 4 N + 1 floats of 4 N^2).
bool eig_mixed_fits(int N, int KP) {
  return KP <= 110 && 4LL * N * KP + 3LL * KP * KP <= (long long)N * N && N >= 2 * KP + 5;
}

void launch_eig_mixed(const Batch& b, const MixedWs& w, double tol, int max_sweeps, cudaStream_t s) {
  const int N = b.n_max, KP = w.KP, T = b.T;
  const size_t NN = (size_t)N * N;
  // 1. FP32 stage, in the X buffer of each problem (4 N^2 floats): C32 and then the
  //    reflectors in floats [0, 2N^2), the kp back-transformed vectors Q32 (N x KP
  //    complex) after them, then the tridiagonal scratch (Z_k in its first KP columns,
  //    d, e, tau). The inverse iteration's factors use the Q buffer, which the
  //    refinement takes over afterwards.
  float* Xf = reinterpret_cast<float*>(b.X);
  const size_t xs = 4 * NN;  // floats per problem in the X and Q buffers
  cudaMemsetAsync(w.st2, 0, sizeof(int) * T, s);
  TridiagArgs a;
  a.C = reinterpret_cast<float2*>(Xf);
  a.scratch = Xf + 2 * NN + 2 * (size_t)N * KP;
  a.sstride = xs;
  a.status = b.status;
  a.n = b.nst;
  a.ld = N;
  a.stride = 2 * NN;
  a.order = b.order;
  launch_tridiag32_reduce(a, T, s);
  float2* Q32 = reinterpret_cast<float2*>(Xf + 2 * NN);  // problem stride 2 N^2 float2, as C32
  SelArgs sa;
  sa.refl = a.C;
  sa.tds = a.scratch;
  sa.sstride = xs;
  sa.Z = a.scratch;
  sa.lam = w.lam;
  sa.lam_ld = N;
  sa.tnorm = w.tnorm;
  sa.n = b.nst;
  sa.neig = b.neig;
  sa.kp = w.kp;
  sa.pad = kPad;
  sa.status = b.status;
  sa.done = nullptr;
  sa.ld = N;
  sa.stride = 2 * NN;
  sa.order = b.order;
  const int sm2 = 2 * N * (int)sizeof(float);
  cudaFuncSetAttribute(k_td_topeig, cudaFuncAttributeMaxDynamicSharedMemorySize, sm2);
  k_td_topeig<<<T, kSelThreads, sm2, s>>>(sa);
  k_td_invit<<<T, kInvitThreads, sm2, s>>>(sa, reinterpret_cast<float*>(b.Q), xs, KP);
  launch_td_apply<false, true>(sa, Q32, 2 * NN, KP, T, s);  // Q32 = H Z_k
  // 2. FP64 refinement of the kp leading pairs; buffers inside the Q buffer
  double2* P0 = b.Q;                       // X (final eigenvectors), n x kp, ld N
  double2* P1 = b.Q + (size_t)N * KP;      // orthonormalised X / FP32 R and its correction
  double2* P2 = b.Q + (size_t)2 * N * KP;  // V L^{-T} X1, then Y U / R
  double2* P3 = b.Q + (size_t)3 * N * KP;  // L^{-T} X1, then Y = C X1, then the shifted solves' factors
  float2* R32 = reinterpret_cast<float2*>(P1);
  const size_t NN2 = 2 * NN;  // per-problem stride of the FP32 views
  double2* Hs = b.Q + (size_t)4 * N * KP;  // S, then H (kp x kp, ld KP)
  double2* Us = Hs + (size_t)KP * KP;      // rotations of H
  double2* Ws = Us + (size_t)KP * KP;      // R^{-1}
  k_mx_pick<<<T, 256, 0, s>>>(b, w, Q32, 2 * NN);
  JacobiArgs h;
  h.C = Hs;
  h.Q = Us;
  h.mu = w.theta;
  h.status = w.st2;
  h.sweeps = w.sw2;
  h.n = w.kp;
  h.ld = KP;
  h.stride = NN;
  h.report_nonconv = 1;
  h.order = b.order;
  // pass 0 diagonalises H in FP32: its eigenvectors need only the FP32 stage's accuracy
  // (the correction that follows is FP32); H and U in FP32 in the R^{-1} block, free by then
  JacobiArgs h32 = h;
  h32.C = reinterpret_cast<float2*>(Ws);
  h32.Q = reinterpret_cast<float2*>(Ws) + (size_t)KP * KP;
  h32.stride = 2 * NN;
  h32.report_nonconv = 0;
  SelArgs sr = sa;  // the refinement's corrections skip converged problems
  sr.done = w.st2;
  const int ew = std::max(1, (N * KP + 255) / 256 / 8);  // blocks per problem of the elementwise kernels
  const int ci_smem = (int)(sizeof(double2) * ((size_t)KP * KP + KP));
  cudaFuncSetAttribute(k_mx_cholinv, cudaFuncAttributeMaxDynamicSharedMemorySize, ci_smem);
  float* lu3 = reinterpret_cast<float*>(P3);  // the shifted solves' factors: Y (P3) is dead once Y U is formed
  const dim3 rgrd((N + GT - 1) / GT, (KP + GT - 1) / GT, T);
  for (int pass = 0; pass < kPasses; ++pass) {
    // pass 0 orthonormalises X and forms H to the FP32 stage's accuracy (FP32 products); the
    // residual's products (Y, X U, Y U) are double-float in every pass
    const bool lo = pass == 0;
    zgemm_df<true>(b, w, DKP, DKP, DN, KP, KP, P0, NN, N, P0, NN, N, Hs, NN, KP, s, lo);   // S = X^H X
    k_mx_cholinv<<<T, 256, ci_smem, s>>>(b, w, Hs, Ws, NN, KP);                                        // W = R^{-1}
    zgemm_df<false>(b, w, DN, DKP, DKP, N, KP, P0, NN, N, Ws, NN, KP, P1, NN, N, s, lo);  // X1 = X W
    // Y = C X1 = L^{-1} (V (L^{-T} X1)); Y lands in P3 and Y U in P2
    k_rgemm_df<true><<<rgrd, 256, 0, s>>>(b, w, P1, P3);                                          // L^{-T} X1
    zgemm_df<false>(b, w, DN, DKP, DN, N, KP, b.vis, NN, N, P3, NN, N, P2, NN, N, s);  // V (.)
    k_rgemm_df<false><<<rgrd, 256, 0, s>>>(b, w, P2, P3);                                         // Y
    zgemm_df<true>(b, w, DKP, DKP, DN, KP, KP, P1, NN, N, P3, NN, N, Hs, NN, KP, s, lo);  // H = X1^H Y
    k_mx_herm<<<T, 256, 0, s>>>(b, w, Hs, NN, KP);
    if (pass == 0) {                                                                              // H = U th U^H
      k_mx_cvt<true><<<T, 256, 0, s>>>(b, w, Hs, reinterpret_cast<float2*>(Ws), NN, KP);
      launch_jacobi_small_f32(h32, T, KP, 1e-6, 30, s);
      k_mx_cvt<false><<<T, 256, 0, s>>>(b, w, Us, reinterpret_cast<float2*>(Ws) + (size_t)KP * KP, NN, KP);
    } else {
      launch_jacobi_small(h, T, KP, 1e-13, 60, s);
    }
    zgemm_df<false>(b, w, DN, DKP, DKP, N, KP, P1, NN, N, Us, NN, KP, P0, NN, N, s);  // X = X1 U
    zgemm_df<false>(b, w, DN, DKP, DKP, N, KP, P3, NN, N, Us, NN, KP, P2, NN, N, s);  // Y U
    k_mx_resid<<<dim3(KP, T), 256, 0, s>>>(b, w, P0, P2, R32, NN);                                // R = YU - X th
    if (pass == kPasses - 1) break;
    k_mx_check<<<T, 128, 0, s>>>(b, w, 1e2 * tol);
    // correction in FP32: H P (T - theta_j)^{-1} P H^H r_j, P = I - Z_k Z_k^T
    launch_td_apply<true, false>(sr, R32, NN2, KP, T, s);                                   // S = H^H R
    k_td_deflate<<<dim3(KP, T), 256, KP * sizeof(float2), s>>>(sr, R32, NN2);
    k_td_shiftsolve<<<dim3((KP + 31) / 32, T), 32, sm2, s>>>(sr, R32, NN2, w.theta, w.KP, lu3, xs, KP);
    k_td_deflate<<<dim3(KP, T), 256, KP * sizeof(float2), s>>>(sr, R32, NN2);
    launch_td_apply<false, false>(sr, R32, NN2, KP, T, s);                                  // D = H U
    k_mx_sub<<<dim3(ew, T), 256, 0, s>>>(b, w, P0, R32, NN, NN2);                                 // X -= D
  }
  k_mx_final<<<T, 128, 0, s>>>(b, w, 1e3 * tol);
  (void)max_sweeps;
}

}  // namespace bipp
