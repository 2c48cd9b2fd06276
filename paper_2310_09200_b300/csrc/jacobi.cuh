// jacobi.cuh — parallel-order complex Jacobi for batched Hermitian matrices,
// generic over the element precision (FP64 for the eigensolve proper, FP32
// for the preconditioning sweeps of the mixed-precision eigensolver).
#pragma once

#include <math.h>

#include "bipp_internal.cuh"

namespace bipp {

template <typename R>
struct CplxOf;
template <>
struct CplxOf<double> {
  using T = double2;
  static __device__ __forceinline__ double2 make(double x, double y) { return make_double2(x, y); }
};
template <>
struct CplxOf<float> {
  using T = float2;
  static __device__ __forceinline__ float2 make(float x, float y) { return make_float2(x, y); }
};

// Operands of one batched Jacobi launch. Problem t: n[t] x n[t] matrix at
// C + t*stride (column-major, leading dimension ld), rotations at Q + t*stride,
// eigenvalues (the final diagonal, unsorted) at mu + t*ld.
struct JacobiArgs {
  void* C;
  void* Q;
  double* mu;
  int* status;       // [T] problems with a status bit set are skipped
  int* sweeps;       // [T] sweeps used
  const int* n;      // [T]
  int ld;
  size_t stride;
  int report_nonconv;  // set kStatusNotConverged when the sweep cap is hit
  const int* order = nullptr;  // [T] problem of each block (Batch::order), or nullptr
};

namespace jac {

template <typename C2, typename R>
__device__ __forceinline__ C2 mul(C2 a, C2 b) {
  return CplxOf<R>::make(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
template <typename C2, typename R>
__device__ __forceinline__ C2 mulc(C2 a, C2 b) {  // a * conj(b)
  return CplxOf<R>::make(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
template <typename C2, typename R>
__device__ __forceinline__ C2 scale(C2 a, R s) { return CplxOf<R>::make(a.x * s, a.y * s); }
template <typename C2, typename R>
__device__ __forceinline__ C2 add(C2 a, C2 b) { return CplxOf<R>::make(a.x + b.x, a.y + b.y); }
template <typename C2, typename R>
__device__ __forceinline__ C2 sub(C2 a, C2 b) { return CplxOf<R>::make(a.x - b.x, a.y - b.y); }

// Round-robin ("circle method") pairing of m (even) indices: in round r the
// pairs are (m-1, r) and ((r+k) mod (m-1), (r-k) mod (m-1)) for k = 1..m/2-1.
// Every pair meets exactly once in m-1 rounds, and the m/2 pairs of a round
// are disjoint, so their rotations commute and are applied together.
__device__ __forceinline__ void rr_pair(int r, int k, int m, int* p, int* q) {
  int a, bb;
  if (k == 0) {
    a = m - 1;
    bb = r;
  } else {
    a = (r + k) % (m - 1);
    bb = (r - k + (m - 1)) % (m - 1);
  }
  *p = min(a, bb);
  *q = max(a, bb);
}

}  // namespace jac

constexpr int kJacobiThreads = 512;

// For pivot (p,q), a = C_pp, b = C_qq, C_pq = r e^{i phi}, the rotation
//   J = [[c, sigma], [-conj(sigma), c]],  sigma = s e^{i phi},
// with (c, s) the symmetric Schur rotation of [[a, r], [r, b]] zeroes C_pq
// (Golub & Van Loan Sec. 8.5 carried over to the Hermitian case). A round
// applies the m/2 disjoint rotations: C <- J^H C J on every 2x2 block, with
// only the blocks on or above the diagonal computed and the ones below
// written as their conjugate transposes, and Q <- Q J. For odd n a phantom
// index n pairs with one real index per round (identity rotation).
// CSM: C is staged in dynamic shared memory (leading dimension n) for the
// sweeps, for small matrices whose scattered 2x2 accesses would otherwise
// wait on L2 every round; only its diagonal goes back (mu), Q stays in place.
template <typename R, bool CSM = false>
__global__ void __launch_bounds__(kJacobiThreads) k_jacobi_t(JacobiArgs a, double tol, int max_sweeps) {
  using C2 = typename CplxOf<R>::T;
  using namespace jac;
  const int t = prob_of(a.order, blockIdx.x);
  const int n = a.n[t];
  if (a.status[t]) return;
  C2* Q = static_cast<C2*>(a.Q) + (size_t)t * a.stride;
  const int NQ = a.ld;  // leading dimension of Q (and of C in global memory)
  C2* C = static_cast<C2*>(a.C) + (size_t)t * a.stride;
  int N = a.ld;         // leading dimension of C where the sweeps run
  if constexpr (CSM) {
    extern __shared__ __align__(16) unsigned char jsm[];
    C2* Cs = reinterpret_cast<C2*>(jsm);
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) Cs[e] = C[(size_t)(e % n) + (size_t)(e / n) * a.ld];
    C = Cs;
    N = n;
    __syncthreads();
  }
  const int m = n + (n & 1);
  const int np = m / 2;

  __shared__ int sp[kMaxStations / 2], sq[kMaxStations / 2];
  __shared__ R sc[kMaxStations / 2];
  __shared__ C2 ssig[kMaxStations / 2];
  __shared__ R sdiag_p[kMaxStations / 2], sdiag_q[kMaxStations / 2];
  __shared__ double red[kJacobiThreads / 32];
  __shared__ double s_fro, s_off;

  double fro = 0.0;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e % n, j = e / n;
    Q[(size_t)i + (size_t)j * NQ] = CplxOf<R>::make(i == j ? R(1) : R(0), R(0));
    const C2 v = C[(size_t)i + (size_t)j * N];
    fro += (double)v.x * v.x + (double)v.y * v.y;
  }
  auto block_sum = [&](double v) -> double {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
      s = (threadIdx.x < (int)(blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    __syncthreads();
    return s;  // valid in warp 0
  };
  fro = block_sum(fro);
  if (threadIdx.x == 0) s_fro = sqrt(fro);
  __syncthreads();
  const double thresh = tol * s_fro;

  int sweep = 0;
  bool converged = false;
  for (;;) {
    double off = 0.0;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int i = e % n, j = e / n;
      if (i != j) {
        const C2 v = C[(size_t)i + (size_t)j * N];
        off += (double)v.x * v.x + (double)v.y * v.y;
      }
    }
    off = block_sum(off);
    if (threadIdx.x == 0) s_off = sqrt(off);
    __syncthreads();
    if (s_off <= thresh || s_fro == 0.0) {
      converged = true;
      break;
    }
    if (sweep >= max_sweeps) break;
    ++sweep;
    for (int r = 0; r < m - 1; ++r) {
      for (int k = threadIdx.x; k < np; k += blockDim.x) {
        int p, q;
        rr_pair(r, k, m, &p, &q);
        sp[k] = p;
        sq[k] = q;
        R c = R(1);
        C2 sig = CplxOf<R>::make(R(0), R(0));
        R dp = C[(size_t)p + (size_t)p * N].x, dq = R(0);  // p < n always
        if (q < n) {
          const R aa = dp;
          const R bq = C[(size_t)q + (size_t)q * N].x;
          const C2 x = C[(size_t)p + (size_t)q * N];
          const R rr = hypot(x.x, x.y);
          dq = bq;
          if (rr > R(0)) {
            const R tau = (bq - aa) / (R(2) * rr);
            const R tt = (tau >= R(0) ? R(1) : R(-1)) / (fabs(tau) + hypot(R(1), tau));
            c = R(1) / sqrt(R(1) + tt * tt);
            const R s = tt * c;
            sig = CplxOf<R>::make(s * x.x / rr, s * x.y / rr);
            dp = aa - tt * rr;
            dq = bq + tt * rr;
          }
        }
        sc[k] = c;
        ssig[k] = sig;
        sdiag_p[k] = dp;
        sdiag_q[k] = dq;
      }
      __syncthreads();
      // C <- J^H C J on the 2x2 blocks (k1 <= k2); the (k2, k1) block is the
      // conjugate transpose of the (k1, k2) block.
      const int nblk = np * (np + 1) / 2;
      for (int e = threadIdx.x; e < nblk; e += blockDim.x) {
        // e -> (k1, k2), k1 <= k2, row-major over the upper triangle
        const float b2 = 2.0f * np + 1.0f;
        int k1 = (int)((b2 - sqrtf(fmaxf(b2 * b2 - 8.0f * e, 0.0f))) * 0.5f);
        k1 = min(max(k1, 0), np - 1);
        while (k1 > 0 && k1 * (2 * np - k1 + 1) / 2 > e) --k1;
        while ((k1 + 1) * (2 * np - k1) / 2 <= e) ++k1;
        const int k2 = k1 + (e - k1 * (2 * np - k1 + 1) / 2);
        const int p1 = sp[k1], q1 = sq[k1], p2 = sp[k2], q2 = sq[k2];
        const bool v1 = q1 < n, v2 = q2 < n;
        if (k1 == k2) {
          C[(size_t)p1 + (size_t)p1 * N] = CplxOf<R>::make(sdiag_p[k1], R(0));
          if (v1) {
            C[(size_t)q1 + (size_t)q1 * N] = CplxOf<R>::make(sdiag_q[k1], R(0));
            C[(size_t)p1 + (size_t)q1 * N] = CplxOf<R>::make(R(0), R(0));
            C[(size_t)q1 + (size_t)p1 * N] = CplxOf<R>::make(R(0), R(0));
          }
          continue;
        }
        const R c1 = sc[k1], c2 = sc[k2];
        const C2 g1 = ssig[k1], g2 = ssig[k2];
        const C2 zero = CplxOf<R>::make(R(0), R(0));
        const C2 x11 = C[(size_t)p1 + (size_t)p2 * N];
        const C2 x12 = v2 ? C[(size_t)p1 + (size_t)q2 * N] : zero;
        const C2 x21 = v1 ? C[(size_t)q1 + (size_t)p2 * N] : zero;
        const C2 x22 = (v1 && v2) ? C[(size_t)q1 + (size_t)q2 * N] : zero;
        // Y = X J2: col p2 -> c2 x_p2 - conj(g2) x_q2 ; col q2 -> g2 x_p2 + c2 x_q2
        const C2 y11 = sub<C2, R>(scale<C2, R>(x11, c2), mulc<C2, R>(x12, g2));
        const C2 y12 = add<C2, R>(mul<C2, R>(x11, g2), scale<C2, R>(x12, c2));
        const C2 y21 = sub<C2, R>(scale<C2, R>(x21, c2), mulc<C2, R>(x22, g2));
        const C2 y22 = add<C2, R>(mul<C2, R>(x21, g2), scale<C2, R>(x22, c2));
        // Z = J1^H Y: row p1 -> c1 y_p1 - g1 y_q1 ; row q1 -> conj(g1) y_p1 + c1 y_q1
        const C2 z11 = sub<C2, R>(scale<C2, R>(y11, c1), mul<C2, R>(g1, y21));
        const C2 z12 = sub<C2, R>(scale<C2, R>(y12, c1), mul<C2, R>(g1, y22));
        const C2 g1c = CplxOf<R>::make(g1.x, -g1.y);
        const C2 z21 = add<C2, R>(mul<C2, R>(g1c, y11), scale<C2, R>(y21, c1));
        const C2 z22 = add<C2, R>(mul<C2, R>(g1c, y12), scale<C2, R>(y22, c1));
        C[(size_t)p1 + (size_t)p2 * N] = z11;
        C[(size_t)p2 + (size_t)p1 * N] = CplxOf<R>::make(z11.x, -z11.y);
        if (v2) {
          C[(size_t)p1 + (size_t)q2 * N] = z12;
          C[(size_t)q2 + (size_t)p1 * N] = CplxOf<R>::make(z12.x, -z12.y);
        }
        if (v1) {
          C[(size_t)q1 + (size_t)p2 * N] = z21;
          C[(size_t)p2 + (size_t)q1 * N] = CplxOf<R>::make(z21.x, -z21.y);
        }
        if (v1 && v2) {
          C[(size_t)q1 + (size_t)q2 * N] = z22;
          C[(size_t)q2 + (size_t)q1 * N] = CplxOf<R>::make(z22.x, -z22.y);
        }
      }
      // Q <- Q J on every row and pair
      for (int e = threadIdx.x; e < n * np; e += blockDim.x) {
        const int i = e % n, k = e / n;
        const int p = sp[k], q = sq[k];
        if (q >= n) continue;
        const R c = sc[k];
        const C2 g = ssig[k];
        const C2 aq = Q[(size_t)i + (size_t)p * NQ];
        const C2 bq = Q[(size_t)i + (size_t)q * NQ];
        Q[(size_t)i + (size_t)p * NQ] = sub<C2, R>(scale<C2, R>(aq, c), mulc<C2, R>(bq, g));
        Q[(size_t)i + (size_t)q * NQ] = add<C2, R>(mul<C2, R>(aq, g), scale<C2, R>(bq, c));
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) a.mu[(size_t)t * NQ + i] = (double)C[(size_t)i + (size_t)i * N].x;
  if (threadIdx.x == 0) {
    a.sweeps[t] = sweep;
    if (!converged && a.report_nonconv) a.status[t] |= kStatusNotConverged;
  }
}

inline void launch_jacobi_args(const JacobiArgs& a, int T, bool fp32, double tol, int max_sweeps, cudaStream_t s) {
  if (fp32) k_jacobi_t<float><<<T, kJacobiThreads, 0, s>>>(a, tol, max_sweeps);
  else k_jacobi_t<double><<<T, kJacobiThreads, 0, s>>>(a, tol, max_sweeps);
}

// FP64 Jacobi of matrices of at most n_max rows with C staged in shared
// memory when it fits (n_max^2 complex doubles beside the static arrays).
inline void launch_jacobi_small(const JacobiArgs& a, int T, int n_max, double tol, int max_sweeps, cudaStream_t s) {
  const size_t smem = sizeof(double2) * (size_t)n_max * n_max;
  if (smem <= 160 * 1024) {
    cudaFuncSetAttribute(k_jacobi_t<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_jacobi_t<double, true><<<T, kJacobiThreads, smem, s>>>(a, tol, max_sweeps);
  } else {
    k_jacobi_t<double><<<T, kJacobiThreads, 0, s>>>(a, tol, max_sweeps);
  }
}

// The same in FP32 (float2 C and Q, FP64 eigenvalues out).
inline void launch_jacobi_small_f32(const JacobiArgs& a, int T, int n_max, double tol, int max_sweeps,
                                    cudaStream_t s) {
  const size_t smem = sizeof(float2) * (size_t)n_max * n_max;
  if (smem <= 160 * 1024) {
    cudaFuncSetAttribute(k_jacobi_t<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_jacobi_t<float, true><<<T, kJacobiThreads, smem, s>>>(a, tol, max_sweeps);
  } else {
    k_jacobi_t<float><<<T, kJacobiThreads, 0, s>>>(a, tol, max_sweeps);
  }
}

}  // namespace bipp
