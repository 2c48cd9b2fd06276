// tridiag_sel.cuh — the leading eigenpairs of the real tridiagonal form of the
// reduced matrix, and the shift-and-invert preconditioner built on it, for the
// mixed-precision eigensolver (Sec. 2.3 keeps only the N_eig largest pairs of
// V a = mu G a, so only kp = n_eig + 16 of the n pairs are computed).
//
// After the Householder reduction C32 = H T H^H (tridiag32.cuh: T real
// symmetric with diagonal d and off-diagonal e, H = H_0 ... H_{n-2} stored as
// reflectors), per problem:
//   k_td_topeig   the kp largest eigenvalues of T by multisection of Sturm
//                 counts: one warp per eigenvalue, its 32 lanes count the
//                 eigenvalues below 32 points of the current interval, so each
//                 sweep narrows the interval 33-fold (FP32 accuracy in ~6 sweeps);
//   k_td_invit    their eigenvectors z_j by inverse iteration on T - lambda_j I
//                 (LU with partial pivoting, three solves), with modified
//                 Gram-Schmidt inside clusters of eigenvalues closer than
//                 1e-5 ||T||_F (the shifts of nearly equal eigenvalues are
//                 separated as in LAPACK's stein);
//   k_td_apply    q_j = H z_j (back-transformation of kp columns only), and, in
//                 the refinement, H or H^H applied to a complex n x kp block;
//   k_td_deflate  s <- s - Z_k (Z_k^T s): removes the kept directions;
//   k_td_shiftsolve u_j = (T - theta_j I)^{-1} s_j (complex right-hand sides).
// Together, H (T - theta I)^{-1} H^H restricted to the complement of the kept
// eigenvectors is the FP32 approximation of (C - theta I)^{-1} that the
// refinement uses as its correction (it equals Q32 (M32 - theta)^{-1} Q32^H on
// the complement of a full FP32 eigendecomposition, without forming Q32).
// All arithmetic is on T / ||T||_F, so that shifted pivots neither overflow nor
// underflow.
#pragma once

#include <math.h>

#include "bipp_internal.cuh"
#include "tridiag32.cuh"

namespace bipp {

constexpr int kSelThreads = 1024;  // k_td_topeig: 32 warps, one eigenvalue at a time each
constexpr float kSelOrtol = 1e-5f;  // cluster threshold (relative to ||T||_F) for Gram-Schmidt
constexpr float kSelEps = 5.96e-8f;  // 2^-24

struct SelArgs {
  const float2* refl;  // [T] reflectors in the Householder storage (ld, stride float2)
  const float* tds;    // [T] tridiagonal scratch (TridiagArgs layout: d, e, tau), sstride floats apart
  size_t sstride;
  float* Z;            // [T] kp tridiagonal eigenvectors, n x kp (ld), sstride apart (first kp columns of the scratch)
  float* lam;          // [T][lam_ld] kp leading eigenvalues of T / tnorm, descending
  int lam_ld;
  float* tnorm;        // [T] ||T||_F
  const int* n;        // [T]
  const int* neig;     // [T]
  int* kp;             // [T] min(n, neig + pad), written by k_td_topeig
  int pad;
  const int* status;   // [T] problems with a status bit are skipped
  const int* done;     // [T] or nullptr: refinement status (the refinement kernels also skip problems with the
                       //     early-exit bit kMxDoneBit or any error bit set)
  int ld;              // leading dimension N
  size_t stride;       // float2 elements between the problems' reflector blocks
  const int* order = nullptr;  // [T] problem of each block (Batch::order), or nullptr
};

constexpr int kMxDoneBit = 8;  // refinement status bit: kept residuals met the early-exit bound

namespace sel {

// The problem takes no part: an error status, or (in the refinement) done.
__device__ __forceinline__ bool skip(const SelArgs& a, int t) { return a.status[t] || (a.done && a.done[t]); }

// Eigenvalues of T below x (Sturm count of the LDL^T factorisation of T - x I).
__device__ __forceinline__ int sturm_count(int n, const float* d, const float* e2, float x, float pivmin) {
  float q = d[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  int c = q < 0.f;
  for (int i = 1; i < n; ++i) {
    q = (d[i] - x) - __fdividef(e2[i - 1], q);
    if (fabsf(q) < pivmin) q = -pivmin;
    c += q < 0.f;
  }
  return c;
}

// LU with partial pivoting of T - s I (rows i: sub e_{i-1}, diagonal d_i - s,
// super e_i), the factors at stride `st`: a (diagonal of U), b (first
// superdiagonal of U), m (multiplier), f (1.f: rows i and i+1 were swapped,
// and U then has e_{i+1} in its second superdiagonal at (i, i+2)).
__device__ __forceinline__ void lu(int n, const float* d, const float* e, float s, float* a_, float* b_, float* m_,
                                   float* f_, int st) {
  float a = d[0] - s;
  float b = (n > 1) ? e[0] : 0.f;
  for (int i = 0; i + 1 < n; ++i) {
    const float c = e[i], an = d[i + 1] - s, bn = (i + 2 < n) ? e[i + 1] : 0.f;
    if (fabsf(a) >= fabsf(c)) {
      const float m = (a != 0.f) ? c / a : 0.f;
      a_[(size_t)i * st] = a;
      b_[(size_t)i * st] = b;
      m_[(size_t)i * st] = m;
      f_[(size_t)i * st] = 0.f;
      a = an - m * b;
      b = bn;
    } else {
      const float m = a / c;
      a_[(size_t)i * st] = c;
      b_[(size_t)i * st] = an;
      m_[(size_t)i * st] = m;
      f_[(size_t)i * st] = 1.f;
      a = b - m * an;
      b = -m * bn;
    }
  }
  a_[(size_t)(n - 1) * st] = a;
  b_[(size_t)(n - 1) * st] = 0.f;
}

__device__ __forceinline__ float guard(float a, float tiny) {
  return (fabsf(a) < tiny) ? (a < 0.f ? -tiny : tiny) : a;
}

}  // namespace sel

// ---- kp largest eigenvalues of T by multisection. One CTA per problem.
// Dynamic shared memory: 2 * ld floats (d, e^2 of T / ||T||_F).
__global__ void __launch_bounds__(kSelThreads, 1) k_td_topeig(SelArgs a) {
  const int t = prob_of(a.order, blockIdx.x);
  if (a.status[t]) return;
  const int n = a.n[t], N = a.ld, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int kp = min(n, a.neig[t] + a.pad);
  const float* dg = a.tds + (size_t)t * a.sstride + td_off_d(N);
  const float* eg = a.tds + (size_t)t * a.sstride + td_off_e(N);
  extern __shared__ __align__(16) float selsm[];
  float* d = selsm;
  float* e2 = d + N;
  __shared__ float red[kSelThreads / 32];
  __shared__ float s_tn, s_gl, s_gu;
  float s2 = 0.f;
  for (int i = tid; i < n; i += kSelThreads) {
    const float di = dg[i], ei = (i + 1 < n) ? eg[i] : 0.f;
    s2 += di * di + 2.f * ei * ei;
  }
  for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  if (lane == 0) red[wid] = s2;
  __syncthreads();
  if (tid == 0) {
    float s = 0.f;
    for (int w = 0; w < kSelThreads / 32; ++w) s += red[w];
    s_tn = (s > 0.f) ? sqrtf(s) : 1.f;
    a.tnorm[t] = s_tn;
    a.kp[t] = kp;
  }
  __syncthreads();
  const float inv = 1.f / s_tn;
  float gl = INFINITY, gu = -INFINITY;
  for (int i = tid; i < n; i += kSelThreads) {
    const float di = dg[i] * inv, el = (i > 0) ? fabsf(eg[i - 1] * inv) : 0.f;
    const float er = (i + 1 < n) ? fabsf(eg[i] * inv) : 0.f;
    d[i] = di;
    e2[i] = (i + 1 < n) ? (eg[i] * inv) * (eg[i] * inv) : 0.f;
    gl = fminf(gl, di - el - er);
    gu = fmaxf(gu, di + el + er);
  }
  for (int o = 16; o > 0; o >>= 1) {
    gl = fminf(gl, __shfl_xor_sync(0xffffffffu, gl, o));
    gu = fmaxf(gu, __shfl_xor_sync(0xffffffffu, gu, o));
  }
  __syncthreads();
  if (lane == 0) red[wid] = gl;
  __syncthreads();
  if (tid == 0) {
    float g = INFINITY;
    for (int w = 0; w < kSelThreads / 32; ++w) g = fminf(g, red[w]);
    s_gl = g;
  }
  __syncthreads();
  if (lane == 0) red[wid] = gu;
  __syncthreads();
  if (tid == 0) {
    float g = -INFINITY;
    for (int w = 0; w < kSelThreads / 32; ++w) g = fmaxf(g, red[w]);
    s_gu = g;
  }
  __syncthreads();
  const float pivmin = 1e-30f;
  const float wid_ = fmaxf(fabsf(s_gl), fabsf(s_gu));
  const float glo = s_gl - 4.f * kSelEps * wid_ - pivmin, ghi = s_gu + 4.f * kSelEps * wid_ + pivmin;
  float* lam = a.lam + (size_t)t * a.lam_ld;
  for (int j = wid; j < kp; j += kSelThreads / 32) {
    const int m = n - 1 - j;  // ascending index of the j-th largest eigenvalue
    float lo = glo, hi = ghi;
    for (int sweep = 0; sweep < 12; ++sweep) {
      const float x = lo + (hi - lo) * ((float)(lane + 1) * (1.f / 33.f));
      const int c = sel::sturm_count(n, d, e2, x, pivmin);
      const unsigned above = __ballot_sync(0xffffffffu, c > m);  // lanes whose point lies above eigenvalue m
      const int f = __ffs(above);                                // first such lane (1-based), 0 if none
      const float xf = __shfl_sync(0xffffffffu, x, (f > 0) ? f - 1 : 0);
      const float xb = __shfl_sync(0xffffffffu, x, (f > 1) ? f - 2 : 31);
      if (f > 0) hi = xf;
      if (f != 1) lo = xb;
      if (hi - lo <= 2.f * kSelEps * fmaxf(fabsf(lo), fabsf(hi)) + 1e-9f) break;
    }
    if (lane == 0) lam[j] = 0.5f * (lo + hi);
  }
}

// ---- eigenvectors of T for the kp eigenvalues, by inverse iteration.
// One CTA of 128 threads per problem; thread v owns the cluster that starts at
// eigenvalue v (if one does) and computes its members in order, each from its
// own LU factors (scratch: 4 arrays of ld x lu_ld floats, interleaved by
// cluster, lu_stride floats per problem). Dynamic shared memory: 2 * ld floats.
constexpr int kInvitThreads = 128;

__global__ void __launch_bounds__(kInvitThreads) k_td_invit(SelArgs a, float* lu0, size_t lu_stride, int lu_ld) {
  const int t = prob_of(a.order, blockIdx.x);
  if (a.status[t]) return;
  const int n = a.n[t], N = a.ld, kp = a.kp[t], tid = threadIdx.x;
  const float* dg = a.tds + (size_t)t * a.sstride + td_off_d(N);
  const float* eg = a.tds + (size_t)t * a.sstride + td_off_e(N);
  float* Z = a.Z + (size_t)t * a.sstride;
  float* lam = a.lam + (size_t)t * a.lam_ld;
  extern __shared__ __align__(16) float ivsm[];
  float* d = ivsm;
  float* e = d + N;
  const float inv = 1.f / a.tnorm[t];
  for (int i = tid; i < n; i += kInvitThreads) {
    d[i] = dg[i] * inv;
    e[i] = (i + 1 < n) ? eg[i] * inv : 0.f;
  }
  // separate the shifts of (nearly) equal eigenvalues, descending order kept
  if (tid == 0) {
    for (int j = 1; j < kp; ++j) {
      const float pert = 10.f * kSelEps * fmaxf(fabsf(lam[j - 1]), 1e-6f);
      if (lam[j - 1] - lam[j] < pert) lam[j] = lam[j - 1] - pert;
    }
  }
  __syncthreads();
  const float tiny = kSelEps;  // pivot guard on the scale of ||T / ||T||_F|| = 1
  for (int v = tid; v < kp; v += kInvitThreads) {
    if (v > 0 && lam[v - 1] - lam[v] <= kSelOrtol) continue;  // not the first member of its cluster
    float* fa = lu0 + (size_t)t * lu_stride + v;
    float* fb = fa + (size_t)N * lu_ld;
    float* fm = fb + (size_t)N * lu_ld;
    float* ff = fm + (size_t)N * lu_ld;
    const int st = lu_ld;
    for (int j = v; j < kp && (j == v || lam[j - 1] - lam[j] <= kSelOrtol); ++j) {
      sel::lu(n, d, e, lam[j], fa, fb, fm, ff, st);
      float* z = Z + (size_t)j * N;
      // start vector: a fixed pseudo-random sequence in [-1, 1)
      unsigned h = 0x9e3779b9u * (unsigned)(j + 1);
      for (int i = 0; i < n; ++i) {
        h ^= h << 13;
        h ^= h >> 17;
        h ^= h << 5;
        z[i] = (float)(h >> 8) * (2.f / 16777216.f) - 1.f;
      }
      for (int it = 0; it < 3; ++it) {
        // forward: the row exchanges and eliminations of the factorisation
        float zi = z[0];
        for (int i = 0; i + 1 < n; ++i) {
          float zn = z[i + 1];
          if (ff[(size_t)i * st] != 0.f) {
            const float tmp = zi;
            zi = zn;
            zn = tmp;
          }
          z[i] = zi;
          zi = zn - fm[(size_t)i * st] * zi;
        }
        z[n - 1] = zi;
        // backward with U (second superdiagonal e_{i+1} where rows were swapped)
        float x2 = 0.f, x1 = z[n - 1] / sel::guard(fa[(size_t)(n - 1) * st], tiny);
        z[n - 1] = x1;
        float mx = fabsf(x1);
        for (int i = n - 2; i >= 0; --i) {
          const float u2 = (ff[(size_t)i * st] != 0.f) ? e[i + 1] : 0.f;
          const float xi = (z[i] - fb[(size_t)i * st] * x1 - u2 * x2) / sel::guard(fa[(size_t)i * st], tiny);
          z[i] = xi;
          x2 = x1;
          x1 = xi;
          mx = fmaxf(mx, fabsf(xi));
        }
        // scale, orthogonalise against the cluster's earlier members, normalise
        const float sc = (mx > 0.f) ? 1.f / mx : 1.f;
        for (int i = 0; i < n; ++i) z[i] *= sc;
        for (int k = v; k < j; ++k) {
          const float* zk = Z + (size_t)k * N;
          float dot = 0.f;
          for (int i = 0; i < n; ++i) dot = fmaf(zk[i], z[i], dot);
          for (int i = 0; i < n; ++i) z[i] = fmaf(-dot, zk[i], z[i]);
        }
        float nrm = 0.f;
        for (int i = 0; i < n; ++i) nrm = fmaf(z[i], z[i], nrm);
        const float ni = (nrm > 0.f) ? rsqrtf(nrm) : 0.f;
        for (int i = 0; i < n; ++i) z[i] *= ni;
      }
    }
  }
}

// ---- apply H (ADJ = false: Q <- H Q, reflectors n-2 .. 0) or H^H (ADJ = true:
// Q <- H^H Q, reflectors 0 .. n-2 with conj(tau)) to the first ncol[t]
// columns of a complex n x ncol block in place, reflectors staged RB at a time
// in shared memory, CPW columns in each warp's registers (lane l holds rows
// l, l + 32, ... of each), so that the CPW dot products of a reflector and
// their shuffle reductions overlap. FROM_Z: the block starts as the real
// columns of Z (k_td_apply then is the back-transformation q_j = H z_j).
// Grid (column groups of 16 CPW, T); dynamic shared memory: ld x (RB + 1) float2.
template <int RB, int RPL, bool ADJ, bool FROM_Z, int CPW>
__global__ void __launch_bounds__(kTdThreads, 1) k_td_apply(SelArgs a, float2* Q0, size_t qstride, int cols_per_cta) {
  using namespace td;
  const int t = prob_of(a.order, blockIdx.y);
  if (sel::skip(a, t)) return;
  const int n = a.n[t], N = a.ld, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int c0 = blockIdx.x * cols_per_cta;
  const int ncol = a.kp[t];
  if (c0 >= ncol) return;
  const int c1 = min(ncol, c0 + cols_per_cta);
  const float2* A = a.refl + (size_t)t * a.stride;
  float2* Q = Q0 + (size_t)t * qstride;
  const float2* tau = reinterpret_cast<const float2*>(a.tds + (size_t)t * a.sstride + td_off_tau(N));
  extern __shared__ __align__(16) unsigned char tasm_[];
  float2* V = reinterpret_cast<float2*>(tasm_);  // [row - (k0 + 1)][j], leading dimension RB + 1
  __shared__ float2 stau[RB];
  if (FROM_Z) {
    const float* Z = a.Z + (size_t)t * a.sstride;
    for (int e0 = tid; e0 < n * (c1 - c0); e0 += kTdThreads) {
      const int r = e0 % n, c = c0 + e0 / n;
      Q[(size_t)r + (size_t)c * N] = make_float2(Z[(size_t)r + (size_t)c * N], 0.f);
    }
  }
  const int nref = n - 1;  // reflectors 0 .. n-2
  const int nblk = (nref + RB - 1) / RB;
  const int cw = c0 + wid * CPW;  // this warp's first column
  for (int bi = 0; bi < nblk; ++bi) {
    const int k0 = ADJ ? bi * RB : (nblk - 1 - bi) * RB;
    const int nb = min(RB, nref - k0), mb = n - k0 - 1;  // reflectors k0..k0+nb-1 act on rows k0+1..n-1
    __syncthreads();
    for (int e0 = tid; e0 < mb * nb; e0 += kTdThreads) {
      const int r = e0 % mb, j = e0 / mb;
      float2 v = make_float2(0.f, 0.f);
      if (r == j) v = make_float2(1.f, 0.f);
      else if (r > j) v = A[(size_t)(k0 + 1 + r) + (size_t)(k0 + j) * N];
      V[(size_t)r * (RB + 1) + j] = v;
    }
    if (tid < nb) {
      const float2 tk = tau[k0 + tid];
      stau[tid] = ADJ ? make_float2(tk.x, -tk.y) : tk;
    }
    __syncthreads();
    if (cw >= c1) continue;
    const int nr = (mb + 31) >> 5;  // row slots in use (uniform): later blocks act on fewer rows
    float2 q[CPW][RPL];
#pragma unroll
    for (int k = 0; k < CPW; ++k) {
      const int c = min(cw + k, c1 - 1);  // a missing column repeats the last one, not stored
      const float2* Qc = Q + (size_t)(k0 + 1) + (size_t)c * N;
#pragma unroll
      for (int i = 0; i < RPL; ++i) {
        const int r = lane + 32 * i;
        q[k][i] = (r < mb) ? Qc[r] : make_float2(0.f, 0.f);
      }
    }
    for (int jj = 0; jj < nb; ++jj) {
      const int j = ADJ ? jj : nb - 1 - jj;
      const float2 tj = stau[j];
      float2 u[CPW];  // v^H q per column
#pragma unroll
      for (int k = 0; k < CPW; ++k) u[k] = make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < RPL; ++i) {
        if (i >= nr) break;
        const int r = lane + 32 * i;
        if (r < mb) {
          const float2 vr = V[(size_t)r * (RB + 1) + j];
#pragma unroll
          for (int k = 0; k < CPW; ++k) {
            u[k].x += vr.x * q[k][i].x + vr.y * q[k][i].y;
            u[k].y += vr.x * q[k][i].y - vr.y * q[k][i].x;
          }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < CPW; ++k) {
          u[k].x += __shfl_xor_sync(0xffffffffu, u[k].x, o);
          u[k].y += __shfl_xor_sync(0xffffffffu, u[k].y, o);
        }
      }
      float2 tu[CPW];
#pragma unroll
      for (int k = 0; k < CPW; ++k) tu[k] = cmul(tj, u[k]);
#pragma unroll
      for (int i = 0; i < RPL; ++i) {
        if (i >= nr) break;
        const int r = lane + 32 * i;
        if (r < mb) {
          const float2 vr = V[(size_t)r * (RB + 1) + j];
#pragma unroll
          for (int k = 0; k < CPW; ++k) {
            const float2 y = cmul(vr, tu[k]);
            q[k][i].x -= y.x;
            q[k][i].y -= y.y;
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < CPW; ++k) {
      if (cw + k >= c1) continue;
      float2* Qc = Q + (size_t)(k0 + 1) + (size_t)(cw + k) * N;
#pragma unroll
      for (int i = 0; i < RPL; ++i) {
        const int r = lane + 32 * i;
        if (r < mb) Qc[r] = q[k][i];
      }
    }
  }
}

// ---- s_j <- s_j - Z_k (Z_k^T s_j) for the first kp columns of a complex
// n x kp block (ld, qstride float2 per problem). Grid (kp_max, T), 256 threads;
// dynamic shared memory: kp_max float2.
__global__ void __launch_bounds__(256) k_td_deflate(SelArgs a, float2* S0, size_t qstride) {
  const int t = prob_of(a.order, blockIdx.y), j = blockIdx.x;
  if (sel::skip(a, t)) return;
  const int n = a.n[t], N = a.ld, kp = a.kp[t];
  if (j >= kp) return;
  const float* Z = a.Z + (size_t)t * a.sstride;
  float2* s = S0 + (size_t)t * qstride + (size_t)j * N;
  extern __shared__ __align__(16) float2 coef[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int m = wid; m < kp; m += 8) {
    const float* zm = Z + (size_t)m * N;
    float2 c = make_float2(0.f, 0.f);
    for (int i = lane; i < n; i += 32) {
      const float z = zm[i];
      const float2 x = s[i];
      c.x = fmaf(z, x.x, c.x);
      c.y = fmaf(z, x.y, c.y);
    }
    for (int o = 16; o > 0; o >>= 1) {
      c.x += __shfl_xor_sync(0xffffffffu, c.x, o);
      c.y += __shfl_xor_sync(0xffffffffu, c.y, o);
    }
    if (lane == 0) coef[m] = c;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += 256) {
    float2 x = s[i];
    for (int m = 0; m < kp; ++m) {
      const float z = Z[(size_t)i + (size_t)m * N];
      x.x = fmaf(-z, coef[m].x, x.x);
      x.y = fmaf(-z, coef[m].y, x.y);
    }
    s[i] = x;
  }
}

// ---- u_j = (T - theta_j I)^{-1} s_j in place for the first kp columns of a
// complex n x kp block (ld, qstride float2 per problem); theta in the units
// of C (FP64, KP apart per problem). One thread per column; the factors of
// each column (a, b, f: ld x lu_ld floats each, interleaved by column) in
// scratch lu_stride floats per problem. Grid (ceil(kp_max / 32), T), 32
// threads; dynamic shared memory: 2 * ld floats.
__global__ void __launch_bounds__(32) k_td_shiftsolve(SelArgs a, float2* S0, size_t qstride, const double* theta,
                                                    int theta_ld, float* lu0, size_t lu_stride, int lu_ld) {
  const int t = prob_of(a.order, blockIdx.y);
  if (sel::skip(a, t)) return;
  const int n = a.n[t], N = a.ld, kp = a.kp[t];
  const int j = blockIdx.x * 32 + threadIdx.x;
  const float* dg = a.tds + (size_t)t * a.sstride + td_off_d(N);
  const float* eg = a.tds + (size_t)t * a.sstride + td_off_e(N);
  extern __shared__ __align__(16) float sssm[];
  float* d = sssm;
  float* e = d + N;
  const float tn = a.tnorm[t], inv = 1.f / tn;
  for (int i = threadIdx.x; i < n; i += 32) {
    d[i] = dg[i] * inv;
    e[i] = (i + 1 < n) ? eg[i] * inv : 0.f;
  }
  __syncwarp();
  if (j >= kp) return;
  const float sft = (float)(theta[(size_t)t * theta_ld + j] / (double)tn);
  float* fa = lu0 + (size_t)t * lu_stride + j;
  float* fb = fa + (size_t)N * lu_ld;
  float* fm = fb + (size_t)N * lu_ld;
  float* ff = fm + (size_t)N * lu_ld;
  const int st = lu_ld;
  sel::lu(n, d, e, sft, fa, fb, fm, ff, st);
  float2* s = S0 + (size_t)t * qstride + (size_t)j * N;
  float2 si = s[0];
  for (int i = 0; i + 1 < n; ++i) {
    float2 sn = s[i + 1];
    if (ff[(size_t)i * st] != 0.f) {
      const float2 tmp = si;
      si = sn;
      sn = tmp;
    }
    s[i] = si;
    const float m = fm[(size_t)i * st];
    si = make_float2(sn.x - m * si.x, sn.y - m * si.y);
  }
  s[n - 1] = si;
  const float tiny = kSelEps;
  float2 x2 = make_float2(0.f, 0.f);
  float2 x1;
  {
    const float ia = 1.f / sel::guard(fa[(size_t)(n - 1) * st], tiny);
    const float2 y = s[n - 1];
    x1 = make_float2(y.x * ia, y.y * ia);
    s[n - 1] = x1;
  }
  for (int i = n - 2; i >= 0; --i) {
    const float u2 = (ff[(size_t)i * st] != 0.f) ? e[i + 1] : 0.f;
    const float b = fb[(size_t)i * st];
    const float ia = 1.f / sel::guard(fa[(size_t)i * st], tiny);
    const float2 y = s[i];
    const float2 xi = make_float2((y.x - b * x1.x - u2 * x2.x) * ia, (y.y - b * x1.y - u2 * x2.y) * ia);
    s[i] = xi;
    x2 = x1;
    x1 = xi;
  }
  // (T/tn - theta/tn)^{-1} = tn (T - theta)^{-1}: undo the scale
  for (int i = 0; i < n; ++i) {
    const float2 x = s[i];
    s[i] = make_float2(x.x * inv, x.y * inv);
  }
}

template <bool ADJ, bool FROM_Z>
inline void launch_td_apply(const SelArgs& a, float2* Q, size_t qstride, int KP, int T, cudaStream_t s) {
  const int N = a.ld;
  if (N <= 512) {
    constexpr int kCpw = 2, kCols = kTdThreads / 32 * kCpw;
    const dim3 grd((KP + kCols - 1) / kCols, T);
    const int smb = N * (32 + 1) * (int)sizeof(float2);
    cudaFuncSetAttribute(k_td_apply<32, 16, ADJ, FROM_Z, kCpw>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb);
    k_td_apply<32, 16, ADJ, FROM_Z, kCpw><<<grd, kTdThreads, smb, s>>>(a, Q, qstride, kCols);
  } else {
    constexpr int kCols = kTdThreads / 32;
    const dim3 grd((KP + kCols - 1) / kCols, T);
    const int smb = N * (16 + 1) * (int)sizeof(float2);
    cudaFuncSetAttribute(k_td_apply<16, 32, ADJ, FROM_Z, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smb);
    k_td_apply<16, 32, ADJ, FROM_Z, 1><<<grd, kTdThreads, smb, s>>>(a, Q, qstride, kCols);
  }
}

}  // namespace bipp
