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

#include "bipp_internal.cuh"
#include "jacobi.cuh"

namespace bipp {

namespace {

__device__ __forceinline__ size_t mat_off(int t, int n_max) { return (size_t)t * n_max * n_max; }

// ---------------------------------------------------------------- Gram

// G_ij = sinc(2 ||p_i - p_j|| / wl) with sinc(x) = sin(pi x)/(pi x) (Eq. gram, App. A).
__global__ void k_gram(Batch b, int gram_identity) {
  const int t = blockIdx.z;
  const int n = b.nst[t];
  const double wl = b.wl[t];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= n || j >= n) return;
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
}

// ---------------------------------------------------------------- Cholesky

// Right-looking Cholesky G = L L^T in place (lower triangle), one CTA per step.
__global__ void k_cholesky(Batch b) {
  const int t = blockIdx.x;
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

// L^{-1} by forward substitution, one thread per column j; stored row-major
// (Linv[i*N + j]) so that a warp's stores and loads are coalesced.
__global__ void k_trinv(Batch b, int gram_identity) {
  const int t = blockIdx.x;
  const int n = b.nst[t];
  const int N = b.n_max;
  const double* L = b.G + mat_off(t, N);
  double* R = b.Linv + mat_off(t, N);
  if (b.status[t]) return;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    for (int i = 0; i < n; ++i) {
      double x;
      if (gram_identity) {
        x = (i == j) ? 1.0 : 0.0;
      } else if (i < j) {
        x = 0.0;
      } else {
        double s = (i == j) ? 1.0 : 0.0;
        for (int k = j; k < i; ++k) s -= L[i + (size_t)k * N] * R[(size_t)k * N + j];
        x = s / L[i + (size_t)i * N];
      }
      R[(size_t)i * N + j] = x;
    }
  }
}

// ---------------------------------------------------------------- reduction C = L^{-1} V L^{-T}

constexpr int GT = 32;  // output tile
constexpr int GK = 16;  // k tile

// mode 0: X = Linv V           X(i,j) = sum_{k <= i} Linv(i,k) V(k,j)
// mode 1: C = X Linv^T         C(i,j) = sum_{k <= j} X(i,k) Linv(j,k)
template <int MODE>
__global__ void k_reduce_gemm(Batch b) {
  const int t = blockIdx.z;
  const int n = b.nst[t];
  const int N = b.n_max;
  if (b.status[t]) return;
  const int i0 = blockIdx.x * GT, j0 = blockIdx.y * GT;
  if (i0 >= n || j0 >= n) return;
  const double* Linv = b.Linv + mat_off(t, N);
  const double2* Z = (MODE == 0) ? (b.vis + mat_off(t, N)) : (b.X + mat_off(t, N));
  double2* out = (MODE == 0) ? (b.X + mat_off(t, N)) : (b.C + mat_off(t, N));
  __shared__ double sR[GK][GT + 1];
  __shared__ double2 sZ[GK][GT + 1];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 256 threads: 32 x 8
  double2 acc[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) acc[u] = make_double2(0.0, 0.0);
  // triangular structure: Linv(i,k) = 0 for k > i (mode 0), Linv(j,k) = 0 for k > j (mode 1)
  const int kend = min(n, (MODE == 0 ? i0 : j0) + GT);
  for (int k0 = 0; k0 < kend; k0 += GK) {
    for (int e = threadIdx.x; e < GK * GT; e += blockDim.x) {
      int kk = e / GT, ii = e % GT;
      int k = k0 + kk;
      if (MODE == 0) {
        int i = i0 + ii;
        sR[kk][ii] = (k < n && i < n) ? Linv[(size_t)i * N + k] : 0.0;
        int j = j0 + ii;
        sZ[kk][ii] = (k < n && j < n) ? Z[(size_t)k + (size_t)j * N] : make_double2(0.0, 0.0);
      } else {
        int i = i0 + ii;
        sZ[kk][ii] = (k < n && i < n) ? Z[(size_t)i + (size_t)k * N] : make_double2(0.0, 0.0);
        int j = j0 + ii;
        sR[kk][ii] = (k < n && j < n) ? Linv[(size_t)j * N + k] : 0.0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        int ii = tx, jj = ty + 8 * u;
        if (MODE == 0) {
          double r = sR[kk][ii];
          double2 z = sZ[kk][jj];
          acc[u].x = fma(r, z.x, acc[u].x);
          acc[u].y = fma(r, z.y, acc[u].y);
        } else {
          double2 z = sZ[kk][ii];
          double r = sR[kk][jj];
          acc[u].x = fma(z.x, r, acc[u].x);
          acc[u].y = fma(z.y, r, acc[u].y);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    int i = i0 + tx, j = j0 + ty + 8 * u;
    if (i < n && j < n) out[(size_t)i + (size_t)j * N] = acc[u];
  }
}

// C <- (C + C^H)/2 (or C <- Hermitian part of V when G = I): removes
// rounding-level asymmetry before the Jacobi sweeps.
__global__ void k_hermitize(Batch b, int from_vis) {
  const int t = blockIdx.z;
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
__global__ void k_select(Batch b, int n_level, const double* all_bounds, int filter) {
  const int t = blockIdx.x;
  const int n = b.nst[t];
  const int N = b.n_max;
  const int K = b.neig[t];
  const int KM = b.k_max;
  const double wl = b.wl[t];
  const double* bounds = all_bounds + (size_t)step_chan(b, t) * 2 * n_level;
  __shared__ int idx[kMaxEig];
  const int st = b.status[t];
  if (st) {
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
  for (int e = threadIdx.x; e < KM; e += blockDim.x) {
    int lev = -1;
    double m = 0.0, w = 0.0;
    if (e < K) {
      m = mu[idx[e]];
      w = (filter == 0) ? m : 1.0;
      for (int l = 0; l < n_level; ++l) {
        if (bounds[l] <= m && m < bounds[n_level + l]) {
          lev = l;
          break;
        }
      }
    }
    b.sel_mu[(size_t)t * KM + e] = m;
    b.wt[(size_t)t * KM + e] = w;
    b.level[(size_t)t * KM + e] = lev;
  }
  // a_e[i] = sum_{k >= i} Linv(k, i) q_{idx[e]}[k]
  const double* Linv = b.Linv + mat_off(t, N);
  const double2* Qm = b.Q + mat_off(t, N);
  for (int w = threadIdx.x; w < K * n; w += blockDim.x) {
    const int i = w % n, e = w / n;
    const double2* qc = Qm + (size_t)idx[e] * N;
    double2 a = make_double2(0.0, 0.0);
    for (int k = i; k < n; ++k) {
      const double r = Linv[(size_t)k * N + i];
      const double2 qk = qc[k];
      a.x = fma(r, qk.x, a.x);
      a.y = fma(r, qk.y, a.y);
    }
    b.W64[((size_t)t * KM + e) * N + i] = a;
    b.W32[((size_t)t * N + i) * KM + e] = make_float2((float)a.x, (float)a.y);
  }
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

}  // namespace

void launch_gram(const Batch& b, int gram_identity, cudaStream_t s) {
  dim3 blk(16, 16), grd((b.n_max + 15) / 16, (b.n_max + 15) / 16, b.T);
  k_gram<<<grd, blk, 0, s>>>(b, gram_identity);
}

void launch_cholesky(const Batch& b, int gram_identity, cudaStream_t s) {
  if (!gram_identity) k_cholesky<<<b.T, 256, 0, s>>>(b);
  k_trinv<<<b.T, 256, 0, s>>>(b, gram_identity);
}

void launch_reduce(const Batch& b, int gram_identity, cudaStream_t s) {
  dim3 hb(16, 16), hg((b.n_max + 15) / 16, (b.n_max + 15) / 16, b.T);
  if (gram_identity) {
    k_hermitize<<<hg, hb, 0, s>>>(b, 1);
    return;
  }
  dim3 grd((b.n_max + GT - 1) / GT, (b.n_max + GT - 1) / GT, b.T);
  k_reduce_gemm<0><<<grd, 256, 0, s>>>(b);
  k_reduce_gemm<1><<<grd, 256, 0, s>>>(b);
  k_hermitize<<<hg, hb, 0, s>>>(b, 0);
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
  launch_jacobi_args(a, b.T, false, tol, max_sweeps, s);
}

void launch_select(const Batch& b, int n_level, const double* d_bounds, int filter, cudaStream_t s) {
  k_select<<<b.T, 256, 0, s>>>(b, n_level, d_bounds, filter);
}

void launch_pixel_split(const double* d_xyz, float* d_hl, int64_t n, cudaStream_t s) {
  k_pixel_split<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d_xyz, d_hl, n);
}

}  // namespace bipp
