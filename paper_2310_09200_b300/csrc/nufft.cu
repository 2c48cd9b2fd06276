// nufft.cu — NUFFT synthesis (Sec. 2.5, Sec. 3.4, Algorithm 3) on B300.
//
// Per channel of a batch (steps [t0, t1) with one wavelength), one type-3
// NUFFT per level maps the baselines of all steps to the pixels:
//
//   1. Spreading onto the grid y_m = (m - M/2) h with the exponential-of-
//      semicircle kernel, the baselines sorted by the grid cell where their
//      w^3-cell footprint starts (a counting sort), so that runs of baselines
//      with the same start are summed in registers and added to the grid once:
//      k_nu_count   one thread per station pair p < q of a step: orientation
//                   (the folded coordinate >= 0; the (q, p) term is the
//                   conjugate one, so Re of the sum is unchanged), input cell
//                   (domain partitioning), spread start; warp-aggregated count
//                   per sort key;
//      k_nu_seg_sum, k_nu_scan, k_nu_seg_scan  exclusive offsets of the keys;
//      k_nu_scatter per pair, the level strengths 2 V'_l,pq = 2 sum_{e in l}
//                   d_e a_pe conj(a_qe) (eigenvectors staged through shared
//                   memory), pre-phased by exp(2 pi i <D, x>), written with the
//                   start and fractions at the pair's sorted place;
//      k_nu_spread  one warp per 256 sorted baselines: lane i owns footprint
//                   cells i, i + 32, ...; runs of equal start cells are summed
//                   in registers and added with vector float atomics.
//      Coordinates and phases are reduced in FP64; kernel weights, strengths and
//      the grid are FP32.
//   2. k_nu_const: the p = q terms (zero baseline): sum_t sum_{e in l} d_e |a_e|^2,
//      a constant per level.
//   3. per level: k_nu_pad divides each grid mode by the second kernel's
//      transform and places it into the twice finer grid; cuFFT's backward
//      C2C transforms evaluate the Fourier series there, pruned: 2-D (x, y)
//      transforms of the M_z planes that hold modes, then the transforms
//      along z out of place, so the other M_z planes stay zero and are never
//      rewritten;
//      k_nu_interp interpolates it at t = (s - D) h with the kernel, applies
//      the trapezoid factor, the diagonal correction 1 / psi_hat(s - D) and
//      the post-phase exp(2 pi i <s - D, C>), and adds Re + the constant to
//      the level image.
//
// The kernel and grid rules are those of the exponential-of-semicircle NUFFT
// (Barnett, Magland and af Klinteberg, SIAM J. Sci. Comput. 41, 2019):
// w = ceil(log10(1/eps)) + 1, beta = 2.30 w, upsampling 2; spacing
// h = pi / (2 S) so the spread function's spectrum aliases only beyond the
// kernel's pass band, and M = 8 X S + w + 2 points (X, S half-widths in cycles
// and direction units) rounded up to an even 2^a 3^b 5^c.
#include <math.h>

#include <algorithm>
#include <vector>

#include "nufft.cuh"

namespace bipp {

namespace {

constexpr double kSigma = 2.0;

__device__ __forceinline__ float es_w(float z, float beta) {
  const float q = 1.0f - z * z;
  return q >= 0.0f ? expf(beta * (sqrtf(q) - 1.0f)) : 0.0f;
}

// Least even integer >= n with prime factors 2, 3, 5 only.
long long next_smooth(long long n) {
  for (long long m = std::max(2LL, n);; ++m) {
    if (m & 1) continue;
    long long r = m;
    for (int p : {2, 3, 5})
      while (r % p == 0) r /= p;
    if (r == 1) return m;
  }
}

// Gauss-Legendre rule of 2 kNuGL points on [-1, 1] (Newton's method on the
// Legendre recurrence); the kNuGL positive nodes and their weights.
void gauss_legendre_half(double* z, double* wq) {
  const int n = 2 * kNuGL;
  for (int i = 0; i < kNuGL; ++i) {
    double x = cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (x * p1 - p0) / (x * x - 1.0);
      const double dx = p1 / dp;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    z[i] = x;
    wq[i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
}

double phi_host(double z, double beta) {
  const double q = 1.0 - z * z;
  return q >= 0.0 ? exp(beta * (sqrt(q) - 1.0)) : 0.0;
}

// psi_hat(xi) = alpha * int_{-1}^{1} phi(z) cos(alpha xi z) dz for the kernel psi(y) = phi(y / alpha).
double es_ft_host(double xi, double alpha, double beta, const double* z, const double* wq) {
  double s = 0.0;
  for (int q = 0; q < kNuGL; ++q) s += wq[q] * phi_host(z[q], beta) * cos(alpha * xi * z[q]);
  return 2.0 * alpha * s;
}

struct SpreadArgs {
  int M[3];
  double invH[3], D[3];
  int P[3];                // input cells per dimension
  double lo[3], delta[3];  // input box corner and cell size
  double idelta[3];        // 1 / delta (0 for a single cell)
  long long cells;         // grid points of one input cell's grid
  int fold, w, L, Lp;
  float beta;
};

// Oriented coordinates, input cell, spread start m0 (inside the cell's grid) and
// fraction m0 - g of the pair (p, q) of step t.
struct PairGeo {
  double x[3];
  int m0[3];
  float fr[3];
  int pid;
  bool flip;
};

__device__ __forceinline__ PairGeo pair_geo(const Batch& b, int t, int p, int q, const SpreadArgs& a) {
  PairGeo g;
  const int N = b.n_max;
  const double* st = b.st + (size_t)t * 3 * N;
  const double iwl = 1.0 / b.wl[t];
#pragma unroll
  for (int d = 0; d < 3; ++d) g.x[d] = -(st[(size_t)d * N + p] - st[(size_t)d * N + q]) * iwl;
  const double xf = a.fold == 0 ? g.x[0] : (a.fold == 1 ? g.x[1] : g.x[2]);
  g.flip = xf < 0.0;
  if (g.flip) {
#pragma unroll
    for (int d = 0; d < 3; ++d) g.x[d] = -g.x[d];
  }
  int ci[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    int c = a.P[d] > 1 ? (int)floor((g.x[d] - a.lo[d]) * a.idelta[d]) : 0;
    c = min(max(c, 0), a.P[d] - 1);
    ci[d] = c;
    const double C = a.lo[d] + (c + 0.5) * a.delta[d];
    const double gg = (g.x[d] - C) * a.invH[d] + 0.5 * a.M[d];
    int m = (int)ceil(gg - 0.5 * a.w);
    m = min(max(m, 0), a.M[d] - a.w);  // never outside the grid (the plan's margin makes this a no-op)
    g.m0[d] = m;
    g.fr[d] = (float)((double)m - gg);
  }
  g.pid = (ci[2] * a.P[1] + ci[1]) * a.P[0] + ci[0];
  return g;
}

// Sort key of a point: its input cell, then the grid cell of its spread start.
__device__ __forceinline__ int cell_of(const PairGeo& g, const SpreadArgs& a) {
  return (int)(g.pid * a.cells + ((long long)g.m0[2] * a.M[1] + g.m0[1]) * a.M[0] + g.m0[0]);
}

// Pair index r -> (p, q), p < q, r = q (q - 1) / 2 + p.
__device__ __forceinline__ void tri_pair(long long r, int* p, int* q) {
  long long qq = (long long)((1.0 + sqrt(8.0 * (double)r + 1.0)) * 0.5);
  while (qq * (qq - 1) / 2 > r) --qq;
  while ((qq + 1) * qq / 2 <= r) ++qq;
  *q = (int)qq;
  *p = (int)(r - qq * (qq - 1) / 2);
}

// Upper-triangle tile (pb <= qb) of linear index r, tiles ordered by qb.
__device__ __forceinline__ void tri_tile(int r, int* pb, int* qb) {
  int q = (int)((sqrt(8.0 * r + 1.0) - 1.0) * 0.5);
  while (q * (q + 1) / 2 > r) --q;
  while ((q + 1) * (q + 2) / 2 <= r) ++q;
  *qb = q;
  *pb = r - q * (q + 1) / 2;
}

// Warp-aggregated counter increment: the lanes of `active` add 1 each to ctr[key];
// returns the counter's value before this lane's increment.
__device__ __forceinline__ int agg_add(int* ctr, int key, unsigned active) {
  const unsigned grp = __match_any_sync(active, key);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(grp) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(ctr + key, __popc(grp));
  base = __shfl_sync(grp, base, leader);
  return base + __popc(grp & ((1u << lane) - 1u));
}

// 1. Points per start cell: one thread per pair slot (t, p < q) of the steps [t0, t0 + T).
__global__ void k_nu_count(Batch b, int t0, int T, SpreadArgs a, int* __restrict__ count) {
  const long long NP = (long long)b.n_max * (b.n_max - 1) / 2;
  const long long total = NP * T;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < total; base += (long long)gridDim.x * blockDim.x) {
    const long long sl = base + threadIdx.x;
    bool active = false;
    int t = 0, p = 0, q = 0;
    if (sl < total) {
      t = t0 + (int)(sl / NP);
      tri_pair(sl % NP, &p, &q);
      active = q < b.nst[t] && b.nkept[t] > 0;
    }
    const unsigned am = __ballot_sync(0xffffffffu, active);
    if (active) {
      const PairGeo g = pair_geo(b, t, p, q, a);
      agg_add(count, cell_of(g, a), am);
    }
  }
}

// Exclusive scan out[0..n] of in (out[n] = total) in one block of 1024 threads.
__global__ void __launch_bounds__(1024) k_nu_scan(const int* __restrict__ in, int n, int* __restrict__ out) {
  __shared__ int part[1024];
  const int per = (n + 1023) / 1024;
  const int i0 = min(n, threadIdx.x * per), i1 = min(n, i0 + per);
  int sum = 0;
  for (int i = i0; i < i1; ++i) sum += in[i];
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {  // inclusive Hillis-Steele scan of the partial sums
    const int v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = part[threadIdx.x] - sum;
  for (int i = i0; i < i1; ++i) {
    out[i] = run;
    run += in[i];
  }
  if (threadIdx.x == 1023) out[n] = part[1023];
}

// Exclusive scan of n ints over many blocks: segments of kSeg elements per
// block; k_nu_seg_sum totals each segment, k_nu_scan scans the totals,
// k_nu_seg_scan writes out[i] (and out[n] = total).
constexpr int kSeg = 8192;

__global__ void __launch_bounds__(1024) k_nu_seg_sum(const int* __restrict__ in, long long n, int* __restrict__ sums) {
  __shared__ int red[32];
  const long long i0 = (long long)blockIdx.x * kSeg + threadIdx.x * 8;
  int v = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (i0 + k < n) v += in[i0 + k];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    int u = red[threadIdx.x];
    for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
    if (threadIdx.x == 0) sums[blockIdx.x] = u;
  }
}

__global__ void __launch_bounds__(1024) k_nu_seg_scan(const int* __restrict__ in, long long n,
                                                      const int* __restrict__ seg_off, int* __restrict__ out) {
  __shared__ int wsum[32];
  const long long i0 = (long long)blockIdx.x * kSeg + threadIdx.x * 8;
  int v[8], tot = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    v[k] = i0 + k < n ? in[i0 + k] : 0;
    tot += v[k];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int inc = tot;  // inclusive warp scan of the thread totals
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int x = wsum[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += u;
    }
    wsum[lane] = x;  // inclusive over warps
  }
  __syncthreads();
  int run = seg_off[blockIdx.x] + (warp > 0 ? wsum[warp - 1] : 0) + inc - tot;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (i0 + k < n) out[i0 + k] = run;
    run += v[k];
  }
  if (i0 <= n - 1 && n - 1 < i0 + 8) out[n] = run;  // the thread holding the last element writes the total
}

constexpr int kTile = 16;
constexpr int kEChunk = 64;
constexpr int kNuRun = 256;  // sorted points per spreading warp

// 2. Level strengths, orientation and pre-phase of every pair, written in start-cell
// order: rm = (m0, cell), rf = (fractions), rc = Lp strengths (pair-major).
template <int MAXL>
__global__ void __launch_bounds__(kTile* kTile)
    k_nu_scatter(Batch b, int t0, SpreadArgs a, const int* __restrict__ cell_off, int* __restrict__ cursor,
                 int4* __restrict__ rm, float4* __restrict__ rf, float2* __restrict__ rc) {
  const int t = t0 + blockIdx.z;
  const int n = b.nst[t];
  const int K = b.nkept[t];
  if (K <= 0) return;  // failed step: nothing kept (the batch flag stops the image update)
  int pb, qb;
  tri_tile(blockIdx.x, &pb, &qb);
  if (qb * kTile >= n) return;
  const int tx = threadIdx.x & (kTile - 1), ty = threadIdx.x / kTile;
  const int p = pb * kTile + ty, q = qb * kTile + tx;
  const int N = b.n_max, KM = b.k_max;
  __shared__ float2 sWp[kEChunk][kTile], sWq[kEChunk][kTile];
  __shared__ float sD[kEChunk];
  __shared__ int sL[kEChunk];
  float2 acc[MAXL];
#pragma unroll
  for (int l = 0; l < MAXL; ++l) acc[l] = make_float2(0.f, 0.f);
  for (int e0 = 0; e0 < K; e0 += kEChunk) {
    for (int i = threadIdx.x; i < kEChunk * kTile; i += kTile * kTile) {
      const int e = e0 + i / kTile, j = i % kTile;
      const int ip = pb * kTile + j, iq = qb * kTile + j;
      double2 vp = make_double2(0.0, 0.0), vq = vp;
      if (e < K && ip < n) vp = b.W64[((size_t)t * KM + e) * N + ip];
      if (e < K && iq < n) vq = b.W64[((size_t)t * KM + e) * N + iq];
      sWp[i / kTile][j] = make_float2((float)vp.x, (float)vp.y);
      sWq[i / kTile][j] = make_float2((float)vq.x, (float)vq.y);
    }
    if (threadIdx.x < kEChunk) {
      const int e = e0 + threadIdx.x;
      sD[threadIdx.x] = e < K ? (float)b.wt[(size_t)t * KM + e] : 0.f;
      sL[threadIdx.x] = e < K ? b.level[(size_t)t * KM + e] : -1;
    }
    __syncthreads();
    const int ne = min(kEChunk, K - e0);
    for (int e = 0; e < ne; ++e) {
      const float2 wp = sWp[e][ty], wq = sWq[e][tx];
      const float pr = fmaf(wp.x, wq.x, wp.y * wq.y), pi = fmaf(wp.y, wq.x, -wp.x * wq.y);
      const int lv = sL[e];
      const float dd = sD[e];
#pragma unroll
      for (int l = 0; l < MAXL; ++l) {
        const float m = (lv == l) ? dd : 0.f;
        acc[l].x = fmaf(m, pr, acc[l].x);
        acc[l].y = fmaf(m, pi, acc[l].y);
      }
    }
    __syncthreads();
  }
  const bool active = p < q && q < n;
  const unsigned am = __ballot_sync(0xffffffffu, active);
  if (!active) return;
  const PairGeo g = pair_geo(b, t, p, q, a);
  const int key = cell_of(g, a);
  const int pos = cell_off[key] + agg_add(cursor, key, am);
  // pre-phase exp(2 pi i <D, x>), reduced to [-1/2, 1/2] cycles in FP64
  const double ph = a.D[0] * g.x[0] + a.D[1] * g.x[1] + a.D[2] * g.x[2];
  float sn, cn;
  sincospif(2.0f * (float)(ph - rint(ph)), &sn, &cn);
  const float cs = g.flip ? -1.f : 1.f;  // the (q, p) orientation carries the conjugate strength
  rm[pos] = make_int4(g.m0[0], g.m0[1], g.m0[2], key);
  rf[pos] = make_float4(g.fr[0], g.fr[1], g.fr[2], 0.f);
#pragma unroll
  for (int l = 0; l < MAXL; ++l) {
    if (l < a.Lp) {
      const float ar = 2.f * acc[l].x, ai = 2.f * cs * acc[l].y;
      rc[(size_t)pos * a.Lp + l] = make_float2(ar * cn - ai * sn, ar * sn + ai * cn);
    }
  }
}

// 3. Spread the sorted points: warp j takes points [j kNuRun, (j + 1) kNuRun).
// Lane i owns the footprint cells i, i + 32, ... (R rounds cover w^3 cells) and
// sums weight x strength of consecutive points with the same start cell in
// registers; at a change of start cell (and at the end) it adds its cells to
// the grid with vector float atomics. LG levels from level lg0 per pass.
template <int R, int LG>
__global__ void __launch_bounds__(256) k_nu_spread(SpreadArgs a, const int* __restrict__ total_pts,
                                                   const int4* __restrict__ rm, const float4* __restrict__ rf,
                                                   const float2* __restrict__ rc, int lg0, float2* __restrict__ F) {
  const int lane = threadIdx.x & 31;
  const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int total = *total_pts;
  const long long i_begin = wid * kNuRun;
  if (i_begin >= total) return;
  const int i_end = (int)min((long long)total, i_begin + kNuRun);
  const int w = a.w, w3 = w * w * w;
  int ix[R];  // lane's footprint cells: i0 | i1 << 4 | i2 << 8, or -1
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int c = r * 32 + lane;
    ix[r] = c < w3 ? ((c % w) | (((c / w) % w) << 4) | ((c / (w * w)) << 8)) : -1;
  }
  float2 acc[R][LG];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int l = 0; l < LG; ++l) acc[r][l] = make_float2(0.f, 0.f);
  const float tw = 2.0f / (float)w;
  const int kd = lane >> 3, kj = lane & 7;  // lane's kernel value: dimension kd, offset kj
  auto flush = [&](int4 m) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (ix[r] >= 0) {
        const int g0 = m.x + (ix[r] & 15), g1 = m.y + ((ix[r] >> 4) & 15), g2 = m.z + (ix[r] >> 8);
        const size_t base = (size_t)(m.w / a.cells) * a.cells;  // the input cell's grid
        float2* dst = F + (base + ((size_t)g2 * a.M[1] + g1) * a.M[0] + g0) * a.Lp + lg0;
        if (LG == 1) {
          atomicAdd(dst, acc[r][0]);
        } else {
#pragma unroll
          for (int l = 0; l < LG; l += 2)
            atomicAdd(reinterpret_cast<float4*>(dst + l),
                      make_float4(acc[r][l].x, acc[r][l].y, acc[r][l + 1].x, acc[r][l + 1].y));
        }
      }
#pragma unroll
      for (int l = 0; l < LG; ++l) acc[r][l] = make_float2(0.f, 0.f);
    }
  };
  int4 cur = rm[i_begin];
  for (int i = (int)i_begin; i < i_end; ++i) {
    const int4 m = rm[i];
    if (m.w != cur.w) {
      flush(cur);
      cur = m;
    }
    const float4 f = rf[i];
    float2 c[LG];
#pragma unroll
    for (int l = 0; l < LG; ++l) c[l] = rc[(size_t)i * a.Lp + lg0 + l];
    const float fd = kd == 0 ? f.x : (kd == 1 ? f.y : f.z);
    const float kv = (kd < 3 && kj < w) ? es_w((fd + kj) * tw, a.beta) : 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int x = ix[r] < 0 ? 0 : ix[r];
      const float wt = __shfl_sync(0xffffffffu, kv, x & 15) * __shfl_sync(0xffffffffu, kv, 8 + ((x >> 4) & 15)) *
                       __shfl_sync(0xffffffffu, kv, 16 + (x >> 8));
#pragma unroll
      for (int l = 0; l < LG; ++l) {
        acc[r][l].x = fmaf(wt, c[l].x, acc[r][l].x);
        acc[r][l].y = fmaf(wt, c[l].y, acc[r][l].y);
      }
    }
  }
  flush(cur);
}

// Zero-baseline terms: cst[l] += sum_{e in l} d_e sum_p |a_pe|^2 for each step.
__global__ void k_nu_const(Batch b, int t0, double* cst) {
  const int t = t0 + blockIdx.x;
  const int n = b.nst[t], K = b.nkept[t], N = b.n_max, KM = b.k_max;
  __shared__ double red[256];
  for (int e = 0; e < K; ++e) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double2 v = b.W64[((size_t)t * KM + e) * N + i];
      s += v.x * v.x + v.y * v.y;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const int l = b.level[(size_t)t * KM + e];
      if (l >= 0 && l < kMaxLevels) atomicAdd(cst + l, b.wt[(size_t)t * KM + e] * red[0]);
    }
    __syncthreads();
  }
}

// Per pixel j of a cell (pixel order[j]): 1 / prod_d psi_hat_d(s_d - D_d),
// psi_hat_d(xi) = alpha_d phi_hat(alpha_d xi), alpha_d = pi w Hc_d.
__global__ void k_nu_corr(const double* __restrict__ pix, int64_t n, const int* __restrict__ order, int64_t cnt,
                          double D0, double D1, double D2, float al0, float al1, float al2, const float* __restrict__ gl,
                          float* __restrict__ corr) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cnt) return;
  const int64_t px = order[j];
  const double D[3] = {D0, D1, D2};
  const float al[3] = {al0, al1, al2};
  float prod = 1.f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float k = al[d] * (float)(pix[(size_t)d * n + px] - D[d]);
    float s = 0.f;
#pragma unroll 8
    for (int q = 0; q < kNuGL; ++q) s = fmaf(gl[kNuGL + q], cosf(k * gl[q]), s);
    prod *= 2.f * al[d] * s;
  }
  corr[j] = 1.f / prod;
}

// First sorted point of each input cell: bnd[i] = cell_off[i * cells], i <= parts.
__global__ void k_nu_bounds(const int* __restrict__ cell_off, long long cells, int parts, int* __restrict__ bnd) {
  for (int i = threadIdx.x; i <= parts; i += blockDim.x) bnd[i] = cell_off[(size_t)i * cells];
}

struct GridArgs {
  int M[3], N2[3], Lp, l;
};

// Fine grid G[j] = F[m(k)] / prod_d psi2_hat_d(k_d) for modes |k_d| < M_d / 2 (k = j or j - N2), else 0,
// on the M_2 planes j2 that hold modes (j2 < M_2 / 2 or j2 >= N2_2 - M_2 / 2; N2_2 = 2 M_2).
__global__ void k_nu_pad(const float2* __restrict__ F, GridArgs a, const float* __restrict__ inv,
                         float2* __restrict__ G) {
  const size_t plane = (size_t)a.N2[0] * a.N2[1];
  const size_t total = plane * a.M[2];
  const float* inv0 = inv;
  const float* inv1 = inv + a.M[0];
  const float* inv2 = inv1 + a.M[1];
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int j0 = (int)(idx % a.N2[0]);
    const size_t r = idx / a.N2[0];
    const int j1 = (int)(r % a.N2[1]);
    const int qz = (int)(r / a.N2[1]);
    const int j2 = qz < a.M[2] / 2 ? qz : qz + a.M[2];
    const int k0 = j0 < a.N2[0] / 2 ? j0 : j0 - a.N2[0];
    const int k1 = j1 < a.N2[1] / 2 ? j1 : j1 - a.N2[1];
    const int k2 = j2 < a.N2[2] / 2 ? j2 : j2 - a.N2[2];
    float2 v = make_float2(0.f, 0.f);
    const int h0 = a.M[0] / 2, h1 = a.M[1] / 2, h2 = a.M[2] / 2;
    if (k0 >= -h0 && k0 < h0 && k1 >= -h1 && k1 < h1 && k2 >= -h2 && k2 < h2) {
      const int m0 = k0 + h0, m1 = k1 + h1, m2 = k2 + h2;
      const float2 f = F[(((size_t)m2 * a.M[1] + m1) * a.M[0] + m0) * a.Lp + a.l];
      const float sc = inv0[m0] * inv1[m1] * inv2[m2];
      v = make_float2(f.x * sc, f.y * sc);
    }
    G[(size_t)j2 * plane + (size_t)j1 * a.N2[0] + j0] = v;
  }
}

struct InterpArgs {
  int N2[3], w;
  float beta;
  double D[3], C[3], HN[3];  // HN = Hc * N2: target offset -> fine-grid coordinate
  double scale;              // trapezoid factor prod_d (2 pi Hc_d)(2 pi / N2_d)
};

// Pixel j of a cell (pixel order[j]) of level l: the transform of one input
// cell, interpolated, corrected and post-phased; Re added to the image, plus
// the level's zero-baseline constant when add_cst.
__global__ void k_nu_interp(const double* __restrict__ pix, int64_t n, const int* __restrict__ order, int64_t cnt,
                            InterpArgs a, const float2* __restrict__ G, const float* __restrict__ corr,
                            const double* __restrict__ cst, int add_cst, int l, const int* __restrict__ flag,
                            double* __restrict__ img) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cnt || *flag) return;
  const int64_t px = order[j];
  double sp[3];
  int m0[3];
  float fr[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    sp[d] = pix[(size_t)d * n + px] - a.D[d];
    const double tg = sp[d] * a.HN[d];
    const int m = (int)ceil(tg - 0.5 * a.w);
    fr[d] = (float)((double)m - tg);
    int mm = m % a.N2[d];
    if (mm < 0) mm += a.N2[d];
    m0[d] = mm;
  }
  const float tw = 2.0f / (float)a.w;
  float k0[kNuMaxW];
  int i0[kNuMaxW];
#pragma unroll
  for (int q = 0; q < kNuMaxW; ++q) {
    k0[q] = (q < a.w) ? es_w((fr[0] + q) * tw, a.beta) : 0.f;
    int ii = m0[0] + q;
    if (ii >= a.N2[0]) ii -= a.N2[0];
    i0[q] = ii;
  }
  float sr = 0.f, si = 0.f;
  for (int j2 = 0; j2 < a.w; ++j2) {
    const float k2 = es_w((fr[2] + j2) * tw, a.beta);
    int i2 = m0[2] + j2;
    if (i2 >= a.N2[2]) i2 -= a.N2[2];
    for (int j1 = 0; j1 < a.w; ++j1) {
      const float k12 = k2 * es_w((fr[1] + j1) * tw, a.beta);
      int i1 = m0[1] + j1;
      if (i1 >= a.N2[1]) i1 -= a.N2[1];
      const float2* row = G + ((size_t)i2 * a.N2[1] + i1) * a.N2[0];
      float rr = 0.f, ri = 0.f;
#pragma unroll
      for (int q = 0; q < kNuMaxW; ++q) {
        if (q < a.w) {
          const float2 g = __ldg(row + i0[q]);
          rr = fmaf(k0[q], g.x, rr);
          ri = fmaf(k0[q], g.y, ri);
        }
      }
      sr = fmaf(k12, rr, sr);
      si = fmaf(k12, ri, si);
    }
  }
  // post-phase exp(2 pi i <s - D, C>), reduced in FP64
  const double ph = sp[0] * a.C[0] + sp[1] * a.C[1] + sp[2] * a.C[2];
  float sn, cn;
  sincospif(2.0f * (float)(ph - rint(ph)), &sn, &cn);
  const double re = (double)(sr * cn - si * sn) * (double)corr[j] * a.scale;
  img[(size_t)l * n + px] += re + (add_cst ? cst[l] : 0.0);
}

template <typename F>
void dispatch_levels(int L, F&& f) {
  if (L <= 1) f(std::integral_constant<int, 1>{});
  else if (L <= 2) f(std::integral_constant<int, 2>{});
  else if (L <= 4) f(std::integral_constant<int, 4>{});
  else if (L <= 8) f(std::integral_constant<int, 8>{});
  else f(std::integral_constant<int, 16>{});
}

template <typename T>
bool grow(T** p, size_t* cap, size_t need) {
  if (need <= *cap && *p) return true;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  if (cudaMalloc((void**)p, sizeof(T) * std::max<size_t>(need, 1)) != cudaSuccess) {
    *p = nullptr;
    return false;
  }
  *cap = need;
  return true;
}

}  // namespace

bool nu_kernel_params(double eps, int* w, float* beta) {
  if (!(eps >= 1e-7 && eps <= 0.1)) return false;
  int ww = (int)ceil(log10(1.0 / eps) - 1e-12) + 1;
  ww = std::min(std::max(ww, 2), kNuMaxW);
  *w = ww;
  *beta = 2.30f * (float)ww;
  return true;
}

NuPixCells nu_pixel_cells(const double* pix, int64_t n, const int P[3]) {
  double lo[3], hi[3];
  for (int d = 0; d < 3; ++d) {
    lo[d] = hi[d] = pix[(size_t)d * n];
    for (int64_t j = 1; j < n; ++j) {
      lo[d] = std::min(lo[d], pix[(size_t)d * n + j]);
      hi[d] = std::max(hi[d], pix[(size_t)d * n + j]);
    }
  }
  const int nc = P[0] * P[1] * P[2];
  std::vector<int> cell(n);
  std::vector<int64_t> cnt(nc, 0);
  for (int64_t j = 0; j < n; ++j) {
    int ci[3];
    for (int d = 0; d < 3; ++d) {
      const double wd = hi[d] - lo[d];
      int c = wd > 0.0 ? (int)floor((pix[(size_t)d * n + j] - lo[d]) / wd * P[d]) : 0;
      ci[d] = std::min(std::max(c, 0), P[d] - 1);
    }
    cell[j] = (ci[2] * P[1] + ci[1]) * P[0] + ci[0];
    ++cnt[cell[j]];
  }
  NuPixCells out;
  out.off.assign(nc + 1, 0);
  for (int c = 0; c < nc; ++c) out.off[c + 1] = out.off[c] + cnt[c];
  out.order.resize(n);
  std::vector<int64_t> cur(out.off.begin(), out.off.end() - 1);
  for (int64_t j = 0; j < n; ++j) out.order[cur[cell[j]]++] = (int)j;
  out.box.resize(nc);
  for (int c = 0; c < nc; ++c) {
    NuPixBox& b = out.box[c];
    for (int d = 0; d < 3; ++d) {
      double l = 0.0, h = 0.0;
      for (int64_t k = out.off[c]; k < out.off[c + 1]; ++k) {
        const double v = pix[(size_t)d * n + out.order[k]];
        if (k == out.off[c] || v < l) l = v;
        if (k == out.off[c] || v > h) h = v;
      }
      b.D[d] = 0.5 * (l + h);
      b.S[d] = 0.5 * (h - l);
    }
  }
  return out;
}

NuPlan nu_plan(const NuPixBox& px, int w, float beta, const int P[3], const double* h_st, int N, const int* nst,
               const double* wl, int t0, int t1) {
  NuPlan p;
  p.w = w;
  p.beta = beta;
  double R[3] = {0, 0, 0};  // largest baseline component per dimension [cycles]
  for (int t = t0; t < t1; ++t)
    for (int d = 0; d < 3; ++d) {
      const double* c = h_st + ((size_t)t * 3 + d) * N;
      double lo = c[0], hi = c[0];
      for (int i = 1; i < nst[t]; ++i) {
        lo = std::min(lo, c[i]);
        hi = std::max(hi, c[i]);
      }
      R[d] = std::max(R[d], (hi - lo) / wl[t]);
    }
  int fold = 0;
  for (int d = 1; d < 3; ++d)
    if (R[d] * px.S[d] > R[fold] * px.S[fold]) fold = d;
  p.fold = fold;
  for (int d = 0; d < 3; ++d) {
    const double lo = (d == fold) ? 0.0 : -R[d], hi = R[d];
    p.P[d] = P[d];
    p.lo[d] = lo;
    p.delta[d] = (hi - lo) / P[d];
    const double X = 0.5 * p.delta[d], S = px.S[d];  // half-widths of one input cell and of the targets
    p.D[d] = px.D[d];
    // grids beyond 2^28 points per dimension are reported as such (the caller
    // rejects them) rather than searched for and cast to int
    const double need = ceil(4.0 * kSigma * X * S * (1.0 + 1e-12)) + w + 2;
    constexpr long long kMaxM = 1LL << 28;
    p.M[d] = !(need <= (double)kMaxM) ? (int)(kMaxM + 2)
                                      : (int)next_smooth(std::max<long long>(2 * w, (long long)need));
    if (S > 0.0)
      p.Hc[d] = 1.0 / (2.0 * kSigma * S);
    else if (X > 0.0)
      p.Hc[d] = 2.0 * X / (p.M[d] - w - 2);
    else
      p.Hc[d] = 1.0 / (2.0 * M_PI);
    p.N2[d] = 2 * p.M[d];
  }
  return p;
}

size_t nu_grid_bytes(const NuPlan& p, int n_level, size_t pair_slots) {
  const int Lp = n_level == 1 ? 1 : n_level + (n_level & 1);
  return (size_t)p.parts() * p.cells() * (Lp * sizeof(float2) + 3 * sizeof(int)) + 2 * p.cells2() * sizeof(float2) +
         pair_slots * (sizeof(int4) + sizeof(float4) + Lp * sizeof(float2));
}

int nu_enqueue(const Batch& b, int t0, int t1, const NuPlan& p, NufftWs* w, const double* d_pix, int64_t n_pix,
               const int* d_order, int64_t pix_off, int64_t pix_cnt, int cell, int n_cells, int n_level,
               double* img, cudaStream_t s, int* launches, const cudaEvent_t* ev) {
  const int Lp = n_level == 1 ? 1 : n_level + (n_level & 1);
  const int parts = p.parts();
  const size_t cells = p.cells();
  const size_t nkeys = (size_t)parts * cells;  // sort keys: input cell, then start cell
  if (nkeys >= (size_t)1 << 31) return -1;
  int nl = 0;
  if (!grow(&w->F, &w->F_cap, nkeys * Lp)) return -1;
  const size_t oldG = w->G_cap;
  const float2* oldGp = w->G;
  if (!grow(&w->G, &w->G_cap, p.cells2())) return -1;
  if (!grow(&w->G2, &w->G2_cap, p.cells2())) return -1;
  if (w->G != oldGp || w->G_cap != oldG) w->have_fft = false;  // new buffer: zero planes to rewrite
  if (!grow(&w->inv, &w->inv_cap, (size_t)p.M[0] + p.M[1] + p.M[2])) return -1;
  size_t corr_cap = (size_t)w->corr_cap;
  if (!grow(&w->corr, &corr_cap, (size_t)n_pix)) return -1;
  if ((int64_t)corr_cap != w->corr_cap || (int)w->corr_key.size() != n_cells) w->corr_key.assign(n_cells, {});
  w->corr_cap = (int64_t)corr_cap;
  if (!grow(&w->bnd, &w->bnd_cap, (size_t)parts + 1)) return -1;
  if (!w->cst && cudaMalloc(&w->cst, sizeof(double) * kMaxLevels) != cudaSuccess) return -1;

  double z[kNuGL], wq[kNuGL];
  gauss_legendre_half(z, wq);
  if (!w->gl || w->gl_w != p.w || w->gl_beta != p.beta) {
    if (!w->gl && cudaMalloc(&w->gl, sizeof(float) * 2 * kNuGL) != cudaSuccess) return -1;
    float hg[2 * kNuGL];
    for (int q = 0; q < kNuGL; ++q) {
      hg[q] = (float)z[q];
      hg[kNuGL + q] = (float)(wq[q] * phi_host(z[q], p.beta));
    }
    if (cudaMemcpy(w->gl, hg, sizeof(hg), cudaMemcpyHostToDevice) != cudaSuccess) return -1;
    w->gl_w = p.w;
    w->gl_beta = p.beta;
    w->corr_key.assign(n_cells, {});
  }
  // per-pixel correction of this image cell: depends on its pixels, the kernel and the spacing only
  const std::vector<double> key = {(double)p.w, p.Hc[0], p.Hc[1], p.Hc[2], p.D[0], p.D[1], p.D[2]};
  if (w->corr_key[cell] != key && pix_cnt > 0) {
    const float al[3] = {(float)(M_PI * p.w * p.Hc[0]), (float)(M_PI * p.w * p.Hc[1]), (float)(M_PI * p.w * p.Hc[2])};
    k_nu_corr<<<(unsigned)((pix_cnt + 255) / 256), 256, 0, s>>>(d_pix, n_pix, d_order + pix_off, pix_cnt, p.D[0],
                                                                p.D[1], p.D[2], al[0], al[1], al[2], w->gl,
                                                                w->corr + pix_off);
    ++nl;
    w->corr_key[cell] = key;
  }
  // 1 / psi2_hat per mode, alpha2 = pi w / N2
  w->h_inv.resize((size_t)p.M[0] + p.M[1] + p.M[2]);
  size_t o = 0;
  for (int d = 0; d < 3; ++d) {
    const double al2 = M_PI * p.w / p.N2[d];
    for (int m = 0; m < p.M[d]; ++m) w->h_inv[o++] = (float)(1.0 / es_ft_host(m - p.M[d] / 2, al2, p.beta, z, wq));
  }
  if (cudaMemcpyAsync(w->inv, w->h_inv.data(), sizeof(float) * o, cudaMemcpyHostToDevice, s) != cudaSuccess) return -1;
  if (cudaMemsetAsync(w->F, 0, sizeof(float2) * nkeys * Lp, s) != cudaSuccess) return -1;
  if (cudaMemsetAsync(w->cst, 0, sizeof(double) * kMaxLevels, s) != cudaSuccess) return -1;

  const int T = t1 - t0;
  SpreadArgs sa;
  for (int d = 0; d < 3; ++d) {
    sa.M[d] = p.M[d];
    sa.invH[d] = 1.0 / p.Hc[d];
    sa.D[d] = p.D[d];
    sa.P[d] = p.P[d];
    sa.lo[d] = p.lo[d];
    sa.delta[d] = p.delta[d];
    sa.idelta[d] = (p.P[d] > 1 && p.delta[d] > 0.0) ? 1.0 / p.delta[d] : 0.0;
  }
  sa.cells = (long long)cells;
  sa.fold = p.fold;
  sa.w = p.w;
  sa.L = n_level;
  sa.Lp = Lp;
  sa.beta = p.beta;
  // points sorted by input cell and the grid cell of their spread start (a counting sort)
  const int LG = Lp == 1 ? 1 : (Lp % 4 == 0 ? 4 : 2);
  const long long nseg = ((long long)nkeys + kSeg - 1) / kSeg;
  const long long NP = (long long)b.n_max * (b.n_max - 1) / 2;
  const size_t slots = (size_t)NP * T;
  if (!grow(&w->count, &w->count_cap, nkeys) || !grow(&w->cursor, &w->cursor_cap, nkeys) ||
      !grow(&w->cell_off, &w->cell_off_cap, nkeys + 1) || !grow(&w->seg_sum, &w->seg_sum_cap, (size_t)nseg) ||
      !grow(&w->seg_off, &w->seg_off_cap, (size_t)nseg + 1) || !grow(&w->rm, &w->rm_cap, slots) ||
      !grow(&w->rf, &w->rf_cap, slots) || !grow(&w->rc, &w->rc_cap, slots * Lp))
    return -1;
  if (cudaMemsetAsync(w->count, 0, sizeof(int) * nkeys, s) != cudaSuccess) return -1;
  if (cudaMemsetAsync(w->cursor, 0, sizeof(int) * nkeys, s) != cudaSuccess) return -1;
  int sms = 148, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);

  if (ev) cudaEventRecord(ev[0], s);
  k_nu_const<<<T, 256, 0, s>>>(b, t0, w->cst);
  if (slots > 0) {
    const unsigned cgrid = (unsigned)std::min<size_t>((slots + 255) / 256, (size_t)sms * 32);
    k_nu_count<<<cgrid, 256, 0, s>>>(b, t0, T, sa, w->count);
  }
  k_nu_seg_sum<<<(unsigned)nseg, 1024, 0, s>>>(w->count, (long long)nkeys, w->seg_sum);
  k_nu_scan<<<1, 1024, 0, s>>>(w->seg_sum, (int)nseg, w->seg_off);
  k_nu_seg_scan<<<(unsigned)nseg, 1024, 0, s>>>(w->count, (long long)nkeys, w->seg_off, w->cell_off);
  const int nb = (b.n_max + kTile - 1) / kTile;
  const dim3 grid(nb * (nb + 1) / 2, 1, T);
  dispatch_levels(n_level, [&](auto ML) {
    constexpr int L = decltype(ML)::value;
    k_nu_scatter<L><<<grid, kTile * kTile, 0, s>>>(b, t0, sa, w->cell_off, w->cursor, w->rm, w->rf, w->rc);
  });
  nl += 6;
  if (ev) cudaEventRecord(ev[7], s);
  if (slots > 0) {
    const unsigned sgrid = (unsigned)((slots + (size_t)kNuRun * 8 - 1) / ((size_t)kNuRun * 8));
    const int* total = w->cell_off + nkeys;
    auto spread = [&](auto kern) {
      for (int g = 0; g < Lp / LG; ++g) {
        kern<<<sgrid, 256, 0, s>>>(sa, total, w->rm, w->rf, w->rc, g * LG, w->F);
        ++nl;
      }
    };
    const int w3 = p.w * p.w * p.w;
    auto by_lg = [&](auto RR) {
      constexpr int R = decltype(RR)::value;
      if (LG == 1) spread(k_nu_spread<R, 1>);
      else if (LG == 2) spread(k_nu_spread<R, 2>);
      else spread(k_nu_spread<R, 4>);
    };
    if (w3 <= 32) by_lg(std::integral_constant<int, 1>{});
    else if (w3 <= 64) by_lg(std::integral_constant<int, 2>{});
    else if (w3 <= 128) by_lg(std::integral_constant<int, 4>{});
    else if (w3 <= 224) by_lg(std::integral_constant<int, 7>{});
    else if (w3 <= 352) by_lg(std::integral_constant<int, 11>{});
    else by_lg(std::integral_constant<int, 16>{});
  }
  if (cudaGetLastError() != cudaSuccess) return -3;
  if (ev) cudaEventRecord(ev[1], s);

  // the input cells that received points (all of them are transformed when there is one)
  std::vector<int> todo;
  if (parts == 1) {
    todo.push_back(0);
  } else {
    k_nu_bounds<<<1, 256, 0, s>>>(w->cell_off, (long long)cells, parts, w->bnd);
    ++nl;
    w->h_bnd.resize(parts + 1);
    if (cudaMemcpyAsync(w->h_bnd.data(), w->bnd, sizeof(int) * (parts + 1), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return -3;
    for (int q = 0; q < parts; ++q)
      if (w->h_bnd[q + 1] > w->h_bnd[q]) todo.push_back(q);
    if (todo.empty()) todo.push_back(0);  // the zero-baseline constants still go into the image
  }

  const long long plane = (long long)p.N2[0] * p.N2[1];
  if (!w->have_fft || w->fft_n[0] != p.N2[0] || w->fft_n[1] != p.N2[1] || w->fft_n[2] != p.N2[2]) {
    if (cudaStreamSynchronize(s) != cudaSuccess) return -2;  // old plans may still be executing
    if (w->fft) cufftDestroy(w->fft);
    if (w->fftz) cufftDestroy(w->fftz);
    w->fft = w->fftz = 0;
    w->have_fft = false;
    size_t ws = 0;
    long long n2[2] = {p.N2[1], p.N2[0]};
    long long nz[1] = {p.N2[2]}, ez[1] = {p.N2[2]};
    if (cufftCreate(&w->fft) != CUFFT_SUCCESS || cufftCreate(&w->fftz) != CUFFT_SUCCESS) return -2;
    if (cufftMakePlanMany64(w->fft, 2, n2, nullptr, 1, plane, nullptr, 1, plane, CUFFT_C2C, p.M[2] / 2, &ws) !=
            CUFFT_SUCCESS ||
        cufftMakePlanMany64(w->fftz, 1, nz, ez, plane, 1, ez, plane, 1, CUFFT_C2C, plane, &ws) != CUFFT_SUCCESS)
      return -2;
    // the planes without modes are zero once and for all
    if (cudaMemsetAsync(w->G, 0, sizeof(float2) * p.cells2(), s) != cudaSuccess) return -2;
    w->have_fft = true;
    for (int d = 0; d < 3; ++d) w->fft_n[d] = p.N2[d];
  }
  if (cufftSetStream(w->fft, s) != CUFFT_SUCCESS || cufftSetStream(w->fftz, s) != CUFFT_SUCCESS) return -2;

  GridArgs ga;
  InterpArgs ia;
  double scale = 1.0;
  for (int d = 0; d < 3; ++d) {
    ga.M[d] = p.M[d];
    ga.N2[d] = p.N2[d];
    ia.N2[d] = p.N2[d];
    ia.D[d] = p.D[d];
    ia.HN[d] = p.Hc[d] * p.N2[d];
    scale *= (2.0 * M_PI * p.Hc[d]) * (2.0 * M_PI / p.N2[d]);
  }
  ia.w = p.w;
  ia.beta = p.beta;
  ia.scale = scale;
  ga.Lp = Lp;
  const unsigned pad_grid = (unsigned)std::min<size_t>(((size_t)plane * p.M[2] + 255) / 256, (size_t)sms * 16);
  const unsigned pix_grid = (unsigned)((pix_cnt + 255) / 256);
  bool first = true;
  for (const int q : todo) {
    for (int d = 0; d < 3; ++d) ia.C[d] = p.C(q, d);
    const float2* Fq = w->F + (size_t)q * cells * Lp;
    for (int l = 0; l < n_level; ++l) {
      ga.l = l;
      const bool mark = ev && first && l == 0;
      if (mark) cudaEventRecord(ev[2], s);
      k_nu_pad<<<pad_grid, 256, 0, s>>>(Fq, ga, w->inv, w->G);
      if (mark) cudaEventRecord(ev[3], s);
      cufftComplex* g = reinterpret_cast<cufftComplex*>(w->G);
      cufftComplex* g_hi = g + (size_t)(p.N2[2] - p.M[2] / 2) * plane;  // the upper planes with modes
      if (cufftExecC2C(w->fft, g, g, CUFFT_INVERSE) != CUFFT_SUCCESS ||
          cufftExecC2C(w->fft, g_hi, g_hi, CUFFT_INVERSE) != CUFFT_SUCCESS ||
          cufftExecC2C(w->fftz, g, reinterpret_cast<cufftComplex*>(w->G2), CUFFT_INVERSE) != CUFFT_SUCCESS)
        return -2;
      if (mark) cudaEventRecord(ev[4], s);
      if (pix_cnt > 0)
        k_nu_interp<<<pix_grid, 256, 0, s>>>(d_pix, n_pix, d_order + pix_off, pix_cnt, ia, w->G2, w->corr + pix_off,
                                             w->cst, first ? 1 : 0, l, b.flag, img);
      if (mark) cudaEventRecord(ev[5], s);
      nl += 2;
    }
    first = false;
  }
  if (ev) cudaEventRecord(ev[6], s);
  if (cudaGetLastError() != cudaSuccess) return -3;
  if (launches) *launches += nl;
  return 0;
}

void nu_free(NufftWs* w) {
  if (w->fft) cufftDestroy(w->fft);
  if (w->fftz) cufftDestroy(w->fftz);
  void* ptrs[] = {w->F, w->G, w->G2, w->inv, w->corr, w->cst, w->gl, w->count, w->cursor, w->cell_off, w->seg_sum,
                  w->seg_off, w->rm, w->rf, w->rc, w->bnd};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  *w = NufftWs{};
}

}  // namespace bipp
