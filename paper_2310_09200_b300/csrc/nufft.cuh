// nufft.cuh — NUFFT synthesis (Sec. 2.5 "NUFFT Image Synthesis", Sec. 3.4
// "NUFFT Synthesis", Algorithm 3): internal interface of nufft.cu.
//
// Per channel and level, the level's Gram-corrected visibilities
// V'_l = sum_{e in l} d_e a_e a_e^H of every step of the batch are summed over
// all baselines with one type-3 NUFFT:
//   I_l(r) += sum_t sum_{p,q} V'_l,pq(t) exp(2 pi i <r, x_pq(t)>),  x_pq = -(p_p - p_q) / wl  [cycles]
// Coordinates are in cycles: the phase of input point x and target s is 2 pi <s, x>.
//
// Domain partitioning (Sec. 3.4.1): the box of the (oriented) baselines is split
// into P0 x P1 x P2 equal input cells and the pixels into image cells; every
// non-empty (input cell, image cell) pair is one type-3 transform with the
// cells' own centres, so each uniform grid spans one cell's extent only.
#pragma once

#include <cufft.h>

#include <vector>

#include "bipp_internal.cuh"

namespace bipp {

constexpr int kNuMaxW = 8;  // kernel width cap: tolerances down to 1e-7
constexpr int kNuGL = 32;   // Gauss-Legendre nodes on (0, 1) for the kernel's Fourier transform

// Target (pixel) box: centre D and half-width S per dimension.
struct NuPixBox {
  double D[3], S[3];
};

// Image cells of a handle: pixel indices sorted by cell (order), the cells'
// ranges in that order (off, n_cells + 1 entries) and their pixel boxes.
struct NuPixCells {
  std::vector<int> order;
  std::vector<int64_t> off;
  std::vector<NuPixBox> box;
};

// Geometry of the type-3 transforms of one channel group and image cell: the
// input cells share the grid size and spacing and differ by their centres.
struct NuPlan {
  int w = 0;         // kernel width (grid points)
  float beta = 0;    // kernel shape, 2.30 w
  int fold = 0;      // dimension on which every point is oriented to x >= 0 (Hermitian symmetry)
  int P[3] = {1, 1, 1};  // input cells per dimension
  double lo[3] = {};     // low corner of the input box [cycles]
  double delta[3] = {};  // input cell size [cycles]
  int M[3] = {};     // spread-grid points per dimension of one input cell (dimension 0 fastest)
  int N2[3] = {};    // type-2 fine grid, 2 M
  double Hc[3] = {}; // spread-grid spacing [cycles]
  double D[3] = {};  // centre of the targets
  size_t cells() const { return (size_t)M[0] * M[1] * M[2]; }
  size_t cells2() const { return (size_t)N2[0] * N2[1] * N2[2]; }
  int parts() const { return P[0] * P[1] * P[2]; }
  // centre of input cell pid (cell index 0 fastest)
  double C(int pid, int d) const {
    const int ci = d == 0 ? pid % P[0] : (d == 1 ? (pid / P[0]) % P[1] : pid / (P[0] * P[1]));
    return lo[d] + (ci + 0.5) * delta[d];
  }
};

struct NufftWs {
  float2* F = nullptr;   // spread grid [M2][M1][M0][Lp] (Lp levels, even unless 1)
  size_t F_cap = 0;      // float2 elements
  float2* G = nullptr;   // fine grid [N2_2][N2_1][N2_0]: the modes; planes without modes stay zero
  size_t G_cap = 0;
  float2* G2 = nullptr;  // its transform (the z-transform writes here, out of place)
  size_t G2_cap = 0;
  float* inv = nullptr;  // 1 / (second kernel's transform) per mode, M0 + M1 + M2
  size_t inv_cap = 0;
  float* corr = nullptr; // per pixel (sorted order) 1 / prod_d psi_hat_d(s_d - D_d)
  int64_t corr_cap = 0;
  int* bnd = nullptr;    // [parts + 1] first sorted point of each input cell
  size_t bnd_cap = 0;
  std::vector<int> h_bnd;
  double* cst = nullptr; // [kMaxLevels] zero-baseline (p = q) terms of the current channel
  // points sorted by the grid cell of their spread start: counts, cursors, offsets
  int* count = nullptr;
  size_t count_cap = 0;
  int* cursor = nullptr;
  size_t cursor_cap = 0;
  int* cell_off = nullptr;  // [cells + 1] exclusive offsets, total at the end
  size_t cell_off_cap = 0;
  int* seg_sum = nullptr;   // scan segments' totals and offsets
  size_t seg_sum_cap = 0;
  int* seg_off = nullptr;
  size_t seg_off_cap = 0;
  int4* rm = nullptr;    // per point: spread start m0 and its cell
  size_t rm_cap = 0;
  float4* rf = nullptr;  // per point: fractions m0 - g
  size_t rf_cap = 0;
  float2* rc = nullptr;  // per point: Lp pre-phased level strengths
  size_t rc_cap = 0;
  float* gl = nullptr;   // [2][kNuGL]: Gauss-Legendre nodes z_q and weights w_q phi(z_q) on (0, 1)
  int gl_w = 0;          // kernel width gl was made for
  float gl_beta = 0;
  // per image cell: the kernel width, spacing and centre its part of corr was made for
  std::vector<std::vector<double>> corr_key;
  cufftHandle fft = 0;   // 2-D (x, y) transforms of the planes that hold modes, in place
  cufftHandle fftz = 0;  // 1-D transforms along z, G -> G2
  bool have_fft = false;
  int fft_n[3] = {};     // the fine grid the plans and G's zero planes were made for
  std::vector<float> h_inv;
};

// Kernel parameters for tolerance eps in [1e-7, 0.1]; false outside.
bool nu_kernel_params(double eps, int* w, float* beta);

// Image cells of n pixels (host, [3][n] column-major): the pixels' box split
// into P[0] x P[1] x P[2] equal cells; empty cells get an empty range.
NuPixCells nu_pixel_cells(const double* pix, int64_t n, const int P[3]);

// Plan of the steps [t0, t1) of a batch for the image cell with box px:
// host station coordinates h_st ([T][3][N] column-major per step), per-step
// station counts and wavelengths; P input cells per dimension.
NuPlan nu_plan(const NuPixBox& px, int w, float beta, const int P[3], const double* h_st, int N, const int* nst,
               const double* wl, int t0, int t1);

// Device bytes of the plan's grids and of the sorted point records for
// pair_slots = steps x n_max (n_max - 1) / 2 (the FFT's own workspace comes on top).
size_t nu_grid_bytes(const NuPlan& p, int n_level, size_t pair_slots);

// Enqueue the NUFFT synthesis of steps [t0, t1) (one channel) onto the pixels
// d_order[pix_off, pix_off + pix_cnt) (image cell `cell` of n_cells) of img
// (n_level x n_pix FP64, accumulated; skipped when *b.flag is set). Returns 0,
// or -1 (allocation failed), -2 (FFT plan or launch failed), -3 (kernel launch
// failed). Synchronises the stream once when there are several input cells
// (to skip the empty ones). ev (optional, 8 events): recorded before the sort,
// after the spreading, around the first transform's pad, FFT and interpolation,
// after the last transform, and between the sort and the spreading.
int nu_enqueue(const Batch& b, int t0, int t1, const NuPlan& p, NufftWs* w, const double* d_pix, int64_t n_pix,
               const int* d_order, int64_t pix_off, int64_t pix_cnt, int cell, int n_cells, int n_level,
               double* img, cudaStream_t s, int* launches, const cudaEvent_t* ev);

void nu_free(NufftWs* w);

}  // namespace bipp
