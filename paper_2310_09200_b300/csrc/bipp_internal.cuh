// bipp_internal.cuh — shared declarations of the B300 standard-synthesis
// library (device layouts, kernel launchers). Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bipp {

constexpr int kMaxStations = 1024;  // per step
constexpr int kMaxLevels = 16;
constexpr int kMaxEig = 1024;

// Per-step status bits written by the device stages.
constexpr int kStatusNotPD = 1;         // Cholesky met a non-positive (or NaN) pivot
constexpr int kStatusNotConverged = 2;  // Jacobi hit its sweep cap
constexpr int kStatusTimeout = 4;       // a bounded device wait gave up
constexpr int kStatusRange = 16;        // a station lies beyond the tensor-core phase's range (2^28 wavelengths)

// Device-side view of one batch of T steps. Step t uses the leading
// nst[t] x nst[t] block of every per-step N x N array (N = n_max).
struct Batch {
  int T;          // steps in the batch
  int n_max;      // leading dimension of per-step station arrays
  int k_max;      // leading dimension of per-step eigen arrays
  const int* nst;   // [T] stations per step
  const int* neig;  // [T] eigenpairs requested per step
  const double* wl; // [T] wavelength of each step [m]
  const int* chan;  // [T] channel of each step (non-decreasing), or nullptr = all channel 0
  const double* st;   // [T][3][n_max] station xyz (metres), column-major per step
  const double2* vis; // [T][n_max][n_max] visibilities, column-major per step
  double* G;      // [T][n_max][n_max] Gram matrix, then its Cholesky factor L (lower)
  double* Linv;   // [T][n_max][n_max] row-major L^{-1}: Linv[t][i*n_max + j] = (L^{-1})_ij
  double2* X;     // [T][n_max][n_max] scratch: L^{-1} V (column-major)
  double2* C;     // [T][n_max][n_max] reduced matrix L^{-1} V L^{-T} (column-major), Jacobi in place
  double2* Q;     // [T][n_max][n_max] Jacobi rotations (column-major)
  double* mu;     // [T][n_max] Jacobi eigenvalues (unsorted)
  int* status;    // [T] status bits
  int* sweeps;    // [T] Jacobi sweeps used (QR steps of the FP32 stage of the mixed eigensolve)
  // selection / packing outputs
  int* nkept;     // [T] eigenpairs kept (== neig[t] on success, 0 on failure)
  double* sel_mu; // [T][k_max] kept eigenvalues, descending
  int* level;     // [T][k_max] level id, -1 = dropped
  double* wt;     // [T][k_max] filter weight d_e
  double2* W64;   // [T][k_max][n_max] kept eigenvectors a_e (G-orthonormal), e-major
  float2* W32;    // [T][n_max][k_max] FP32 copy, station-major
  float* q;       // [T][6][n_max] station p/wl as float hi/lo: xh,yh,zh,xl,yl,zl
  int* flag;      // [1] OR of all step statuses (synthesis skips the batch if set)
  int eigen;      // 1: one image per kept eigenpair (level = rank) instead of energy levels
  // [T] the problems by descending station count, or nullptr (identity): the
  // per-problem kernels of the Gram, reduction and eigensolve stages take
  // problem order[block], so that in a batch of uneven steps the largest
  // (longest-running) problems start in the first wave of CTAs
  const int* order = nullptr;
};
__device__ __forceinline__ int prob_of(const int* order, int blk) { return order ? order[blk] : blk; }

// Eigenimages use the level kernels with kEigSlots register slots per thread:
// every synthesis thread owns a fixed quarter of the <= 64 eigenvectors.
constexpr int kMaxEigenimages = 64;
constexpr int kEigSlots = 16;

// Small per-step arrays of the mixed-precision eigensolver (eig_mixed.cu).
struct MixedWs {
  int KP;          // leading dimension of the per-step kp-sized arrays (max kp of the batch)
  int* kp;         // [T] pairs refined per step: min(n, n_eig + 16)
  float* lam;      // [T][n_max] the kp leading eigenvalues of the FP32 tridiagonal form / tnorm, descending
  float* tnorm;    // [T] ||T||_F of the FP32 tridiagonal form (= ||C||_F to FP32 rounding)
  double* theta;   // [T][KP] refined eigenvalues
  double* rnorm;   // [T][KP] residual norms of the last pass
  double* cnorm;   // [T] ||C||_F
  int* st2;        // [T] status of the small FP64 Jacobi solves
  int* sw2;        // [T] their sweeps
};

struct Pixels {
  int64_t n;
  const double* xyz;  // [3][n] FP64 unit vectors (column-major)
  const float* hl;    // [6][n] float hi/lo split: xh,yh,zh,xl,yl,zl
};

// Channel of step t and whether t is the last step of its channel in the batch
// (the synthesis kernels flush their per-channel register sums there).
__device__ __forceinline__ int step_chan(const Batch& b, int t) { return b.chan ? b.chan[t] : 0; }
__device__ __forceinline__ bool last_of_chan(const Batch& b, int t) {
  return t == b.T - 1 || (b.chan && b.chan[t + 1] != b.chan[t]);
}

// ---- launchers (stream-ordered, no synchronisation) ----
void launch_gram(const Batch& b, int gram_identity, cudaStream_t s);
void launch_cholesky(const Batch& b, int gram_identity, cudaStream_t s);
void launch_reduce(const Batch& b, int gram_identity, cudaStream_t s);
// The mixed eigensolver's reduction: C32 = L^{-1} V L^{-T} (or the Hermitian
// part of V when G = I) in FP32 into the first half of each step's X buffer;
// the FP64 C is not formed (the refinement applies L^{-1} V L^{-T} in factored
// form). 2 launches (1 with G = I).
void launch_reduce32(const Batch& b, int gram_identity, cudaStream_t s);
void launch_jacobi(const Batch& b, double tol, int max_sweeps, cudaStream_t s);
// Mixed-precision eigensolve (the leading pairs of the FP32 tridiagonal form +
// FP64-class refinement); needs the X and Q buffers of the batch as scratch,
// which fits when eig_mixed_fits(n_max, KP).
bool eig_mixed_fits(int n_max, int KP);
constexpr int kMixedLaunches = 77;  // kernels launched by launch_eig_mixed
void launch_eig_mixed(const Batch& b, const MixedWs& w, double tol, int max_sweeps, cudaStream_t s);
// Error message of calls without a handle (returned by bipp_ss_last_error(NULL)).
int set_global_error(int code, const char* msg);
// d_bounds: per channel, n_level x 2 column-major blocks.
void launch_select(const Batch& b, int n_level, const double* d_bounds, int filter, cudaStream_t s);
void launch_pixel_split(const double* d_xyz, float* d_hl, int64_t n, cudaStream_t s);
// n complex64 values widened into complex128 (the batch visibility buffer).
void launch_vis_widen(const float2* d_in, double2* d_out, size_t n, cudaStream_t s);

// Synthesis of a whole batch into img (per channel c: n_pix x n_level FP64 at
// img + c * n_level * n_pix, accumulated).
void launch_synth_simt_f64(const Batch& b, const Pixels& px, int n_level, double* img, cudaStream_t s);
void launch_synth_simt_f32(const Batch& b, const Pixels& px, int n_level, double* img, cudaStream_t s);

}  // namespace bipp
