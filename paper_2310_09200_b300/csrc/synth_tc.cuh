// synth_tc.cuh — tcgen05 fused synthesis (split BF16 / FP16 hi+lo products on
// the 5th-generation tensor cores). Internal to libbipp_ss.so.
#pragma once

#include <stdint.h>

#include <vector>

#include "bipp_internal.cuh"

namespace bipp {

constexpr int kTcMaxEig = 128;  // eigenvectors per step on the tensor-core path (N = 2*K <= 256)
// Per step in TcWorkspace::lwt: kTcMaxEig (level, weight) words, then one word per
// block of 8 accumulator column pairs whose x is the level common to the block's
// imaged pairs (-1: none imaged, -2: more than one level).
constexpr int kLwtStride = kTcMaxEig + kTcMaxEig / 8;

// Per-step geometry of the tensor-core GEMM: B operand chunks of 64 K-rows
// (32 stations) packed at b_off, n_chunks of them, ncols = 2*K rounded up to
// a multiple of 16, and the tcgen05 instruction descriptors for N = ncols and
// N = 2 ncols (the hi and lo images of B side by side).
struct TcStep {
  long long b_off;
  int n_chunks;
  int ncols;
  uint32_t idesc;
  uint32_t idesc2;
};

// Device workspace of the tensor-core path.
struct TcWorkspace {
  unsigned char* B = nullptr;  // packed, pre-swizzled hi/lo operand chunks of every step
  size_t B_bytes = 0;
  TcStep* steps = nullptr;     // [cap_T] device copy of the step table
  TcStep* h_steps = nullptr;   // [cap_T] pinned host step table (source of the copy, graph-safe)
  float* scale = nullptr;      // [cap_T] operand scale of the FP16 variant (W * scale)
  uint32_t* qph = nullptr;     // [cap_T][chunks * 16][20] station phase words, in pairs of stations (k_tc_pack)
  int qph_stride = 0;          // stations per step in qph (32 * chunks of n_max)
  int2* lwt = nullptr;         // [cap_T][kLwtStride] (level, FP32 weight / scale^2) per accumulator column pair, block levels
  int* status = nullptr;       // [2] device error word (0 = ok), fault-injection word (0 = off)
  int cap_T = 0;
};

// Output of the adjoint's first stage (k_synth_tc with EPI = 1): R = dL/dI
// (n_level x n_pix FP64) in, Y out. Y holds, per step t and 64-pixel chunk c,
// at ((t * nc64 + c) * 2 ncols) * 128 bytes, a BF16 hi image and then a lo
// image of ncols rows of 128 bytes (64 pixels, 16-byte pieces XOR-swizzled by
// row & 7): row n = accumulator column n (Re / Im of Y_e for n = 2e / 2e+1).
struct TcYOut {
  const double* R = nullptr;
  unsigned char* Y = nullptr;
  int nc64 = 0;  // 64-pixel chunks of the image, ceil(n_pix / 64)
};

// Launch geometry of one batch.
struct TcPlan {
  bool fp16 = false;
  int ncols_max = 16;   // widest accumulator (2 * n_eig rounded to 16)
  int max_chunks = 1;   // most 32-station chunks of a step
  int ncols_buf = 32;   // TMEM columns per accumulator buffer (power of two)
  bool fused = false;   // A_hi [B_hi | B_lo] as one MMA of N = 2 ncols (ncols_max <= 128); autotuned
  int n_stages = 2;     // shared-memory ring depth
  bool epw = true;      // level images: dedicated epilogue warps (else the producers run the epilogue); autotuned
  bool tuned = false;   // n_stages, fused and epw come from the autotuner
};

int tc_alloc(TcWorkspace* w, int T, int N, int K);
void tc_free(TcWorkspace* w);
int tc_read_status(TcWorkspace* w);  // 0 or the device error word
// Fault injection for tests: while on, the synthesis kernel's MMA issuer waits
// on a barrier phase that nothing completes until its bounded wait runs out.
// Synchronous; 0, or -1 if the copy failed. No-op before the workspace exists.
int tc_set_fail_wait(TcWorkspace* w, int on);
// Host side: step table into pinned memory and the launch plan. Returns 0,
// -3 if some step has n_eig > kTcMaxEig, other negatives on capacity errors.
int tc_prepare(const std::vector<int>& nst, const std::vector<int>& neig, bool fp16, TcWorkspace* w, TcPlan* p);
// Stream-ordered (graph-capturable): step table upload, FP16 scales, operand packing.
int tc_enqueue_pack(const Batch& b, const TcPlan& p, TcWorkspace* w, cudaStream_t s);
// Stream-ordered (graph-capturable): the fused synthesis kernel.
int tc_enqueue_synth(const Batch& b, const Pixels& px, int n_level, double* img, const TcPlan& p, TcWorkspace* w,
                     cudaStream_t s);
// Stream-ordered: the adjoint's first stage (z recomputed on the tensor
// cores, Y = d R z written to yo.Y instead of level images); n_level <= 4 and
// a fused plan (2 n_eig <= 128 accumulator columns) only, else nonzero.
int tc_enqueue_yout(const Batch& b, const Pixels& px, int n_level, const TcPlan& p, TcWorkspace* w, TcYOut yo,
                    cudaStream_t s);
// The adjoint's pixel contraction on the tensor cores (adjoint_tc.cu):
// grad_W' (n_t blocks of n_eig x n_st complex128, e-major) from Y and the
// phase words (qph) of the packed batch; part is scratch of
// n_t * grid * 2 * n_st * ncols floats. n_eig <= 64. Stream-ordered.
int launch_adjoint_tc(const Pixels& px, int T, int n_st, int K, int ncols, const uint32_t* qph, int qph_stride,
                      const unsigned char* Y, int nc64, float* part, int grid, double2* gWp, int* status,
                      cudaStream_t s);
int adj_tc_smem_bytes(int ncols);
// The fused MMA shape (N = 2 ncols) whatever the tuner chose; needs
// 2 ncols_max <= 256 (else p stays unfused).
void tc_plan_force_fused(TcPlan* p);
// Not capturable (synchronises): time each feasible launch shape (MMA shape:
// fused N = 2 ncols or three N = ncols MMAs; stage-ring depth; epilogue in
// dedicated warps or in the producers, for level images) on a subset of
// the packed batch into a scratch image, keep the fastest in p and in a
// process-wide cache keyed by (ncols_max, chunk count rounded up to a power of
// two, operand type).
int tc_autotune(const Batch& b, const Pixels& px, int n_level, int n_chan_sub, TcPlan* p, TcWorkspace* w,
                cudaStream_t s);

}  // namespace bipp
