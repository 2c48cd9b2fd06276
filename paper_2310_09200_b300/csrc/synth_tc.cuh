// synth_tc.cuh — tcgen05 fused synthesis (split BF16 / FP16 hi+lo products on
// the 5th-generation tensor cores). Internal to libbipp_ss.so.
#pragma once

#include <stdint.h>

#include <vector>

#include "bipp_internal.cuh"

namespace bipp {

constexpr int kTcMaxEig = 128;  // eigenvectors per step on the tensor-core path (N = 2*K <= 256)

// Per-step geometry of the tensor-core GEMM: B operand chunks of 64 K-rows
// (32 stations) packed at b_off, n_chunks of them, ncols = 2*K rounded up to
// a multiple of 16, and the tcgen05 instruction descriptor.
struct TcStep {
  long long b_off;
  int n_chunks;
  int ncols;
  uint32_t idesc;
  int pad;
};

// Device workspace of the tensor-core path.
struct TcWorkspace {
  unsigned char* B = nullptr;  // packed, pre-swizzled hi/lo operand chunks of every step
  size_t B_bytes = 0;
  TcStep* steps = nullptr;     // [cap_T]
  float* scale = nullptr;      // [cap_T] operand scale of the FP16 variant (W * scale)
  int* status = nullptr;       // [1] device error word (0 = ok)
  int cap_T = 0;
};

int tc_alloc(TcWorkspace* w, int T, int N, int K);
void tc_free(TcWorkspace* w);
int tc_read_status(TcWorkspace* w);  // 0 or the device error word
// Returns 0, or a negative value if the batch exceeds the path's limits
// (n_eig > kTcMaxEig) or a CUDA call failed.
int launch_synth_tc(const Batch& b, const std::vector<int>& nst, const std::vector<int>& neig, const Pixels& px,
                    int n_level, double* img, bool fp16, TcWorkspace* w, cudaStream_t s);

}  // namespace bipp
