// synth_tc.cuh — tcgen05 fused synthesis (split BF16 / FP16 hi+lo products on
// the 5th-generation tensor cores). Internal to libbipp_ss.so.
#pragma once

#include "bipp_internal.cuh"

namespace bipp {

// Device workspace of the tensor-core path: packed hi/lo B operands per step
// and a status word for the bounded mbarrier waits.
struct TcWorkspace {
  void* B = nullptr;       // packed operand tiles
  size_t B_bytes = 0;
  float* scale = nullptr;  // [T] per-step operand scale (FP16 variant)
  int* status = nullptr;   // [1] device error word (0 = ok)
  int cap_T = 0, cap_N = 0, cap_K = 0;
};

int tc_alloc(TcWorkspace* w, int T, int N, int K);
void tc_free(TcWorkspace* w);
int tc_read_status(TcWorkspace* w);  // 0 or a nonzero device error code
int launch_synth_tc(const Batch& b, const Pixels& px, int n_level, double* img, bool fp16, TcWorkspace* w,
                    cudaStream_t s);

}  // namespace bipp
