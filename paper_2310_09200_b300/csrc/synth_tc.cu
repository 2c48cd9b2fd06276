// synth_tc.cu — tcgen05 synthesis path: not built yet; every launch reports
// failure so that the split precisions return an error instead of running.
#include "synth_tc.cuh"

namespace bipp {

int tc_alloc(TcWorkspace* w, int T, int N, int K) {
  w->cap_T = T; w->cap_N = N; w->cap_K = K;
  return 0;
}
void tc_free(TcWorkspace* w) { *w = TcWorkspace{}; }
int tc_read_status(TcWorkspace*) { return 0; }
int launch_synth_tc(const Batch&, const Pixels&, int, double*, bool, TcWorkspace*, cudaStream_t) { return -1; }

}  // namespace bipp
