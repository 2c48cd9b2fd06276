// api.cu — the C ABI of libbipp_ss.so (declared in include/bipp_ss.h).
//
// A handle is the paper's StandardSynthesis imaging object (Sec. 3.1),
// generalised to n_chan frequency channels that share one pixel grid: it
// holds the pixels, per-channel wavelengths, level intervals and level
// images on one device, plus a batch workspace that grows to the largest
// batch seen. collect() runs Algorithm 1 for a batch of steps (any mix of
// channels, ragged station counts and n_eig) as one stream-ordered chain of
// kernels with no host round trip until the final status check; the
// synthesis kernels read a device flag and commit nothing if any step of the
// batch failed. A batch geometry seen a second time is captured into a CUDA
// graph and replayed from then on.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "bipp_internal.cuh"
#include "bipp_ss.h"
#include "nufft.cuh"
#include "synth_tc.cuh"

using namespace bipp;

namespace {

// Everything that determines the kernels and arguments of a batch.
struct GraphKey {
  int T = 0, N = 0, K = 0;
  const void* st = nullptr;
  const void* vis = nullptr;
  cudaStream_t stream = nullptr;
  std::vector<int> nst, neig, chan;
  int n_stages = 0;
  bool operator==(const GraphKey& o) const {
    return T == o.T && N == o.N && K == o.K && st == o.st && vis == o.vis && stream == o.stream && nst == o.nst &&
           neig == o.neig && chan == o.chan && n_stages == o.n_stages;
  }
};

}  // namespace

struct bipp_ss {
  int device = 0;
  cudaStream_t stream = nullptr;
  int64_t n_pix = 0;
  int n_level = 0;
  int n_chan = 1;
  std::vector<double> wl;      // [n_chan]
  bipp_ss_options opt{};
  double* d_pix = nullptr;     // [3][n_pix]
  float* d_pix_hl = nullptr;   // [6][n_pix]
  double* d_img = nullptr;     // [n_chan][n_level][n_pix]
  double* d_bounds = nullptr;  // [n_chan][2][n_level]
  // batch workspace
  int cap_T = 0, cap_N = 0, cap_K = 0;
  double* d_st = nullptr;
  double2* d_vis = nullptr;
  double* d_G = nullptr;
  double* d_Linv = nullptr;
  double2* d_X = nullptr;
  double2* d_C = nullptr;
  double2* d_Q = nullptr;
  double* d_mu = nullptr;
  int* d_status = nullptr;
  int* d_sweeps = nullptr;
  int* d_nkept = nullptr;
  double* d_sel_mu = nullptr;
  int* d_level = nullptr;
  double* d_wt = nullptr;
  double2* d_W64 = nullptr;
  float2* d_W32 = nullptr;
  float* d_q = nullptr;
  int* d_nst = nullptr;
  int* d_order = nullptr;  // [T] steps by descending station count (Batch::order)
  int* d_neig = nullptr;
  int* d_chan = nullptr;
  double* d_wl = nullptr;
  int* d_flag = nullptr;
  // pinned host staging of the per-step tables (sources of graph memcpy nodes)
  int* h_nst = nullptr;
  int* h_order = nullptr;
  int* h_neig = nullptr;
  int* h_chan = nullptr;
  double* h_wl = nullptr;
  TcWorkspace tc{};
  MixedWs mx{};
  int mixed_kp = 0;  // KP of the current batch when the mixed eigensolver runs, else 0
  int fail_wait = 0; // fault injection into the tensor-core kernel's bounded waits (tests)
  // NUFFT synthesis: pixel box, kernel, and the current batch's per-channel plans
  NuPixCells nu_cells;     // image cells (pixels sorted by cell, ranges, boxes)
  int* d_nu_order = nullptr;  // the sorted pixel order on the device
  int nu_w = 0;
  float nu_beta = 0.f;
  NufftWs nu;
  std::vector<NuPlan> nu_plans;
  std::vector<int> nu_t0;  // first step of each channel group, plus n_t at the end
  std::vector<double> nu_st;  // host copy of device station coordinates
  int nu_launches = 0;
  cudaEvent_t nu_ev[8] = {};
  double nu_timings[11] = {};
  // graph cache: the last geometry seen, and the captured graph of it
  GraphKey last_key;
  bool have_key = false;
  GraphKey graph_key;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // the batch before and from the reduction on
  // host-buffer collects: the visibilities' upload runs on copy_stream while the
  // Gram matrix, its Cholesky factor and inverse (which do not read them) run
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t vis_ready = nullptr, ev_order = nullptr;
  bool vis_pending = false;
  // last batch
  int last_T = 0, last_N = 0, last_K = 0;
  double timings[6] = {0, 0, 0, 0, 0, 0};
  int synth_shape[4] = {0, 0, 0, 0};  // bipp_ss_get_synth_shape
  cudaEvent_t ev[5] = {};
  std::string err;
};

// per calling thread, so that creates on distinct threads do not share it
static thread_local std::string g_create_err = "no error";

// Error message of calls without a handle (create, the estimation functions).
int bipp::set_global_error(int code, const char* msg) {
  g_create_err = msg;
  return code;
}

static int fail(bipp_ss* h, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (h) h->err = buf; else g_create_err = buf;
  return code;
}

#define CUDA_TRY(h, call)                                                                        \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) {                                                                     \
      return fail((h), e_ == cudaErrorMemoryAllocation ? BIPP_ERR_OUT_OF_MEMORY : BIPP_ERR_CUDA, \
                  "%s failed: %s", #call, cudaGetErrorString(e_));                               \
    }                                                                                            \
  } while (0)

template <typename T>
static cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc((void**)p, count * sizeof(T));
}

static void drop_graph(bipp_ss* h) {
  for (auto& g : h->graph) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
  h->have_key = false;
}

static void free_batch(bipp_ss* h) {
  drop_graph(h);
  void* ptrs[] = {h->d_st, h->d_vis, h->d_G, h->d_Linv, h->d_X, h->d_C, h->d_Q, h->d_mu, h->d_status,
                  h->d_sweeps, h->d_nkept, h->d_sel_mu, h->d_level, h->d_wt, h->d_W64, h->d_W32, h->d_q,
                  h->d_nst, h->d_order, h->d_neig, h->d_chan, h->d_wl, h->d_flag, h->mx.kp, h->mx.lam, h->mx.tnorm, h->mx.theta,
                  h->mx.rnorm, h->mx.cnorm, h->mx.st2, h->mx.sw2};
  for (void* p : ptrs) if (p) cudaFree(p);
  h->mx = MixedWs{};
  void* hp[] = {h->h_nst, h->h_order, h->h_neig, h->h_chan, h->h_wl};
  for (void* p : hp) if (p) cudaFreeHost(p);
  h->d_st = nullptr; h->d_vis = nullptr; h->d_G = nullptr; h->d_Linv = nullptr; h->d_X = nullptr;
  h->d_C = nullptr; h->d_Q = nullptr; h->d_mu = nullptr; h->d_status = nullptr; h->d_sweeps = nullptr;
  h->d_nkept = nullptr; h->d_sel_mu = nullptr; h->d_level = nullptr; h->d_wt = nullptr; h->d_W64 = nullptr;
  h->d_W32 = nullptr; h->d_q = nullptr; h->d_nst = nullptr; h->d_order = nullptr; h->d_neig = nullptr; h->d_chan = nullptr;
  h->d_wl = nullptr; h->d_flag = nullptr;
  h->h_nst = nullptr; h->h_order = nullptr; h->h_neig = nullptr; h->h_chan = nullptr; h->h_wl = nullptr;
  tc_free(&h->tc);
  h->cap_T = h->cap_N = h->cap_K = 0;
}

static int ensure_batch(bipp_ss* h, int T, int N, int K) {
  if (T <= h->cap_T && N <= h->cap_N && K <= h->cap_K) return BIPP_OK;
  T = std::max(T, h->cap_T);
  N = std::max(N, h->cap_N);
  K = std::max(K, h->cap_K);
  free_batch(h);
  const size_t NN = (size_t)N * N;
  CUDA_TRY(h, dalloc(&h->d_st, (size_t)T * 3 * N));
  CUDA_TRY(h, dalloc(&h->d_vis, (size_t)T * NN));
  CUDA_TRY(h, dalloc(&h->d_G, (size_t)T * NN));
  CUDA_TRY(h, dalloc(&h->d_Linv, (size_t)T * NN));
  CUDA_TRY(h, dalloc(&h->d_X, (size_t)T * NN));
  CUDA_TRY(h, dalloc(&h->d_C, (size_t)T * NN));
  CUDA_TRY(h, dalloc(&h->d_Q, (size_t)T * NN));
  CUDA_TRY(h, dalloc(&h->d_mu, (size_t)T * N));
  CUDA_TRY(h, dalloc(&h->d_status, (size_t)T));
  CUDA_TRY(h, dalloc(&h->d_sweeps, (size_t)T));
  CUDA_TRY(h, dalloc(&h->d_nkept, (size_t)T));
  CUDA_TRY(h, dalloc(&h->d_sel_mu, (size_t)T * K));
  CUDA_TRY(h, dalloc(&h->d_level, (size_t)T * K));
  CUDA_TRY(h, dalloc(&h->d_wt, (size_t)T * K));
  CUDA_TRY(h, dalloc(&h->d_W64, (size_t)T * K * N));
  CUDA_TRY(h, dalloc(&h->d_W32, (size_t)T * K * N));
  CUDA_TRY(h, dalloc(&h->d_q, (size_t)T * 6 * N));
  CUDA_TRY(h, dalloc(&h->d_nst, (size_t)T));
  CUDA_TRY(h, dalloc(&h->d_order, (size_t)T));
  CUDA_TRY(h, dalloc(&h->d_neig, (size_t)T));
  CUDA_TRY(h, dalloc(&h->d_chan, (size_t)T));
  CUDA_TRY(h, dalloc(&h->d_wl, (size_t)T));
  CUDA_TRY(h, dalloc(&h->d_flag, 1));
  CUDA_TRY(h, dalloc(&h->mx.kp, (size_t)T));
  CUDA_TRY(h, dalloc(&h->mx.lam, (size_t)T * N));
  CUDA_TRY(h, dalloc(&h->mx.tnorm, (size_t)T));
  CUDA_TRY(h, dalloc(&h->mx.theta, (size_t)T * N));
  CUDA_TRY(h, dalloc(&h->mx.rnorm, (size_t)T * N));
  CUDA_TRY(h, dalloc(&h->mx.cnorm, (size_t)T));
  CUDA_TRY(h, dalloc(&h->mx.st2, (size_t)T));
  CUDA_TRY(h, dalloc(&h->mx.sw2, (size_t)T));
  CUDA_TRY(h, cudaMallocHost(&h->h_nst, sizeof(int) * T));
  CUDA_TRY(h, cudaMallocHost(&h->h_order, sizeof(int) * T));
  CUDA_TRY(h, cudaMallocHost(&h->h_neig, sizeof(int) * T));
  CUDA_TRY(h, cudaMallocHost(&h->h_chan, sizeof(int) * T));
  CUDA_TRY(h, cudaMallocHost(&h->h_wl, sizeof(double) * T));
  if (tc_alloc(&h->tc, T, N, K)) return fail(h, BIPP_ERR_OUT_OF_MEMORY, "tensor-core workspace allocation failed");
  if (h->fail_wait && tc_set_fail_wait(&h->tc, 1)) return fail(h, BIPP_ERR_CUDA, "fault-injection word");
  h->cap_T = T;
  h->cap_N = N;
  h->cap_K = K;
  return BIPP_OK;
}

static Batch make_batch(bipp_ss* h, int T, int N, int K, const double* st, const double2* vis) {
  Batch b;
  b.T = T; b.n_max = N; b.k_max = K;
  b.nst = h->d_nst; b.neig = h->d_neig; b.wl = h->d_wl; b.chan = h->d_chan; b.order = h->d_order;
  b.st = st; b.vis = vis;
  b.G = h->d_G; b.Linv = h->d_Linv; b.X = h->d_X; b.C = h->d_C; b.Q = h->d_Q; b.mu = h->d_mu;
  b.status = h->d_status; b.sweeps = h->d_sweeps; b.nkept = h->d_nkept;
  b.sel_mu = h->d_sel_mu; b.level = h->d_level; b.wt = h->d_wt; b.W64 = h->d_W64; b.W32 = h->d_W32;
  b.q = h->d_q; b.flag = h->d_flag;
  b.eigen = h->opt.eigenimages;
  return b;
}

extern "C" void bipp_ss_default_options(bipp_ss_options* opt) {
  if (!opt) return;
  memset(opt, 0, sizeof(*opt));
  opt->n_eig = 0;
  opt->precision = BIPP_PREC_FP32;
  opt->filter = BIPP_FILTER_LSQ;
  opt->gram_identity = 0;
  opt->max_jacobi_sweeps = 40;
  opt->jacobi_tol = 1e-13;
  opt->device = -1;
  opt->eig_mode = BIPP_EIG_JACOBI64;
  opt->use_graph = 1;
  opt->autotune = 1;
  opt->synthesis = BIPP_SYNTH_STANDARD;
  opt->nufft_eps = 1e-5;
  for (int i = 0; i < 6; ++i) opt->nufft_partition[i] = 1;
}

extern "C" int bipp_ss_destroy(bipp_ss_t h) {
  if (!h) return BIPP_OK;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  free_batch(h);
  nu_free(&h->nu);
  if (h->d_nu_order) cudaFree(h->d_nu_order);
  if (h->d_pix) cudaFree(h->d_pix);
  if (h->d_pix_hl) cudaFree(h->d_pix_hl);
  if (h->d_img) cudaFree(h->d_img);
  if (h->d_bounds) cudaFree(h->d_bounds);
  for (auto& e : h->ev) if (e) cudaEventDestroy(e);
  for (auto& e : h->nu_ev) if (e) cudaEventDestroy(e);
  if (h->vis_ready) cudaEventDestroy(h->vis_ready);
  if (h->ev_order) cudaEventDestroy(h->ev_order);
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  if (h->stream) cudaStreamDestroy(h->stream);
  delete h;
  return BIPP_OK;
}

extern "C" int bipp_ss_create_channels(bipp_ss_t* out, int64_t n_pix, const double* pix_xyz, int32_t n_chan,
                                       const double* wl, int32_t n_level, const double* level_bounds,
                                       const bipp_ss_options* opt) {
  if (!out) return fail(nullptr, BIPP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n_pix < 1 || !pix_xyz) return fail(nullptr, BIPP_ERR_INVALID_ARG, "need n_pix >= 1 and pix_xyz");
  if (n_chan < 1 || n_chan > 4096 || !wl) return fail(nullptr, BIPP_ERR_INVALID_ARG, "need 1 <= n_chan <= 4096 and wl");
  for (int c = 0; c < n_chan; ++c)
    if (!(wl[c] > 0.0) || !isfinite(wl[c]))
      return fail(nullptr, BIPP_ERR_INVALID_ARG, "wavelength of channel %d must be finite and > 0", c);
  bipp_ss_options o;
  if (opt) o = *opt; else bipp_ss_default_options(&o);
  for (int i = 0; i < 2; ++i)
    if (o.reserved[i]) return fail(nullptr, BIPP_ERR_INVALID_ARG, "reserved option fields must be zero");
  for (int i = 0; i < 6; ++i)
    if (o.nufft_partition[i] < 1 || o.nufft_partition[i] > 64)
      return fail(nullptr, BIPP_ERR_INVALID_ARG, "nufft_partition[%d] must be in [1, 64]", i);
  if (o.synthesis != BIPP_SYNTH_STANDARD && o.synthesis != BIPP_SYNTH_NUFFT)
    return fail(nullptr, BIPP_ERR_INVALID_ARG, "unknown synthesis %d", o.synthesis);
  int nu_w = 0;
  float nu_beta = 0.f;
  if (o.synthesis == BIPP_SYNTH_NUFFT) {
    if (!nu_kernel_params(o.nufft_eps, &nu_w, &nu_beta))
      return fail(nullptr, BIPP_ERR_INVALID_ARG, "nufft_eps must be in [1e-7, 0.1]");
    if (o.eigenimages) return fail(nullptr, BIPP_ERR_UNSUPPORTED, "NUFFT synthesis makes level images, not eigenimages");
    if (n_pix >= ((int64_t)1 << 31)) return fail(nullptr, BIPP_ERR_UNSUPPORTED, "NUFFT synthesis needs n_pix < 2^31");
  }
  if (o.eigenimages != 0 && o.eigenimages != 1)
    return fail(nullptr, BIPP_ERR_INVALID_ARG, "eigenimages must be 0 or 1");
  if (o.eigenimages) {
    if (o.n_eig < 1 || o.n_eig > kMaxEigenimages || n_level != o.n_eig)
      return fail(nullptr, BIPP_ERR_INVALID_ARG, "eigenimages need 1 <= n_eig <= %d and n_level == n_eig",
                  kMaxEigenimages);
  } else if (n_level < 1 || n_level > kMaxLevels || !level_bounds) {
    return fail(nullptr, BIPP_ERR_INVALID_ARG, "need 1 <= n_level <= %d and level_bounds", kMaxLevels);
  }
  if (o.precision < BIPP_PREC_FP64 || o.precision > BIPP_PREC_SPLIT_FP16)
    return fail(nullptr, BIPP_ERR_INVALID_ARG, "unknown precision %d", o.precision);
  if (o.filter != BIPP_FILTER_LSQ && o.filter != BIPP_FILTER_STD)
    return fail(nullptr, BIPP_ERR_INVALID_ARG, "unknown filter %d", o.filter);
  if (o.eig_mode != BIPP_EIG_JACOBI64 && o.eig_mode != BIPP_EIG_MIXED)
    return fail(nullptr, BIPP_ERR_INVALID_ARG, "unknown eig_mode %d", o.eig_mode);
  if (o.n_eig < 0 || o.max_jacobi_sweeps < 1 || !(o.jacobi_tol > 0.0))
    return fail(nullptr, BIPP_ERR_INVALID_ARG, "bad n_eig / max_jacobi_sweeps / jacobi_tol");
  for (int64_t i = 0; !o.eigenimages && i < (int64_t)2 * n_level * n_chan; ++i)
    if (isnan(level_bounds[i])) return fail(nullptr, BIPP_ERR_INVALID_ARG, "level bound %lld is NaN", (long long)i);
  for (int64_t i = 0; i < 3 * n_pix; ++i)
    if (!isfinite(pix_xyz[i]))
      return fail(nullptr, BIPP_ERR_INVALID_ARG, "pixel coordinate %lld is not finite", (long long)i);

  (void)cudaGetLastError();  // errors of earlier, unrelated calls are not ours to report
  bipp_ss* h = new bipp_ss();
  h->opt = o;
  h->n_pix = n_pix;
  h->n_level = n_level;
  h->n_chan = n_chan;
  h->wl.assign(wl, wl + n_chan);
  h->nu_w = nu_w;
  h->nu_beta = nu_beta;
  if (o.synthesis == BIPP_SYNTH_NUFFT) h->nu_cells = nu_pixel_cells(pix_xyz, n_pix, o.nufft_partition + 3);
  if (o.device >= 0 && cudaSetDevice(o.device) != cudaSuccess) {
    delete h;
    return fail(nullptr, BIPP_ERR_CUDA, "cudaSetDevice(%d) failed", o.device);
  }
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return fail(nullptr, BIPP_ERR_CUDA, "no CUDA device");
  }
  auto bail = [&](int code, const char* what, cudaError_t e) {
    fail(nullptr, code, "%s: %s", what, cudaGetErrorString(e));
    bipp_ss_destroy(h);
    return code;
  };
  const size_t n_img = (size_t)n_chan * n_level * n_pix;
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking)) != cudaSuccess) return bail(BIPP_ERR_CUDA, "stream", e);
  for (auto& ev : h->ev)
    if ((e = cudaEventCreate(&ev)) != cudaSuccess) return bail(BIPP_ERR_CUDA, "event", e);
  for (auto& ev : h->nu_ev)
    if ((e = cudaEventCreate(&ev)) != cudaSuccess) return bail(BIPP_ERR_CUDA, "event", e);
  if ((e = cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return bail(BIPP_ERR_CUDA, "stream", e);
  if ((e = cudaEventCreateWithFlags(&h->vis_ready, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&h->ev_order, cudaEventDisableTiming)) != cudaSuccess)
    return bail(BIPP_ERR_CUDA, "event", e);
  if ((e = dalloc(&h->d_pix, (size_t)3 * n_pix)) != cudaSuccess) return bail(BIPP_ERR_OUT_OF_MEMORY, "pixels", e);
  if ((e = dalloc(&h->d_pix_hl, (size_t)6 * n_pix)) != cudaSuccess) return bail(BIPP_ERR_OUT_OF_MEMORY, "pixels", e);
  if ((e = dalloc(&h->d_img, n_img)) != cudaSuccess) return bail(BIPP_ERR_OUT_OF_MEMORY, "images", e);
  if ((e = dalloc(&h->d_bounds, (size_t)2 * n_level * n_chan)) != cudaSuccess) return bail(BIPP_ERR_OUT_OF_MEMORY, "bounds", e);
  if ((e = cudaMemcpy(h->d_pix, pix_xyz, sizeof(double) * 3 * n_pix, cudaMemcpyHostToDevice)) != cudaSuccess)
    return bail(BIPP_ERR_CUDA, "pixel upload", e);
  if (o.synthesis == BIPP_SYNTH_NUFFT) {
    if ((e = dalloc(&h->d_nu_order, (size_t)n_pix)) != cudaSuccess) return bail(BIPP_ERR_OUT_OF_MEMORY, "pixel order", e);
    if ((e = cudaMemcpy(h->d_nu_order, h->nu_cells.order.data(), sizeof(int) * n_pix, cudaMemcpyHostToDevice)) !=
        cudaSuccess)
      return bail(BIPP_ERR_CUDA, "pixel order upload", e);
  }
  if (o.eigenimages) {  // levels are ranks; the bounds are unused
    if ((e = cudaMemset(h->d_bounds, 0, sizeof(double) * 2 * n_level * n_chan)) != cudaSuccess)
      return bail(BIPP_ERR_CUDA, "bounds", e);
  } else if ((e = cudaMemcpy(h->d_bounds, level_bounds, sizeof(double) * 2 * n_level * n_chan,
                             cudaMemcpyHostToDevice)) != cudaSuccess) {
    return bail(BIPP_ERR_CUDA, "bounds upload", e);
  }
  if ((e = cudaMemset(h->d_img, 0, sizeof(double) * n_img)) != cudaSuccess) return bail(BIPP_ERR_CUDA, "memset", e);
  launch_pixel_split(h->d_pix, h->d_pix_hl, n_pix, h->stream);
  if ((e = cudaGetLastError()) != cudaSuccess) return bail(BIPP_ERR_CUDA, "pixel split launch", e);
  if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return bail(BIPP_ERR_CUDA, "pixel split", e);
  *out = h;
  return BIPP_OK;
}

extern "C" int bipp_ss_create(bipp_ss_t* out, int64_t n_pix, const double* pix_xyz, double wl, int32_t n_level,
                              const double* level_bounds, const bipp_ss_options* opt) {
  return bipp_ss_create_channels(out, n_pix, pix_xyz, 1, &wl, n_level, level_bounds, opt);
}

// Validate the ragged batch description; returns K_max or a negative code.
static int check_sizes(bipp_ss* h, int n_t, int n_st_max, const int32_t* chan, const int32_t* n_st,
                       const int32_t* n_eig, std::vector<int>& nst_v, std::vector<int>& neig_v,
                       std::vector<int>& chan_v) {
  if (n_t < 1) return fail(h, BIPP_ERR_INVALID_ARG, "n_t must be >= 1");
  if (n_st_max < 1 || n_st_max > kMaxStations)
    return fail(h, BIPP_ERR_UNSUPPORTED, "n_st_max must be in [1, %d]", kMaxStations);
  if (!n_st) return fail(h, BIPP_ERR_INVALID_ARG, "n_st is NULL");
  nst_v.resize(n_t);
  neig_v.resize(n_t);
  chan_v.resize(n_t);
  int kmax = 1;
  for (int t = 0; t < n_t; ++t) {
    const int n = n_st[t];
    if (n < 1 || n > n_st_max) return fail(h, BIPP_ERR_INVALID_ARG, "step %d: n_st=%d outside [1, %d]", t, n, n_st_max);
    const int k = n_eig ? n_eig[t] : (h->opt.n_eig > 0 ? h->opt.n_eig : n);
    if (k < 1) return fail(h, BIPP_ERR_INVALID_ARG, "step %d: n_eig=%d must be >= 1", t, k);
    if (k > n) return fail(h, BIPP_ERR_UNSUPPORTED, "step %d: n_eig=%d exceeds n_st=%d", t, k, n);
    if (h->opt.eigenimages && k > h->n_level)
      return fail(h, BIPP_ERR_INVALID_ARG, "step %d: n_eig=%d exceeds the handle's %d eigenimages", t, k, h->n_level);
    const int c = chan ? chan[t] : 0;
    if (c < 0 || c >= h->n_chan) return fail(h, BIPP_ERR_INVALID_ARG, "step %d: channel %d outside [0, %d)", t, c, h->n_chan);
    if (t > 0 && c < chan_v[t - 1])
      return fail(h, BIPP_ERR_INVALID_ARG, "steps must be grouped by channel in non-decreasing order (step %d)", t);
    if (h->opt.precision >= BIPP_PREC_SPLIT_BF16 && k > kTcMaxEig)
      return fail(h, BIPP_ERR_UNSUPPORTED, "step %d: split precisions support n_eig <= %d", t, kTcMaxEig);
    nst_v[t] = n;
    neig_v[t] = k;
    chan_v[t] = c;
    kmax = std::max(kmax, k);
  }
  return kmax;
}

// Stage-timing events: recorded as external event nodes when captured, so
// that they are also recorded when the graph is replayed.
static cudaError_t record(cudaEvent_t ev, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &cs);
  if (e != cudaSuccess) return e;
  return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal)
                                             : cudaEventRecord(ev, s);
}

// Everything between the per-step table upload and the synthesis: stream
// ordered, no host synchronisation, so it can be captured into graphs. Part 0
// (tables, Gram matrix, Cholesky factor and its inverse) does not read the
// visibilities; part 1 (reduction onwards) does.
static int enqueue_batch(bipp_ss* h, const Batch& b, const TcPlan& plan, cudaStream_t s, int part);

// Both parts, with the wait for a pending visibility upload between them.
static int enqueue_all(bipp_ss* h, const Batch& b, const TcPlan& plan, cudaStream_t s) {
  int rc = enqueue_batch(h, b, plan, s, 0);
  if (rc) return rc;
  if (h->vis_pending) CUDA_TRY(h, cudaStreamWaitEvent(s, h->vis_ready, 0));
  return enqueue_batch(h, b, plan, s, 1);
}

static int enqueue_batch(bipp_ss* h, const Batch& b, const TcPlan& plan, cudaStream_t s, int part) {
  const int T = b.T;
  const int gi = h->opt.gram_identity;
  if (part == 0) {
    CUDA_TRY(h, cudaMemcpyAsync(h->d_nst, h->h_nst, sizeof(int) * T, cudaMemcpyHostToDevice, s));
    CUDA_TRY(h, cudaMemcpyAsync(h->d_order, h->h_order, sizeof(int) * T, cudaMemcpyHostToDevice, s));
    CUDA_TRY(h, cudaMemcpyAsync(h->d_neig, h->h_neig, sizeof(int) * T, cudaMemcpyHostToDevice, s));
    CUDA_TRY(h, cudaMemcpyAsync(h->d_chan, h->h_chan, sizeof(int) * T, cudaMemcpyHostToDevice, s));
    CUDA_TRY(h, cudaMemcpyAsync(h->d_wl, h->h_wl, sizeof(double) * T, cudaMemcpyHostToDevice, s));
    CUDA_TRY(h, cudaMemsetAsync(h->d_status, 0, sizeof(int) * T, s));
    CUDA_TRY(h, cudaMemsetAsync(h->d_sweeps, 0, sizeof(int) * T, s));
    CUDA_TRY(h, cudaMemsetAsync(h->d_flag, 0, sizeof(int), s));
    CUDA_TRY(h, record(h->ev[0], s));
    launch_gram(b, gi, s);
    launch_cholesky(b, gi, s);
    return cudaGetLastError() == cudaSuccess ? BIPP_OK : fail(h, BIPP_ERR_CUDA, "Gram / Cholesky launch failed");
  }
  if (h->mixed_kp > 0) launch_reduce32(b, gi, s);  // FP32 C for the FP32 stage; the refinement factors C
  else launch_reduce(b, gi, s);
  CUDA_TRY(h, record(h->ev[1], s));
  if (h->mixed_kp > 0) {
    MixedWs w = h->mx;
    w.KP = h->mixed_kp;
    launch_eig_mixed(b, w, h->opt.jacobi_tol, h->opt.max_jacobi_sweeps, s);
  } else {
    launch_jacobi(b, h->opt.jacobi_tol, h->opt.max_jacobi_sweeps, s);
  }
  CUDA_TRY(h, record(h->ev[2], s));
  launch_select(b, h->n_level, h->d_bounds, h->opt.filter, s);
  const bool tc = h->opt.synthesis == BIPP_SYNTH_STANDARD && h->opt.precision >= BIPP_PREC_SPLIT_BF16;
  if (tc && tc_enqueue_pack(b, plan, &h->tc, s)) return fail(h, BIPP_ERR_CUDA, "operand packing launch failed");
  CUDA_TRY(h, record(h->ev[3], s));
  Pixels px{h->n_pix, h->d_pix, h->d_pix_hl};
  if (h->opt.synthesis == BIPP_SYNTH_NUFFT) {
    h->nu_launches = 0;
    const int nc = (int)h->nu_cells.box.size();
    bool first = true;
    for (size_t g = 0; g + 1 < h->nu_t0.size(); ++g) {
      const int t0 = h->nu_t0[g], t1 = h->nu_t0[g + 1];
      double* img = h->d_img + (size_t)h->h_chan[t0] * h->n_level * h->n_pix;
      for (int c = 0; c < nc; ++c) {
        const int64_t off = h->nu_cells.off[c], cnt = h->nu_cells.off[c + 1] - off;
        if (cnt == 0) continue;
        const int rc = nu_enqueue(b, t0, t1, h->nu_plans[g * nc + c], &h->nu, h->d_pix, h->n_pix, h->d_nu_order,
                                  off, cnt, c, nc, h->n_level, img, s, &h->nu_launches, first ? h->nu_ev : nullptr);
        first = false;
        if (rc == -1) return fail(h, BIPP_ERR_OUT_OF_MEMORY, "NUFFT grid allocation failed");
        if (rc == -2) return fail(h, BIPP_ERR_CUDA, "NUFFT: cuFFT plan or execution failed");
        if (rc) return fail(h, BIPP_ERR_CUDA, "NUFFT kernel launch failed");
      }
    }
    CUDA_TRY(h, cudaGetLastError());
    CUDA_TRY(h, record(h->ev[4], s));
    return BIPP_OK;
  }
  switch (h->opt.precision) {
    case BIPP_PREC_FP64: launch_synth_simt_f64(b, px, h->n_level, h->d_img, s); break;
    case BIPP_PREC_FP32: launch_synth_simt_f32(b, px, h->n_level, h->d_img, s); break;
    default:
      if (tc_enqueue_synth(b, px, h->n_level, h->d_img, plan, &h->tc, s))
        return fail(h, BIPP_ERR_CUDA, "tensor-core synthesis launch failed");
  }
  CUDA_TRY(h, cudaGetLastError());
  CUDA_TRY(h, record(h->ev[4], s));
  return BIPP_OK;
}

// NUFFT synthesis: one plan per channel group of the batch, from the host
// station coordinates (copied back when the caller passed device memory).
static int plan_nufft(bipp_ss* h, int n_t, int N, const std::vector<int>& nst_v, const std::vector<int>& chan_v,
                      const double* h_st, const double* d_st, cudaStream_t s) {
  if (!h_st) {
    h->nu_st.resize((size_t)n_t * 3 * N);
    CUDA_TRY(h, cudaMemcpyAsync(h->nu_st.data(), d_st, sizeof(double) * h->nu_st.size(), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(h, cudaStreamSynchronize(s));
    h_st = h->nu_st.data();
    // the grids are planned from these values: device positions are checked here
    for (int t = 0; t < n_t; ++t)
      for (int c = 0; c < 3; ++c)
        for (int i = 0; i < nst_v[t]; ++i)
          if (!isfinite(h_st[((size_t)t * 3 + c) * N + i]))
            return fail(h, BIPP_ERR_INVALID_ARG, "step %d: station %d coordinate %d is not finite", t, i, c);
  }
  h->nu_t0.clear();
  h->nu_plans.clear();
  std::vector<double> wl_t(n_t);
  for (int t = 0; t < n_t; ++t) wl_t[t] = h->wl[chan_v[t]];
  size_t need = 0;
  for (int t = 0; t < n_t; ++t)
    if (t == 0 || chan_v[t] != chan_v[t - 1]) h->nu_t0.push_back(t);
  h->nu_t0.push_back(n_t);
  const int nc = (int)h->nu_cells.box.size();
  size_t fine = 0;
  for (size_t g = 0; g + 1 < h->nu_t0.size(); ++g)
    for (int c = 0; c < nc; ++c) {
      const NuPlan p = nu_plan(h->nu_cells.box[c], h->nu_w, h->nu_beta, h->opt.nufft_partition, h_st, N,
                               nst_v.data(), wl_t.data(), h->nu_t0[g], h->nu_t0[g + 1]);
      h->nu_plans.push_back(p);
      if (h->nu_cells.off[c + 1] == h->nu_cells.off[c]) continue;  // empty image cell: no transform
      for (int d = 0; d < 3; ++d)
        if (p.M[d] > (1 << 28))
          return fail(h, BIPP_ERR_UNSUPPORTED, "NUFFT grid dimension %d needs %d points", d, p.M[d]);
      if ((size_t)p.parts() * p.cells() >= ((size_t)1 << 31))
        return fail(h, BIPP_ERR_UNSUPPORTED, "NUFFT grids of %d input cells x %zu points exceed 2^31 points",
                    p.parts(), p.cells());
      const size_t slots = (size_t)(h->nu_t0[g + 1] - h->nu_t0[g]) * N * (N - 1) / 2;
      need = std::max(need, nu_grid_bytes(p, h->n_level, slots));
      fine = std::max(fine, p.cells2() * sizeof(float2));
    }
  size_t free_b = 0, total_b = 0;
  CUDA_TRY(h, cudaMemGetInfo(&free_b, &total_b));
  const size_t have = (h->nu.F_cap + h->nu.G_cap + h->nu.G2_cap + h->nu.rc_cap) * sizeof(float2) +
                      (h->nu.rm_cap + h->nu.rf_cap) * sizeof(int4);
  // grids plus the FFT's workspace (of the order of the fine grid) must fit
  if (need + fine > free_b + have)
    return fail(h, BIPP_ERR_UNSUPPORTED,
                "NUFFT grids need %.1f GB but %.1f GB are free; partition the domain (nufft_partition), "
                "image a smaller field or collect fewer steps per batch",
                (need + fine) / 1e9, (free_b + have) / 1e9);
  return BIPP_OK;
}

static int run_batch(bipp_ss* h, int n_t, int N, const std::vector<int>& nst_v, const std::vector<int>& neig_v,
                     const std::vector<int>& chan_v, int K, const double* d_st, const double2* d_vis,
                     cudaStream_t s, const double* h_st) {
  (void)cudaGetLastError();  // errors of earlier, unrelated calls are not ours to report
  for (int t = 0; t < n_t; ++t) {
    h->h_nst[t] = nst_v[t];
    h->h_neig[t] = neig_v[t];
    h->h_chan[t] = chan_v[t];
    h->h_wl[t] = h->wl[chan_v[t]];
    h->h_order[t] = t;
  }
  std::stable_sort(h->h_order, h->h_order + n_t, [&](int x, int y) { return nst_v[x] > nst_v[y]; });
  Batch b = make_batch(h, n_t, N, K, d_st, d_vis);
  bool ident = true;  // steps already largest first (e.g. all of one size): no indirection in the kernels
  for (int t = 0; t < n_t; ++t) ident = ident && h->h_order[t] == t;
  if (ident) b.order = nullptr;
  // mixed-precision eigensolve when asked for and its scratch fits the batch buffers
  h->mixed_kp = 0;
  if (h->opt.eig_mode == BIPP_EIG_MIXED) {
    int kp = 1;
    for (int t = 0; t < n_t; ++t) kp = std::max(kp, std::min(nst_v[t], neig_v[t] + 16));
    if (eig_mixed_fits(N, kp)) h->mixed_kp = kp;
  }
  const bool nufft = h->opt.synthesis == BIPP_SYNTH_NUFFT;
  const bool tc = !nufft && h->opt.precision >= BIPP_PREC_SPLIT_BF16;
  if (nufft) {
    const int rc = plan_nufft(h, n_t, N, nst_v, chan_v, h_st, d_st, s);
    if (rc) return rc;
  }
  TcPlan plan;
  if (tc) {
    const int rc = tc_prepare(nst_v, neig_v, h->opt.precision == BIPP_PREC_SPLIT_FP16, &h->tc, &plan);
    if (rc == -3) return fail(h, BIPP_ERR_UNSUPPORTED, "split precisions support n_eig <= %d per step", kTcMaxEig);
    if (rc) return fail(h, BIPP_ERR_CUDA, "tensor-core plan failed (%d)", rc);
  }
  // the shape this collect's synthesis runs with (the tuning collect runs the default one)
  h->synth_shape[0] = tc ? plan.n_stages : 0;
  h->synth_shape[1] = tc && plan.fused ? 1 : 0;
  h->synth_shape[2] = tc && plan.epw && !h->opt.eigenimages ? 1 : 0;
  h->synth_shape[3] = tc && plan.tuned ? 1 : 0;
  GraphKey key;
  key.T = n_t; key.N = N; key.K = K; key.st = d_st; key.vis = d_vis; key.stream = s;
  key.nst = nst_v; key.neig = neig_v; key.chan = chan_v; key.n_stages = tc ? plan.n_stages + (plan.fused ? 16 : 0) + (plan.epw ? 32 : 0) : 0;

  if (nufft) {
    // host-planned grids and cuFFT: enqueued directly, not captured
    const int rc = enqueue_all(h, b, plan, s);
    if (rc) return rc;
  } else if (tc && h->opt.autotune && !plan.tuned) {
    // first batch of this accumulator width: run up to the packing, tune, then synthesise
    Batch bb = b;
    int rc = enqueue_all(h, bb, plan, s);  // ... runs the synthesis with the default plan too
    if (rc) return rc;
    CUDA_TRY(h, cudaStreamSynchronize(s));
    const int chan_sub = chan_v[std::min(n_t, 4) - 1] + 1;
    Pixels px{h->n_pix, h->d_pix, h->d_pix_hl};
    if (tc_autotune(b, px, h->n_level, chan_sub, &plan, &h->tc, s)) {
      cudaGetLastError();
      // keep the default stage count; tuning failure is not a collect failure
    }
  } else if (h->opt.use_graph && h->graph[0] && h->graph[1] && key == h->graph_key) {
    CUDA_TRY(h, cudaGraphLaunch(h->graph[0], s));
    if (h->vis_pending) CUDA_TRY(h, cudaStreamWaitEvent(s, h->vis_ready, 0));
    CUDA_TRY(h, cudaGraphLaunch(h->graph[1], s));
  } else if (h->opt.use_graph && h->have_key && key == h->last_key) {
    // second batch of the same geometry: capture once (two graphs, so that a pending
    // visibility upload can be waited for between them), replay from now on
    drop_graph(h);
    for (int part = 0; part < 2; ++part) {
      cudaGraph_t g = nullptr;
      CUDA_TRY(h, cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
      const int rc = enqueue_batch(h, b, plan, s, part);
      const cudaError_t ce = cudaStreamEndCapture(s, &g);
      if (rc) {
        if (g) cudaGraphDestroy(g);
        drop_graph(h);
        return rc;
      }
      if (ce != cudaSuccess) {
        drop_graph(h);
        return fail(h, BIPP_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ce));
      }
      const cudaError_t ie = cudaGraphInstantiate(&h->graph[part], g, 0);
      cudaGraphDestroy(g);
      if (ie != cudaSuccess) {
        h->graph[part] = nullptr;
        drop_graph(h);
        return fail(h, BIPP_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(ie));
      }
    }
    h->graph_key = key;
    CUDA_TRY(h, cudaGraphLaunch(h->graph[0], s));
    if (h->vis_pending) CUDA_TRY(h, cudaStreamWaitEvent(s, h->vis_ready, 0));
    CUDA_TRY(h, cudaGraphLaunch(h->graph[1], s));
  } else {
    const int rc = enqueue_all(h, b, plan, s);
    if (rc) return rc;
  }
  h->last_key = key;
  h->have_key = true;
  CUDA_TRY(h, cudaStreamSynchronize(s));
  h->last_T = n_t;
  h->last_N = N;
  h->last_K = K;
  float ms[4] = {0, 0, 0, 0};
  for (int i = 0; i < 4; ++i)
    if (cudaEventElapsedTime(&ms[i], h->ev[i], h->ev[i + 1]) != cudaSuccess) {
      ms[i] = NAN;
      (void)cudaGetLastError();  // a missing timing is not a collect failure
    }
  std::vector<int> status(n_t), sweeps(n_t);
  CUDA_TRY(h, cudaMemcpy(status.data(), h->d_status, sizeof(int) * n_t, cudaMemcpyDeviceToHost));
  CUDA_TRY(h, cudaMemcpy(sweeps.data(), h->d_sweeps, sizeof(int) * n_t, cudaMemcpyDeviceToHost));
  const int tc_status = tc ? tc_read_status(&h->tc) : 0;
  for (int i = 0; i < 4; ++i) h->timings[i] = ms[i];
  for (double& v : h->nu_timings) v = 0.0;
  if (nufft) {
    const int pairs[6][2] = {{0, 7}, {7, 1}, {2, 3}, {3, 4}, {4, 5}, {2, 6}};
    for (int i = 0; i < 6; ++i) {
      float v = 0.f;
      if (cudaEventElapsedTime(&v, h->nu_ev[pairs[i][0]], h->nu_ev[pairs[i][1]]) != cudaSuccess) {
        v = NAN;
        (void)cudaGetLastError();
      }
      h->nu_timings[i] = v;
    }
    for (int d = 0; d < 3; ++d) h->nu_timings[6 + d] = h->nu_plans[0].M[d];
    h->nu_timings[9] = h->nu_plans[0].w;
    double pairs_spread = 0;
    for (int t = h->nu_t0[0]; t < h->nu_t0[1]; ++t) pairs_spread += 0.5 * (double)nst_v[t] * (nst_v[t] - 1);
    h->nu_timings[10] = pairs_spread;
  }
  h->timings[4] = 0;
  for (int t = 0; t < n_t; ++t) h->timings[4] += sweeps[t];
  // gram, [cholesky], trinv, reduction (G = I: 1; mixed: 2 FP32 GEMMs; else 2 GEMMs + hermitize),
  // eigensolve (Jacobi: 1; mixed: kMixedLaunches), select, [scale], [pack], synthesis
  {
    const bool gi = h->opt.gram_identity != 0, mixed = h->mixed_kp > 0;
    h->timings[5] = 1 + (gi ? 0 : 1) + 1 + (gi ? 1 : (mixed ? 2 : 3)) + (mixed ? kMixedLaunches : 1) + 2 +
                    (tc ? 1 + (h->opt.precision == BIPP_PREC_SPLIT_FP16) : 0) + (nufft ? h->nu_launches - 1 : 0);
  }
  for (int t = 0; t < n_t; ++t) {
    if (status[t] & kStatusNotPD)
      return fail(h, BIPP_ERR_GRAM_NOT_PD, "step %d: Gram matrix is not positive definite (Cholesky pivot <= 0 or NaN)", t);
    if (status[t] & kStatusNotConverged)
      return h->mixed_kp > 0
                 ? fail(h, BIPP_ERR_EIG_NOT_CONVERGED,
                        "step %d: mixed eigensolver did not converge (refinement Jacobi sweep cap %d, "
                        "or a kept residual above 1e3 * jacobi_tol * ||C||_F)",
                        t, h->opt.max_jacobi_sweeps)
                 : fail(h, BIPP_ERR_EIG_NOT_CONVERGED, "step %d: Jacobi did not converge in %d sweeps", t,
                        h->opt.max_jacobi_sweeps);
    if (status[t] & kStatusRange)
      return fail(h, BIPP_ERR_UNSUPPORTED,
                  "step %d: a station lies 2^28 wavelengths or more from the origin (beyond the range of the "
                  "tensor-core synthesis phase)", t);
  }
  if (tc_status) return fail(h, BIPP_ERR_DEVICE_TIMEOUT, "tensor-core synthesis: bounded wait gave up (code %d)", tc_status);
  return BIPP_OK;
}

// on_device: the inputs are device memory; vis_c64: (device only) the
// visibilities are complex64 and are widened into the batch buffer first.
static int collect_common(bipp_ss_t h, int32_t n_t, int32_t n_st_max, const int32_t* chan, const int32_t* n_st,
                          const int32_t* n_eig, const double* st_xyz, const void* vis, int on_device,
                          void* stream, int vis_c64 = 0) {
  if (!h) return fail(nullptr, BIPP_ERR_INVALID_ARG, "handle is NULL");
  if (!st_xyz || !vis) return fail(h, BIPP_ERR_INVALID_ARG, "st_xyz / vis is NULL");
  std::vector<int> nst_v, neig_v, chan_v;
  const int K = check_sizes(h, n_t, n_st_max, chan, n_st, n_eig, nst_v, neig_v, chan_v);
  if (K < 0) return K;
  CUDA_TRY(h, cudaSetDevice(h->device));
  if (on_device) {
    cudaPointerAttributes a1{}, a2{};
    if (cudaPointerGetAttributes(&a1, st_xyz) != cudaSuccess || cudaPointerGetAttributes(&a2, vis) != cudaSuccess ||
        a1.type != cudaMemoryTypeDevice || a2.type != cudaMemoryTypeDevice || a1.device != h->device ||
        a2.device != h->device) {
      cudaGetLastError();
      return fail(h, BIPP_ERR_INVALID_ARG, "st_xyz and vis must be device memory on device %d", h->device);
    }
    // the kernels load doubles and complex pairs
    if ((reinterpret_cast<uintptr_t>(st_xyz) & 7) || (reinterpret_cast<uintptr_t>(vis) & (vis_c64 ? 7 : 15)))
      return fail(h, BIPP_ERR_INVALID_ARG, "d_st_xyz must be 8-byte and d_vis %d-byte aligned", vis_c64 ? 8 : 16);
  } else {
    for (int t = 0; t < n_t; ++t)
      for (int c = 0; c < 3; ++c)
        for (int i = 0; i < nst_v[t]; ++i)
          if (!isfinite(st_xyz[((size_t)t * 3 + c) * n_st_max + i]))
            return fail(h, BIPP_ERR_INVALID_ARG, "step %d: station %d coordinate %d is not finite", t, i, c);
  }
  int rc = ensure_batch(h, n_t, n_st_max, K);
  if (rc) return rc;
  if (on_device) {
    cudaStream_t s = stream ? (cudaStream_t)stream : h->stream;
    const double2* d_vis = reinterpret_cast<const double2*>(vis);
    if (vis_c64) {  // stream-ordered after the caller's writes; the batch then reads the widened copy
      launch_vis_widen(reinterpret_cast<const float2*>(vis), h->d_vis, (size_t)n_t * n_st_max * n_st_max, s);
      CUDA_TRY(h, cudaGetLastError());
      d_vis = h->d_vis;
    }
    return run_batch(h, n_t, n_st_max, nst_v, neig_v, chan_v, K, st_xyz, d_vis, s, nullptr);
  }
  const size_t N = (size_t)n_st_max;
  CUDA_TRY(h, cudaMemcpyAsync(h->d_st, st_xyz, sizeof(double) * 3 * N * n_t, cudaMemcpyHostToDevice, h->stream));
  // the visibilities on the copy stream, after the stream's earlier work (which may read d_vis)
  CUDA_TRY(h, cudaEventRecord(h->ev_order, h->stream));
  CUDA_TRY(h, cudaStreamWaitEvent(h->copy_stream, h->ev_order, 0));
  CUDA_TRY(h, cudaMemcpyAsync(h->d_vis, vis, sizeof(double2) * N * N * n_t, cudaMemcpyHostToDevice, h->copy_stream));
  CUDA_TRY(h, cudaEventRecord(h->vis_ready, h->copy_stream));
  h->vis_pending = true;
  const int rb = run_batch(h, n_t, n_st_max, nst_v, neig_v, chan_v, K, h->d_st, h->d_vis, h->stream, st_xyz);
  h->vis_pending = false;
  if (rb) cudaStreamSynchronize(h->copy_stream);  // no upload may outlive a failed collect
  return rb;
}

extern "C" int bipp_ss_collect_batch(bipp_ss_t h, int32_t n_t, int32_t n_st_max, const int32_t* n_st,
                                     const int32_t* n_eig, const double* st_xyz, const double* vis) {
  return collect_common(h, n_t, n_st_max, nullptr, n_st, n_eig, st_xyz, vis, 0, nullptr);
}

extern "C" int bipp_ss_collect(bipp_ss_t h, int32_t n_st, const double* st_xyz, const double* vis) {
  return bipp_ss_collect_batch(h, 1, n_st, &n_st, nullptr, st_xyz, vis);
}

extern "C" int bipp_ss_collect_device(bipp_ss_t h, int32_t n_t, int32_t n_st_max, const int32_t* n_st,
                                      const int32_t* n_eig, const double* d_st_xyz, const double* d_vis,
                                      void* stream) {
  return collect_common(h, n_t, n_st_max, nullptr, n_st, n_eig, d_st_xyz, d_vis, 1, stream);
}

extern "C" int bipp_ss_collect_device_c64(bipp_ss_t h, int32_t n_t, int32_t n_st_max, const int32_t* n_st,
                                          const int32_t* n_eig, const double* d_st_xyz, const float* d_vis,
                                          void* stream) {
  return collect_common(h, n_t, n_st_max, nullptr, n_st, n_eig, d_st_xyz, d_vis, 1, stream, 1);
}

extern "C" int bipp_ss_collect_channels(bipp_ss_t h, int32_t n_t, int32_t n_st_max, const int32_t* chan,
                                        const int32_t* n_st, const int32_t* n_eig, const double* st_xyz,
                                        const double* vis, int32_t on_device, void* stream) {
  if (h && !chan) return fail(h, BIPP_ERR_INVALID_ARG, "chan is NULL");
  return collect_common(h, n_t, n_st_max, chan, n_st, n_eig, st_xyz, vis, on_device, stream);
}

static size_t n_img(const bipp_ss* h) { return (size_t)h->n_chan * h->n_level * h->n_pix; }

extern "C" int bipp_ss_get_f64(bipp_ss_t h, double* out) {
  if (!h) return fail(nullptr, BIPP_ERR_INVALID_ARG, "handle is NULL");
  if (!out) return fail(h, BIPP_ERR_INVALID_ARG, "out is NULL");
  CUDA_TRY(h, cudaSetDevice(h->device));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  CUDA_TRY(h, cudaMemcpy(out, h->d_img, sizeof(double) * n_img(h), cudaMemcpyDeviceToHost));
  return BIPP_OK;
}

extern "C" int bipp_ss_get(bipp_ss_t h, float* out) {
  if (!h) return fail(nullptr, BIPP_ERR_INVALID_ARG, "handle is NULL");
  if (!out) return fail(h, BIPP_ERR_INVALID_ARG, "out is NULL");
  std::vector<double> tmp(n_img(h));
  const int rc = bipp_ss_get_f64(h, tmp.data());
  if (rc) return rc;
  for (size_t i = 0; i < tmp.size(); ++i) out[i] = (float)tmp[i];
  return BIPP_OK;
}

extern "C" int bipp_ss_get_device_f64(bipp_ss_t h, double* d_out, void* stream) {
  if (!h) return fail(nullptr, BIPP_ERR_INVALID_ARG, "handle is NULL");
  if (!d_out) return fail(h, BIPP_ERR_INVALID_ARG, "d_out is NULL");
  CUDA_TRY(h, cudaSetDevice(h->device));
  cudaStream_t s = stream ? (cudaStream_t)stream : h->stream;
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(d_out, h->d_img, sizeof(double) * n_img(h), cudaMemcpyDeviceToDevice, s));
  return BIPP_OK;
}

extern "C" int bipp_ss_reset(bipp_ss_t h) {
  if (!h) return fail(nullptr, BIPP_ERR_INVALID_ARG, "handle is NULL");
  CUDA_TRY(h, cudaSetDevice(h->device));
  CUDA_TRY(h, cudaMemsetAsync(h->d_img, 0, sizeof(double) * n_img(h), h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return BIPP_OK;
}

extern "C" int bipp_ss_set_images(bipp_ss_t h, const double* img) {
  if (!h) return fail(nullptr, BIPP_ERR_INVALID_ARG, "handle is NULL");
  if (!img) return fail(h, BIPP_ERR_INVALID_ARG, "img is NULL");
  CUDA_TRY(h, cudaSetDevice(h->device));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  CUDA_TRY(h, cudaMemcpy(h->d_img, img, sizeof(double) * n_img(h), cudaMemcpyHostToDevice));
  return BIPP_OK;
}

extern "C" int bipp_ss_last_eigvals(bipp_ss_t h, int32_t n_t_cap, int32_t n_eig_cap, int32_t* n_t_out,
                                    int32_t* n_kept, double* mu, int32_t* level) {
  if (!h) return fail(nullptr, BIPP_ERR_INVALID_ARG, "handle is NULL");
  if (n_t_out) *n_t_out = h->last_T;
  if (h->last_T == 0) return BIPP_OK;
  CUDA_TRY(h, cudaSetDevice(h->device));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  const int T = std::min(n_t_cap, h->last_T), K = h->last_K;
  if (T <= 0) return BIPP_OK;
  std::vector<int> nk(h->last_T);
  std::vector<double> m((size_t)h->last_T * K);
  std::vector<int> lv((size_t)h->last_T * K);
  CUDA_TRY(h, cudaMemcpy(nk.data(), h->d_nkept, sizeof(int) * h->last_T, cudaMemcpyDeviceToHost));
  CUDA_TRY(h, cudaMemcpy(m.data(), h->d_sel_mu, sizeof(double) * m.size(), cudaMemcpyDeviceToHost));
  CUDA_TRY(h, cudaMemcpy(lv.data(), h->d_level, sizeof(int) * lv.size(), cudaMemcpyDeviceToHost));
  for (int t = 0; t < T; ++t) {
    if (n_kept) n_kept[t] = nk[t];
    for (int e = 0; e < std::min(n_eig_cap, K); ++e) {
      if (mu) mu[(size_t)t * n_eig_cap + e] = m[(size_t)t * K + e];
      if (level) level[(size_t)t * n_eig_cap + e] = lv[(size_t)t * K + e];
    }
  }
  return BIPP_OK;
}

extern "C" int bipp_ss_debug_fail_wait(bipp_ss_t h, int32_t on) {
  if (!h) return fail(nullptr, BIPP_ERR_INVALID_ARG, "handle is NULL");
  if (on != 0 && on != 1) return fail(h, BIPP_ERR_INVALID_ARG, "on must be 0 or 1");
  CUDA_TRY(h, cudaSetDevice(h->device));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  if (tc_set_fail_wait(&h->tc, on)) return fail(h, BIPP_ERR_CUDA, "fault-injection word");
  h->fail_wait = on;
  return BIPP_OK;
}

extern "C" int bipp_ss_get_timings(bipp_ss_t h, double* out6) {
  if (!h) return fail(nullptr, BIPP_ERR_INVALID_ARG, "handle is NULL");
  if (!out6) return fail(h, BIPP_ERR_INVALID_ARG, "out6 is NULL");
  for (int i = 0; i < 6; ++i) out6[i] = h->timings[i];
  return BIPP_OK;
}

extern "C" int bipp_ss_get_nufft_timings(bipp_ss_t h, double* out11) {
  if (!h) return fail(nullptr, BIPP_ERR_INVALID_ARG, "handle is NULL");
  if (!out11) return fail(h, BIPP_ERR_INVALID_ARG, "out11 is NULL");
  for (int i = 0; i < 11; ++i) out11[i] = h->nu_timings[i];
  return BIPP_OK;
}

extern "C" int bipp_ss_get_synth_shape(bipp_ss_t h, int32_t* out4) {
  if (!h) return fail(nullptr, BIPP_ERR_INVALID_ARG, "handle is NULL");
  if (!out4) return fail(h, BIPP_ERR_INVALID_ARG, "out4 is NULL");
  for (int i = 0; i < 4; ++i) out4[i] = h->synth_shape[i];
  return BIPP_OK;
}

extern "C" const char* bipp_ss_last_error(bipp_ss_t h) { return h ? h->err.c_str() : g_create_err.c_str(); }
