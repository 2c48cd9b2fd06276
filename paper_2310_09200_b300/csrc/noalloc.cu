// noalloc.cu — bipp_ss_collect_noalloc: one collect() step that allocates no
// device memory.
//
// Some callers cannot call cudaMalloc: a real-time telescope pipeline that
// reserves all of its device memory at start-up and forbids any later
// allocation, or a host framework that owns the device memory budget and
// whose allocator must not be bypassed. For them this entry point runs the
// whole step (Gram matrix, generalised eigensolve, selection, FP64 synthesis)
// with every intermediate in one file-scope device array of fixed size; the
// caller passes only its inputs and its output image.
//
// The array is a module global: every GPU that loads the library holds it
// until the process exits, every call shares it and it keeps the contents
// of the last call, so calls that overlap on a GPU race with each other.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "bipp_internal.cuh"
#include "bipp_ss.h"

namespace {

using namespace bipp;

constexpr int kN = BIPP_NOALLOC_MAX_STATIONS;
constexpr int kK = BIPP_NOALLOC_MAX_EIG;
constexpr size_t kAlign = 256;
// The eigensolve of the step: FP64 Jacobi with the handle's default stopping
// rule (off(C) <= 1e-13 ||C||_F) and sweep cap.
constexpr double kJacobiTol = 1e-13;
constexpr int kJacobiSweeps = 40;

constexpr size_t up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Byte offsets of the regions inside the scratch array (sized for kN, kK).
constexpr size_t kOffInts = 0;                                   // nst, neig, status, sweeps, nkept, flag
constexpr size_t kOffBounds = kOffInts + up(8 * sizeof(int));    // 2 x kMaxLevels doubles
constexpr size_t kOffG = kOffBounds + up(2 * kMaxLevels * sizeof(double));
constexpr size_t kOffLinv = kOffG + up((size_t)kN * kN * sizeof(double));
constexpr size_t kOffX = kOffLinv + up((size_t)kN * kN * sizeof(double));
constexpr size_t kOffC = kOffX + up((size_t)kN * kN * sizeof(double2));
constexpr size_t kOffQ = kOffC + up((size_t)kN * kN * sizeof(double2));
constexpr size_t kOffMu = kOffQ + up((size_t)kN * kN * sizeof(double2));
constexpr size_t kOffSelMu = kOffMu + up((size_t)kN * sizeof(double));
constexpr size_t kOffLevel = kOffSelMu + up((size_t)kK * sizeof(double));
constexpr size_t kOffWt = kOffLevel + up((size_t)kK * sizeof(int));
constexpr size_t kOffW64 = kOffWt + up((size_t)kK * sizeof(double));
constexpr size_t kOffW32 = kOffW64 + up((size_t)kK * kN * sizeof(double2));
constexpr size_t kOffQst = kOffW32 + up((size_t)kK * kN * sizeof(float2));
constexpr size_t kOffWl = kOffQst + up((size_t)6 * kN * sizeof(float));  // the step's wavelength
constexpr size_t kScratchBytes = kOffWl + up(sizeof(double));
static_assert(kScratchBytes <= (size_t)BIPP_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the stated size");

// The scratch itself. In host code this name is only a stand-in for the
// device symbol; kernels receive the address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[BIPP_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_dev_ptr[kMaxDevices] = {};

int report(char* msg, int len, int code, const char* fmt, ...) {
  if (msg && len > 0) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, (size_t)len, fmt, ap);
    va_end(ap);
  }
  return code;
}

}  // namespace

extern "C" int bipp_ss_collect_noalloc(int64_t n_pix, const double* d_pix_xyz, double wl, int32_t n_level,
                                       const double* level_bounds, int32_t n_eig, int32_t filter,
                                       int32_t gram_identity, int32_t n_st, const double* d_st_xyz,
                                       const double* d_vis, double* d_img, void* stream, char* err_msg,
                                       int32_t err_len) {
  if (err_msg && err_len > 0) err_msg[0] = '\0';
  if (n_st < 1 || n_st > kN)
    return report(err_msg, err_len, BIPP_ERR_UNSUPPORTED,
                  "n_st=%d outside [1, %d]: the fixed scratch of the no-allocation path holds at most %d stations",
                  n_st, kN, kN);
  if (n_eig < 1 || n_eig > n_st || n_eig > kK)
    return report(err_msg, err_len, BIPP_ERR_UNSUPPORTED, "n_eig=%d outside [1, min(n_st=%d, %d)]", n_eig, n_st, kK);
  if (n_level < 1 || n_level > kMaxLevels)
    return report(err_msg, err_len, BIPP_ERR_UNSUPPORTED, "n_level=%d outside [1, %d]", n_level, kMaxLevels);
  if (n_pix < 1 || !d_pix_xyz || !level_bounds || !d_st_xyz || !d_vis || !d_img)
    return report(err_msg, err_len, BIPP_ERR_INVALID_ARG, "need n_pix >= 1 and non-NULL buffers");
  if (!(wl > 0.0) || !isfinite(wl) || filter < 0 || filter > 1)
    return report(err_msg, err_len, BIPP_ERR_INVALID_ARG, "need a finite wl > 0 and filter LSQ (0) or STD (1)");
  for (int l = 0; l < 2 * n_level; ++l)
    if (isnan(level_bounds[l]))
      return report(err_msg, err_len, BIPP_ERR_INVALID_ARG, "level bound %d of %d is NaN", l, 2 * n_level);

  (void)cudaGetLastError();  // an error left by an earlier, unrelated call is not this call's
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return report(err_msg, err_len, BIPP_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return report(err_msg, err_len, BIPP_ERR_UNSUPPORTED, "device %d", dev);
  // Every buffer is read or written by kernels on the current device: it must
  // be device memory there, and aligned for the kernels' double and complex
  // loads (a host pointer or a misaligned view would fault on the device).
  {
    const void* ptrs[4] = {d_pix_xyz, d_st_xyz, d_vis, d_img};
    const char* names[4] = {"d_pix_xyz", "d_st_xyz", "d_vis", "d_img"};
    const uintptr_t align[4] = {8, 8, 16, 8};
    for (int i = 0; i < 4; ++i) {
      cudaPointerAttributes a{};
      if (cudaPointerGetAttributes(&a, ptrs[i]) != cudaSuccess || a.type != cudaMemoryTypeDevice || a.device != dev) {
        (void)cudaGetLastError();
        return report(err_msg, err_len, BIPP_ERR_INVALID_ARG, "%s must be device memory on the current device %d",
                      names[i], dev);
      }
      if (reinterpret_cast<uintptr_t>(ptrs[i]) % align[i])
        return report(err_msg, err_len, BIPP_ERR_INVALID_ARG, "%s must be %d-byte aligned", names[i],
                      (int)align[i]);
    }
  }
  unsigned char* base;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // with `dev` current
      if (e != cudaSuccess)
        return report(err_msg, err_len, BIPP_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      g_dev_ptr[dev] = static_cast<unsigned char*>(p);
    }
    base = g_dev_ptr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  int* ints = reinterpret_cast<int*>(base + kOffInts);
  Batch b{};
  b.T = 1;
  b.n_max = n_st;
  b.k_max = n_eig;
  b.nst = ints + 0;
  b.neig = ints + 1;
  b.status = ints + 2;
  b.sweeps = ints + 3;
  b.nkept = ints + 4;
  b.flag = ints + 5;
  b.st = d_st_xyz;
  b.vis = reinterpret_cast<const double2*>(d_vis);
  b.G = reinterpret_cast<double*>(base + kOffG);
  b.Linv = reinterpret_cast<double*>(base + kOffLinv);
  b.X = reinterpret_cast<double2*>(base + kOffX);
  b.C = reinterpret_cast<double2*>(base + kOffC);
  b.Q = reinterpret_cast<double2*>(base + kOffQ);
  b.mu = reinterpret_cast<double*>(base + kOffMu);
  b.sel_mu = reinterpret_cast<double*>(base + kOffSelMu);
  b.level = reinterpret_cast<int*>(base + kOffLevel);
  b.wt = reinterpret_cast<double*>(base + kOffWt);
  b.W64 = reinterpret_cast<double2*>(base + kOffW64);
  b.W32 = reinterpret_cast<float2*>(base + kOffW32);
  b.q = reinterpret_cast<float*>(base + kOffQst);
  double* d_wl = reinterpret_cast<double*>(base + kOffWl);
  b.wl = d_wl;
  b.chan = nullptr;
  double* d_bounds = reinterpret_cast<double*>(base + kOffBounds);

  // sizes and level bounds into the scratch; status words start at zero
  const int hdr[8] = {n_st, n_eig, 0, 0, 0, 0, 0, 0};
  e = cudaMemcpyAsync(ints, hdr, sizeof(hdr), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    double bnd[2 * kMaxLevels];
    memcpy(bnd, level_bounds, sizeof(double) * 2 * n_level);
    e = cudaMemcpyAsync(d_bounds, bnd, sizeof(double) * 2 * n_level, cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_wl, &wl, sizeof(double), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return report(err_msg, err_len, BIPP_ERR_CUDA, "upload: %s", cudaGetErrorString(e));

  launch_gram(b, gram_identity, s);
  launch_cholesky(b, gram_identity, s);
  launch_reduce(b, gram_identity, s);
  launch_jacobi(b, kJacobiTol, kJacobiSweeps, s);
  launch_select(b, n_level, d_bounds, filter, s);
  Pixels px{n_pix, d_pix_xyz, nullptr};
  launch_synth_simt_f64(b, px, n_level, d_img, s);
  if ((e = cudaGetLastError()) != cudaSuccess)
    return report(err_msg, err_len, BIPP_ERR_CUDA, "launch: %s", cudaGetErrorString(e));
  int status = 0;
  e = cudaMemcpyAsync(&status, b.status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return report(err_msg, err_len, BIPP_ERR_CUDA, "run: %s", cudaGetErrorString(e));
  if (status & kStatusNotPD)
    return report(err_msg, err_len, BIPP_ERR_GRAM_NOT_PD, "Gram matrix is not positive definite");
  if (status & kStatusNotConverged)
    return report(err_msg, err_len, BIPP_ERR_EIG_NOT_CONVERGED, "Jacobi did not converge in %d sweeps", kJacobiSweeps);
  return BIPP_OK;
}
