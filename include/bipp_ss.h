/*
 * bipp_ss.h — C ABI of the B300-native Bluebild standard-synthesis library
 * (libbipp_ss.so). BIPP, arXiv:2310.09200.
 *
 * The library computes, per time step t (Algorithm 1 "Standard Synthesis"):
 *   1. the Gram matrix G_ij = sinc(2 ||p_i - p_j|| / wl), sinc(x) = sin(pi x)/(pi x)
 *      (Sec. 2.2, Eq. gram; App. A),
 *   2. the generalised Hermitian eigenpairs V a = mu G a with A^H G A = I
 *      (Sec. 2.3, Eq. eigenvaleq),
 *   3. the n_eig algebraically largest pairs, their filter weights d_e
 *      (LSQ: d = mu, STD: d = 1) and levels [lo, hi) (Sec. 2.6),
 *   4. the level images I_l(r) += sum_{e in l} d_e |sum_i exp(-j 2 pi <r, p_i>/wl) a_ie|^2
 *      (Sec. 2.4, Eq. standard_synthesis; Algorithm 2 "GEMMEXP"),
 * accumulated over collect() calls (Sec. 2.3: the time-integrated image is the
 * sum of the per-step images).
 *
 * Conventions
 *   - All arrays are column-major (Sec. 3.2 "Input data"). An n x 3 position
 *     array holds x[0..n), then y[0..n), then z[0..n). Complex arrays are
 *     interleaved (re, im) doubles.
 *   - Pixel directions are unit vectors; station positions are in metres;
 *     wl is the wavelength in metres.
 *   - Level l takes every kept eigenvalue mu with lo_l <= mu < hi_l (first
 *     matching level); eigenpairs outside every interval are dropped. Bounds
 *     may be +-INFINITY.
 *   - Images are n_pix x n_level, column-major.
 *
 * Ownership: the caller owns every input and output buffer. create() copies
 * pixels and bounds to the device; collect*() consumes its inputs before it
 * returns (host variants) or in stream order (device variant); get*() writes
 * caller memory. The handle owns its device buffers until destroy().
 *
 * Errors: every call returns BIPP_OK (0) or a negative BIPP_ERR_* code and
 * records a message readable with bipp_ss_last_error(h). No C++ exception
 * crosses this boundary. A collect that fails leaves the accumulated images
 * unchanged (a batch commits only when every step in it succeeded).
 *
 * Threads: a handle is not thread-safe; distinct handles are independent.
 * Each handle owns one CUDA stream on its device.
 */
#ifndef BIPP_SS_H
#define BIPP_SS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BIPP_OK 0
#define BIPP_ERR_INVALID_ARG (-1)       /* bad size, pointer, value or option */
#define BIPP_ERR_CUDA (-2)              /* a CUDA runtime call failed */
#define BIPP_ERR_OUT_OF_MEMORY (-3)     /* device allocation failed */
#define BIPP_ERR_GRAM_NOT_PD (-4)       /* Cholesky of G met a non-positive (or NaN) pivot */
#define BIPP_ERR_EIG_NOT_CONVERGED (-5) /* an eigensolver iteration cap was hit (or a kept residual too large) */
#define BIPP_ERR_DEVICE_TIMEOUT (-6)    /* a bounded device-side wait gave up */
#define BIPP_ERR_UNSUPPORTED (-7)       /* e.g. n_eig > n_st, sizes beyond limits */

/* Arithmetic of the synthesis stage (steps 1-3 always reach FP64 accuracy). */
#define BIPP_PREC_FP64 0       /* FP64 phases, sincos and sums (CUDA cores) */
#define BIPP_PREC_FP32 1       /* exact phase reduction, SFU sincos, FP32 CUDA-core sums */
#define BIPP_PREC_SPLIT_BF16 2 /* exact phase reduction, SFU sincos, tcgen05 hi/lo BF16 x3, FP32 accumulate */
#define BIPP_PREC_SPLIT_FP16 3 /* as SPLIT_BF16 with FP16 hi/lo operands (scaled W): finer
                                  operands, so it meets the FP32 path's 1e-5 relative L2 per level
                                  up to ~512 stations (6.5e-6 measured at 512); the error grows with
                                  K = 2 n_st (1.27e-5 measured at 1024), bounded by FP32 summation
                                  over K terms, 2 n_st 2^-24. Both split forms take station
                                  coordinates below 2^28 wavelengths (|p|/wl); a step with a station
                                  farther out fails with BIPP_ERR_UNSUPPORTED and adds nothing */

#define BIPP_FILTER_LSQ 0 /* d_e = mu_e (Sec. 2.6, least-squares image) */
#define BIPP_FILTER_STD 1 /* d_e = 1    (Sec. 2.6, standardised image) */

#define BIPP_EIG_JACOBI64 0 /* FP64 parallel-order Jacobi on the reduced matrix */
#define BIPP_EIG_MIXED 1    /* FP32 tridiagonal eigendecomposition, then FP64-class refinement of the kept pairs */

typedef struct bipp_ss* bipp_ss_t;

typedef struct {
  int32_t n_eig;             /* eigenpairs kept per step (Sec. 2.6 "Truncation"); 0 = all */
  int32_t precision;         /* BIPP_PREC_*; default BIPP_PREC_FP32 */
  int32_t filter;            /* BIPP_FILTER_*; default LSQ */
  int32_t gram_identity;     /* 1: G = I (back-projection decomposition, Sec. 6.3); default 0 */
  int32_t max_jacobi_sweeps; /* default 40 */
  double jacobi_tol;         /* stop when off(C) <= tol * ||C||_F; default 1e-13 */
  int32_t device;            /* CUDA device ordinal; default -1 = current device */
  int32_t eig_mode;          /* BIPP_EIG_*; default BIPP_EIG_JACOBI64 */
  int32_t use_graph;         /* 1: capture each batch geometry once in a CUDA graph and replay it; default 1 */
  int32_t autotune;          /* 1: time the tensor-core kernel's stage count on the first batch of a
                                geometry and keep the fastest; default 1 */
  int32_t eigenimages;       /* 1: one image per kept eigenpair instead of energy levels: image e holds
                                sum over steps of d_e |Phi^H a_e|^2 for the e-th largest kept eigenvalue
                                (filter weight d_e as for levels); needs 1 <= n_eig <= BIPP_MAX_EIGENIMAGES
                                and n_level = n_eig at create, level_bounds may be NULL; default 0 */
  int32_t synthesis;         /* BIPP_SYNTH_*; default BIPP_SYNTH_STANDARD */
  double nufft_eps;          /* BIPP_SYNTH_NUFFT: type-3 NUFFT tolerance in [1e-7, 0.1]; default 1e-5 */
  int32_t nufft_partition[6]; /* BIPP_SYNTH_NUFFT domain partitioning (Sec. 3.4.1), each in [1, 64]:
                                 [0..2] input cells of the baseline box per dimension (x, y, z),
                                 [3..5] image cells of the pixels' box per dimension; each non-empty
                                 (input, image) cell pair is one type-3 transform whose grid spans
                                 that cell only. Default all 1 (one transform per level) */
  int32_t reserved[2];       /* must be zero */
} bipp_ss_options;

/* Image synthesis strategy (Sec. 2.5, 3.4).
 * STANDARD: Phi^H W per pixel and step, then the level reduction (Algorithm 2).
 * NUFFT:    per level, the Gram-corrected visibilities of the level's eigenpairs,
 *           V'_l = sum_{e in l} d_e a_e a_e^H, summed over all baselines of the
 *           batch's steps with one type-3 NUFFT per level and channel
 *           (Algorithm 3): I_l(r) = sum_t sum_{p,q} V'_l,pq exp(-j 2 pi/wl <p_p - p_q, r>).
 *           Same images as STANDARD up to the NUFFT tolerance (relative L2 of
 *           the order of nufft_eps). Grids and sums are FP32 with coordinates
 *           and phases reduced in FP64; `precision` does not apply. The uniform
 *           grid spans the batch's baseline extent times the pixels' extent per
 *           dimension (of the order of 2 max|b|/wl x (pixel extent) points), so
 *           it suits fields whose pixels resolve the array (small fields of
 *           view); nufft_partition splits it into smaller transforms, and
 *           BIPP_ERR_UNSUPPORTED reports grids that do not fit in device
 *           memory. The grids are planned on the host from the batch's station
 *           coordinates, so a collect with device inputs copies those back
 *           (one synchronisation), and collects are not captured in CUDA
 *           graphs. The spreading sums with float atomics, so results are
 *           reproducible to FP32 rounding, not bitwise. Not with eigenimages. */
#define BIPP_SYNTH_STANDARD 0
#define BIPP_SYNTH_NUFFT 1

#define BIPP_MAX_EIGENIMAGES 64

/* Fill *opt with the defaults listed above. */
void bipp_ss_default_options(bipp_ss_options* opt);

/* Create an imaging handle (the paper's StandardSynthesis object, Sec. 3.1).
 *   pix_xyz      n_pix x 3 unit vectors (host), copied; must be finite.
 *   wl           wavelength [m], finite and > 0.
 *   level_bounds n_level x 2 (host): column 0 = lo, column 1 = hi; copied
 *                (unused, may be NULL, with opt->eigenimages).
 *   opt          NULL for defaults.
 * n_pix >= 1, 1 <= n_level <= 16 (n_level = n_eig <= 64 with eigenimages).
 * Images start at zero. */
int bipp_ss_create(bipp_ss_t* out, int64_t n_pix, const double* pix_xyz, double wl,
                   int32_t n_level, const double* level_bounds, const bipp_ss_options* opt);

/* Create a handle for n_chan frequency channels sharing one pixel grid
 * (Sec. 2.3: the eigendecomposition is repeated per step and per frequency
 * band). Channel c has wavelength wl[c] [m], its own level intervals (block c
 * of level_bounds, each block n_level x 2 as in bipp_ss_create) and its own
 * level images: get*() returns n_chan consecutive n_pix x n_level blocks.
 * bipp_ss_create is the n_chan = 1 case. 1 <= n_chan <= 4096. */
int bipp_ss_create_channels(bipp_ss_t* out, int64_t n_pix, const double* pix_xyz, int32_t n_chan,
                            const double* wl, int32_t n_level, const double* level_bounds,
                            const bipp_ss_options* opt);

/* Collect a batch of steps from any channels in one launch sequence: step t
 * belongs to channel chan[t]; steps must be grouped by channel in
 * non-decreasing order. Layout and the other arguments as in
 * bipp_ss_collect_batch (on_device = 0, host buffers) or
 * bipp_ss_collect_device (on_device = 1, device buffers ordered on stream). */
int bipp_ss_collect_channels(bipp_ss_t h, int32_t n_t, int32_t n_st_max, const int32_t* chan,
                             const int32_t* n_st, const int32_t* n_eig, const double* st_xyz, const double* vis,
                             int32_t on_device, void* stream);

/* Collect one time step (Algorithm 1 "collect"), host buffers.
 *   st_xyz  n_st x 3 station positions [m] (must be finite).
 *   vis     n_st x n_st Hermitian visibility matrix, complex128 interleaved.
 * 1 <= n_eig <= n_st <= 1024. Synchronous: returns after the step is
 * accumulated (or failed). */
int bipp_ss_collect(bipp_ss_t h, int32_t n_st, const double* st_xyz, const double* vis);

/* Collect n_t time steps in one batched launch sequence, host buffers.
 * Step t has n_st[t] stations (ragged, e.g. after flagging) and keeps
 * n_eig[t] eigenpairs (n_eig == NULL: the handle's n_eig for every step).
 *   st_xyz  n_t blocks, block t = n_st_max x 3 (only the first n_st[t] rows
 *           of each column are read).
 *   vis     n_t blocks, block t = n_st_max x n_st_max complex128 (leading
 *           n_st[t] x n_st[t] submatrix read).
 * Commits all n_t steps or none. */
int bipp_ss_collect_batch(bipp_ss_t h, int32_t n_t, int32_t n_st_max, const int32_t* n_st,
                          const int32_t* n_eig, const double* st_xyz, const double* vis);

/* As bipp_ss_collect_batch with the position and visibility blocks already
 * on the device (e.g. memory owned by PyTorch), stream-ordered on `stream`
 * (a cudaStream_t; NULL = the handle's stream). n_st / n_eig are host arrays
 * of n_t int32 (n_eig NULL = handle default). Values are not inspected on the
 * host: a non-finite position surfaces as BIPP_ERR_GRAM_NOT_PD (as
 * BIPP_ERR_INVALID_ARG with BIPP_SYNTH_NUFFT, which plans its grids from a
 * host copy of the positions). d_st_xyz
 * must be 8-byte and d_vis 16-byte aligned (BIPP_ERR_INVALID_ARG otherwise).
 * Returns after the batch has run and its per-step status was read (one host
 * sync). */
int bipp_ss_collect_device(bipp_ss_t h, int32_t n_t, int32_t n_st_max, const int32_t* n_st,
                           const int32_t* n_eig, const double* d_st_xyz, const double* d_vis,
                           void* stream);

/* As bipp_ss_collect_device with complex64 visibilities: d_vis holds n_t
 * blocks of n_st_max x n_st_max interleaved (re, im) floats, column-major
 * (8-byte aligned). They are widened to complex128 on the device, in stream
 * order, into the handle's batch buffer; the rest of the batch is identical
 * to bipp_ss_collect_device on the widened values. */
int bipp_ss_collect_device_c64(bipp_ss_t h, int32_t n_t, int32_t n_st_max, const int32_t* n_st,
                               const int32_t* n_eig, const double* d_st_xyz, const float* d_vis,
                               void* stream);

/* Copy the accumulated images (n_pix x n_level column-major per channel,
 * channels consecutive) to host memory. */
int bipp_ss_get(bipp_ss_t h, float* out);
int bipp_ss_get_f64(bipp_ss_t h, double* out);

/* Copy the accumulated images to device memory d_out (n_pix x n_level FP64),
 * ordered on `stream` (NULL = the handle's stream). */
int bipp_ss_get_device_f64(bipp_ss_t h, double* d_out, void* stream);

/* Zero the accumulated images. */
int bipp_ss_reset(bipp_ss_t h);

/* Replace the accumulated images (checkpoint/resume: images are additive
 * over steps), host n_pix x n_level FP64. */
int bipp_ss_set_images(bipp_ss_t h, const double* img);

/* Diagnostics of the most recent batch: for step t < n_t_cap, the kept
 * eigenvalues mu (descending) and their level ids (-1 = dropped) into
 * mu[t * n_eig_cap + e], level[t * n_eig_cap + e]; n_kept[t] = eigenpairs
 * kept; *n_t_out = steps in that batch. Any output pointer may be NULL. */
int bipp_ss_last_eigvals(bipp_ss_t h, int32_t n_t_cap, int32_t n_eig_cap, int32_t* n_t_out,
                         int32_t* n_kept, double* mu, int32_t* level);

/* Statistics of the most recent batch, measured with CUDA events on the
 * stream the batch ran on: out[0] Gram + Cholesky + reduction [ms],
 * out[1] eigensolve [ms], out[2] select/pack [ms], out[3] synthesis [ms],
 * out[4] Jacobi sweeps summed over the steps, out[5] kernels launched. */
int bipp_ss_get_timings(bipp_ss_t h, double* out6);

/* Kernel times of the last collect's NUFFT synthesis (BIPP_SYNTH_NUFFT; CUDA
 * events on the collect's stream, first channel of the batch):
 * out[0] sorting the baselines and forming their level strengths (k_nu_const,
 * k_nu_count, the scans, k_nu_scatter) [ms], out[1] spreading (k_nu_spread,
 * all level groups) [ms], out[2] one level's deconvolve/pad (k_nu_pad) [ms],
 * out[3] one level's FFT (cuFFT) [ms], out[4] one level's interpolation
 * (k_nu_interp) [ms], out[5] all levels' pad + FFT + interpolation [ms],
 * out[6..8] the spread grid's points per dimension (M), out[9] the kernel
 * width w, out[10] the number of baselines spread. Zeros for STANDARD. */
int bipp_ss_get_nufft_timings(bipp_ss_t h, double* out11);

/* Launch shape of the tensor-core synthesis of the last collect (split
 * precisions; the paper has no counterpart: it reports the autotuner's pick):
 * out[0] shared-memory ring stages, out[1] 1 if A_hi [B_hi | B_lo] ran as one
 * fused MMA (else three), out[2] 1 if dedicated warps ran the epilogue (else
 * the producer warps), out[3] 1 if the shape came from the autotuner (0: the
 * default shape, as on the collect that runs the tuning). All zeros for the
 * FP32 / FP64 precisions and for NUFFT synthesis. */
int bipp_ss_get_synth_shape(bipp_ss_t h, int32_t* out4);

/* Fault injection for tests of failure detection (no GPU fault): while on
 * (1), the tensor-core synthesis kernel (BIPP_PREC_SPLIT_*) makes its MMA
 * issuer wait on a shared-memory barrier phase that nothing completes. Its
 * bounded wait runs out after ~2 s; the kernel then sets its abort flag, the
 * other warps leave their own bounded waits, copies in flight land, TMEM is
 * released, and the collect returns BIPP_ERR_DEVICE_TIMEOUT with the images
 * unchanged (nothing is added before the first accumulator is complete).
 * Off (0, the default) restores normal operation; the switch is a device
 * word read at launch, so captured CUDA graphs follow it. Other synthesis
 * paths have no such waits and ignore it. */
int bipp_ss_debug_fail_wait(bipp_ss_t h, int32_t on);

/* Differentiable synthesis with complex station gains (device pointers,
 * e.g. PyTorch memory; stream-ordered on `stream`, NULL = default stream;
 * returns after the work has finished).
 *   z_te(r) = sum_i conj(g_i exp(j 2 pi <r, p_ti>/wl)) W_t[i,e]       (Sec. 2.1 gains in the
 *   I_l(r)  = sum_t sum_{e: level[t,e] = l} d[t,e] |z_te(r)|^2         sampling operator, Eq.
 *                                                                      standard_synthesis, Alg. 1)
 *   d_pix     n_pix x 3 FP64 unit vectors (column-major).
 *   d_st_xyz  n_t blocks of n_st x 3 FP64 [m];  d_W: n_t blocks of n_st x n_eig complex128
 *             (column-major);  d_d: n_t x n_eig FP64 weights (row t contiguous);
 *   d_level   n_t x n_eig int32 level ids (-1 = dropped);  d_gains: n_st complex128.
 *   precision BIPP_PREC_FP32: exact phase reduction, SFU sincos, FP32 sums on
 *             the CUDA cores; BIPP_PREC_SPLIT_FP16 / _BF16: the tensor-core
 *             synthesis kernel of collect() on W' = diag(conj g) W (n_eig <=
 *             128), to the same accuracy as collect() in that precision, with
 *             the same station range (|p|/wl below 2^28, else
 *             BIPP_ERR_UNSUPPORTED; the adjoint alike).
 * bipp_ss_synth_levels_device writes d_img (n_pix x n_level FP64, overwritten).
 * 1 <= n_eig <= n_st <= 1024, 1 <= n_level <= 16; another precision returns
 * BIPP_ERR_INVALID_ARG. */
int bipp_ss_synth_levels_device(int64_t n_pix, const double* d_pix, double wl, int32_t n_t, int32_t n_st,
                                int32_t n_eig, int32_t n_level, const double* d_st_xyz, const double* d_W,
                                const double* d_d, const int32_t* d_level, const double* d_gains, double* d_img,
                                int32_t precision, void* stream);

/* Adjoint of bipp_ss_synth_levels_device: given d_grad_img = dL/dI (n_pix x
 * n_level FP64) of a real loss L, writes the complex gradients (convention
 * dL/dRe + j dL/dIm) d_grad_W (n_t blocks of n_st x n_eig complex128) and
 * d_grad_g (n_st complex128). The phase matrix is recomputed, not stored;
 * the pixel reduction is deterministic (fixed-order two-stage sum).
 *   precision BIPP_PREC_FP32: CUDA-core kernels; BIPP_PREC_SPLIT_FP16 / _BF16
 *             (n_eig <= 64 and n_level <= 4, else BIPP_ERR_UNSUPPORTED): z
 *             recomputed by the tensor-core synthesis kernel (hi/lo products
 *             in that type), Y = d R z written in BF16 hi/lo, and the pixel
 *             contraction grad_W' = 2 sum_r Phi Y as split BF16 products on the
 *             tensor cores with FP32 accumulation; BIPP_ERR_DEVICE_TIMEOUT if
 *             a bounded device wait gave up. Calls on one device serialise on
 *             the library's tensor-core workspace for that device. */
int bipp_ss_synth_adjoint_device(int64_t n_pix, const double* d_pix, double wl, int32_t n_t, int32_t n_st,
                                 int32_t n_eig, int32_t n_level, const double* d_st_xyz, const double* d_W,
                                 const double* d_d, const int32_t* d_level, const double* d_gains,
                                 const double* d_grad_img, double* d_grad_W, double* d_grad_g, int32_t precision,
                                 void* stream);

/* No-allocation variant of one collect() step. The paper has no counterpart:
 * this entry point exists for callers that may not allocate device memory,
 * e.g. a real-time pipeline that reserves all of its GPU memory at start-up
 * and forbids later allocation, or a host framework that owns the device
 * memory budget. It runs Gram, eigensolve, selection and FP64 synthesis of
 * one step with every intermediate held in one fixed array of
 * BIPP_NOALLOC_SCRATCH_BYTES that the library keeps in device memory (every
 * GPU that loads the library holds it until the process exits); it calls no
 * cudaMalloc/cudaFree and no allocating library routine.
 *   d_pix_xyz    n_pix x 3 FP64 unit vectors (device, column-major).
 *   level_bounds n_level x 2 (host), as in bipp_ss_create.
 *   n_eig, filter (BIPP_FILTER_*), gram_identity: as in bipp_ss_options.
 *   d_st_xyz     n_st x 3 FP64 (device); d_vis n_st x n_st complex128 (device).
 *   d_img        n_pix x n_level FP64 (device): the step's level images are
 *                ADDED to it (the caller zeroes it before the first step).
 *   stream       cudaStream_t or NULL; work runs on the current device.
 *   err_msg      optional buffer of err_len bytes for a message (may be NULL).
 * The eigensolve is the FP64 Jacobi with the handle defaults (stop at
 * off(C) <= 1e-13 ||C||_F, at most 40 sweeps). Every device buffer must be
 * device memory on the current device (d_vis 16-byte, the others 8-byte
 * aligned) and level bounds must not be NaN (BIPP_ERR_INVALID_ARG otherwise).
 * A step that fails (e.g. BIPP_ERR_GRAM_NOT_PD) adds nothing to d_img.
 * Limits: 1 <= n_eig <= n_st <= BIPP_NOALLOC_MAX_STATIONS,
 * n_eig <= BIPP_NOALLOC_MAX_EIG, 1 <= n_level <= 16; larger sizes return
 * BIPP_ERR_UNSUPPORTED with a message naming the limit. The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.
 * Every call shares the one array and the array keeps the last call's
 * contents (the call resets what must start at zero itself), so calls that
 * overlap on the same GPU race: serialise them. Returns after the step has
 * run (one stream synchronisation), with the same error codes as collect(). */
#define BIPP_NOALLOC_MAX_STATIONS 128
#define BIPP_NOALLOC_MAX_EIG 128
#define BIPP_NOALLOC_SCRATCH_BYTES (1536 * 1024)
int bipp_ss_collect_noalloc(int64_t n_pix, const double* d_pix_xyz, double wl, int32_t n_level,
                            const double* level_bounds, int32_t n_eig, int32_t filter, int32_t gram_identity,
                            int32_t n_st, const double* d_st_xyz, const double* d_vis, double* d_img,
                            void* stream, char* err_msg, int32_t err_len);

/* Measurement of the special-function-unit rate that bounds the phase
 * generation of the synthesis (Algorithm 2 evaluates exp(j theta) for every
 * pixel-station pair, Sec. 2.9): a kernel of independent __sincosf chains
 * (the intrinsic the synthesis kernels use) over 4 CTAs of 256 threads per SM
 * of `device` (-1 = current), timed with CUDA events after one warm-up launch;
 * *pairs_per_s receives the best of `repeats` (1..100) launches, in sine +
 * cosine pairs per second. Allocates and frees a small output buffer; takes a
 * few milliseconds per launch. */
int bipp_ss_measure_sincos_rate(int32_t device, int32_t repeats, double* pairs_per_s);

/* The FP32 and FP64 FMA rates of `device` (-1 = current) in flop/s (2 per
 * FMA): kernels of 8 independent FMA chains per thread over 4 CTAs of 256
 * threads per SM, best of `repeats` (1..100) launches after a warm-up, for the
 * rooflines of the CUDA-core stages (the eigensolve of Sec. 2.3). Allocates
 * and frees a small output buffer. */
int bipp_ss_measure_fma_rates(int32_t device, int32_t repeats, double* fp32_flops, double* fp64_flops);

/* Release the handle and its device memory. NULL is accepted. */
int bipp_ss_destroy(bipp_ss_t h);

/* Message of the last failing call on h (or, when h is NULL, of this
 * thread's last failing call without a handle: create and the estimation
 * functions); valid until the next such call. Never NULL. */
const char* bipp_ss_last_error(bipp_ss_t h);

/* ---- parameter estimation (Sec. 2.6 "Energy Levels & Partitioning"), host only
 *
 * bipp_ss_energy_neig: the least number of leading eigenpairs holding at least
 * `fraction` (0 < fraction <= 1) of the energy of one step, energy being the
 * sum of the positive eigenvalues. mu_desc: n eigenvalues in descending order
 * (host); *n_eig receives the count (>= 1). BIPP_ERR_INVALID_ARG on bad sizes,
 * non-finite or unordered values. */
int bipp_ss_energy_neig(int32_t n, const double* mu_desc, double fraction, int32_t* n_eig);

/* bipp_ss_kmeans_bounds: level intervals from k-means clustering of n values
 * (e.g. eigenvalues pooled over an observation's steps): the exact partition
 * of the sorted values into n_level contiguous clusters of least
 * within-cluster sum of squares. Writes level_bounds (host, n_level x 2
 * column-major, the layout of bipp_ss_create): level 0 is the highest
 * cluster, inner edges lie halfway between neighbouring clusters, outer edges
 * are -inf and +inf. 1 <= n_level <= n; BIPP_ERR_INVALID_ARG otherwise or on
 * non-finite values. Error text via bipp_ss_last_error(NULL). */
int bipp_ss_kmeans_bounds(int32_t n, const double* values, int32_t n_level, double* level_bounds);

/* bipp_ss_quantile_bounds: level intervals at the quantiles of n values
 * (eigenvalues pooled over an observation's steps; Sec. 2.6 "Partitioning"
 * leaves the partition rule to the user, this is the equal-count one). The
 * values are sorted; inner edge q (1 <= q < n_level) lies halfway between the
 * sorted values k-1 and k, k = q n / n_level rounded half to even and clamped
 * to [1, n-1], so no value sits on an edge unless two values are equal.
 * Writes level_bounds (host, n_level x 2 column-major, the layout of
 * bipp_ss_create): level 0 holds the largest values, outer edges are -inf and
 * +inf. 1 <= n_level <= n; BIPP_ERR_INVALID_ARG otherwise or on non-finite
 * values. Error text via bipp_ss_last_error(NULL). */
int bipp_ss_quantile_bounds(int32_t n, const double* values, int32_t n_level, double* level_bounds);

#ifdef __cplusplus
}
#endif
#endif
