/*
 * bipp_oracle.h — FP64 CPU oracle for Bluebild standard synthesis.
 *
 * TEST INFRASTRUCTURE ONLY. This library is the slow, plain, obviously
 * correct statement of what the standard-synthesis path computes (BIPP,
 * arXiv:2310.09200, Sec. 2.2-2.6 and Algorithms 1-2). Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it; the
 * GPU library never includes, links or calls it, and it shares no code with
 * the GPU library.
 *
 * Conventions (all arrays column-major, as the paper's interface prescribes,
 * Sec. 3.2 "Input data"):
 *   - positions / directions: n x 3 doubles, column j holds coordinate j.
 *   - complex matrices: interleaved (re, im) doubles, C99 double complex.
 *   - level bounds: n_level x 2 doubles, column 0 = lo, column 1 = hi, and an
 *     eigenvalue mu belongs to level l iff lo_l <= mu < hi_l (first match).
 *   - phase sign: the synthesised field of eigenvector w at direction r is
 *     z(r) = sum_i exp(-j 2 pi <r, p_i> / wl) w_i  (Eq. standard_synthesis),
 *     so that a source emitting exp(+j 2 pi <r_s, p_i>/wl) images at r_s.
 *
 * Error codes: 0 ok, -1 invalid argument, -2 Gram not positive definite,
 * -3 Jacobi did not converge within max_sweeps.
 */
#ifndef BIPP_ORACLE_H
#define BIPP_ORACLE_H
#include <complex.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Gram matrix, Eq. gram with sinc(x) = sin(pi x)/(pi x) (App. A):
 * G_ij = sinc(2 ||p_i - p_j|| / wl). G: n x n. */
int orc_gram(int n, const double* xyz, double wl, double* G);

/* Cholesky G = L L^T (lower L, n x n, upper part zeroed). -2 if not PD. */
int orc_cholesky(int n, const double* G, double* L);

/* Cyclic-by-row complex Jacobi on Hermitian C (n x n, overwritten by the
 * rotated matrix). On return mu[i] = C_ii (unsorted) and Q (n x n) holds the
 * accumulated unitary with C_in = Q diag(mu) Q^H. Stops when
 * off(C) <= tol * ||C||_F. *sweeps_out = sweeps used. */
int orc_jacobi_herm(int n, double complex* C, double* mu, double complex* Q,
                    double tol, int max_sweeps, int* sweeps_out);

/* Generalised Hermitian eigenproblem V a = mu G a (Eq. eigenvaleq).
 * G == NULL means G = I. Returns all n eigenpairs sorted by descending mu
 * (ties: lower Jacobi index first), A columns G-orthonormal (A^H G A = I). */
int orc_geneig(int n, const double complex* V, const double* G, double* mu,
               double complex* A, double tol, int max_sweeps, int* sweeps_out);

/* Level id of each of the n_eig leading eigenvalues (Sec. 2.6, Alg. 1):
 * level_id[e] = first l with lo_l <= mu[e] < hi_l, or -1 (dropped). */
int orc_select_levels(int n_eig, const double* mu, int n_level,
                      const double* bounds, int* level_id);

/* Per-pixel direct sum (Alg. 2 + Alg. 1 accumulation):
 *   img[r + l n_pix] += sum_{e: level_id[e]==l} d[e] |sum_i exp(-j k <r,p_i>) W_ie|^2
 * with k = 2 pi / wl. W: n_st x n_eig. img: n_pix x n_level (accumulated). */
void orc_synth_levels(int64_t n_pix, const double* pix, int n_st,
                      const double* st_xyz, double wl, int n_eig,
                      const double complex* W, const double* d,
                      const int* level_id, int n_level, double* img);

/* One full collect() step (Alg. 1): Gram -> generalised eigensolve -> keep
 * the n_eig leading pairs -> filter weights -> levels -> synthesis into img.
 * filter: 0 = LSQ (d = mu), 1 = STD (d = 1). gram_identity: 1 => G = I.
 * Optional outputs (may be NULL): mu_out (n_eig), level_out (n_eig),
 * W_out (n_st x n_eig). */
int orc_ss_step(int64_t n_pix, const double* pix, double wl, int n_level,
                const double* bounds, int n_eig, int filter, int gram_identity,
                int n_st, const double* st_xyz, const double complex* V,
                double* img, double* mu_out, int* level_out,
                double complex* W_out, double tol, int max_sweeps);

/* Gradient of L = sum_{l,r} (I_l(r) - T_l(r))^2 for the gain-corrected model
 *   z_{t,e}(r) = sum_i conj(g_i) exp(-j k <r, p_{t,i}>) W_{t,ie},
 *   I_l(r)     = sum_t sum_{e: level==l} d_{t,e} |z_{t,e}(r)|^2,
 * with complex gradients in the convention grad = dL/dRe + j dL/dIm.
 * st_xyz: n_t blocks of n_st x 3; W, grad_W: n_t blocks of n_st x n_eig;
 * d, level_id: n_t blocks of n_eig; target, img_out: n_pix x n_level.
 * Returns L in *loss. Any of img_out, grad_g, grad_W may be NULL. */
int orc_grad(int64_t n_pix, const double* pix, double wl, int n_level,
             int n_t, int n_st, int n_eig, const double* st_xyz,
             const double complex* W, const double* d, const int* level_id,
             const double complex* g, const double* target, double* loss,
             double* img_out, double complex* grad_g, double complex* grad_W);

#ifdef __cplusplus
}
#endif
#endif
