/*
 * bipp_oracle.c — FP64 CPU oracle for Bluebild standard synthesis.
 *
 * TEST INFRASTRUCTURE ONLY (see bipp_oracle.h). Every routine is the plain
 * definition of one step of BIPP's standard-synthesis path (arXiv:2310.09200),
 * written for readability, not speed: no blocking, fusion or reordering
 * beyond what the definition states. The only concession to run time is an
 * OpenMP loop over independent pixels in the synthesis and gradient sums.
 */
#include "bipp_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define IDX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

/* Normalised sinc, App. A: sinc(x) = sin(pi x) / (pi x), sinc(0) = 1. */
static double sinc_normalised(double x) {
  if (x == 0.0) return 1.0;
  return sin(M_PI * x) / (M_PI * x);
}

/* Sec. 2.2, Eq. gram: for omnidirectional calibrated antennas the Gram matrix
 * is G_pq = sinc(2 ||b_pq||) with baseline b_pq = (x_p - x_q) / wl. */
int orc_gram(int n, const double* xyz, double wl, double* G) {
  if (n <= 0 || !xyz || !G || !(wl > 0)) return -1;
  for (int q = 0; q < n; ++q) {
    for (int p = 0; p < n; ++p) {
      double bx = (xyz[IDX(p, 0, n)] - xyz[IDX(q, 0, n)]) / wl;
      double by = (xyz[IDX(p, 1, n)] - xyz[IDX(q, 1, n)]) / wl;
      double bz = (xyz[IDX(p, 2, n)] - xyz[IDX(q, 2, n)]) / wl;
      double len = sqrt(bx * bx + by * by + bz * bz);
      G[IDX(p, q, n)] = sinc_normalised(2.0 * len);
    }
  }
  return 0;
}

/* Textbook Cholesky-Banachiewicz factorisation G = L L^T of the real
 * symmetric Gram matrix (used to reduce V a = mu G a to standard form,
 * Sec. 2.3). */
int orc_cholesky(int n, const double* G, double* L) {
  if (n <= 0 || !G || !L) return -1;
  memset(L, 0, sizeof(double) * (size_t)n * n);
  for (int j = 0; j < n; ++j) {
    double s = G[IDX(j, j, n)];
    for (int k = 0; k < j; ++k) s -= L[IDX(j, k, n)] * L[IDX(j, k, n)];
    if (!(s > 0.0)) return -2;
    double ljj = sqrt(s);
    L[IDX(j, j, n)] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double t = G[IDX(i, j, n)];
      for (int k = 0; k < j; ++k) t -= L[IDX(i, k, n)] * L[IDX(j, k, n)];
      L[IDX(i, j, n)] = t / ljj;
    }
  }
  return 0;
}

static double off_norm(int n, const double complex* C) {
  double s = 0.0;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i)
      if (i != j) {
        double a = cabs(C[IDX(i, j, n)]);
        s += a * a;
      }
  return sqrt(s);
}

static double fro_norm(int n, const double complex* C) {
  double s = 0.0;
  for (size_t k = 0; k < (size_t)n * n; ++k) {
    double a = cabs(C[k]);
    s += a * a;
  }
  return sqrt(s);
}

/* Cyclic-by-row Jacobi for a complex Hermitian matrix (the classical method,
 * Golub & Van Loan, "Matrix Computations", Sec. 8.5, carried over to the
 * Hermitian case). For a pivot (p,q) with a = C_pp, b = C_qq and
 * C_pq = r e^{i phi}, the unitary
 *     J = [[ c,            s e^{i phi} ],
 *          [ -s e^{-i phi}, c          ]]   (c, s real)
 * equals diag(1, e^{-i phi}) R diag(1, e^{i phi}) where R = [[c, s], [-s, c]]
 * is the real symmetric Schur rotation of [[a, r], [r, b]]; hence
 * (J^H C J)_pq = 0. C <- J^H C J and Q <- Q J on the two affected columns and
 * rows. */
int orc_jacobi_herm(int n, double complex* C, double* mu, double complex* Q,
                    double tol, int max_sweeps, int* sweeps_out) {
  if (n <= 0 || !C || !mu || !Q) return -1;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) Q[IDX(i, j, n)] = (i == j) ? 1.0 : 0.0;
  double fn = fro_norm(n, C);
  int sweep = 0;
  int converged = (fn == 0.0) || off_norm(n, C) <= tol * fn;
  while (!converged && sweep < max_sweeps) {
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        double complex cpq = C[IDX(p, q, n)];
        double r = cabs(cpq);
        if (r == 0.0) continue;
        double complex eiphi = cpq / r; /* e^{i phi} */
        double a = creal(C[IDX(p, p, n)]);
        double b = creal(C[IDX(q, q, n)]);
        /* symmetric Schur rotation of [[a, r], [r, b]] (GvL Alg. 8.5.1) */
        double tau = (b - a) / (2.0 * r);
        double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t);
        double s = t * c;
        double complex jpq = s * eiphi;        /* J_pq */
        double complex jqp = -s * conj(eiphi); /* J_qp */
        /* columns: C <- C J */
        for (int k = 0; k < n; ++k) {
          double complex ckp = C[IDX(k, p, n)];
          double complex ckq = C[IDX(k, q, n)];
          C[IDX(k, p, n)] = ckp * c + ckq * jqp;
          C[IDX(k, q, n)] = ckp * jpq + ckq * c;
        }
        /* rows: C <- J^H C */
        for (int k = 0; k < n; ++k) {
          double complex cpk = C[IDX(p, k, n)];
          double complex cqk = C[IDX(q, k, n)];
          C[IDX(p, k, n)] = c * cpk + conj(jqp) * cqk;
          C[IDX(q, k, n)] = conj(jpq) * cpk + c * cqk;
        }
        /* the rotated 2x2 block is diagonal by construction */
        C[IDX(p, q, n)] = 0.0;
        C[IDX(q, p, n)] = 0.0;
        C[IDX(p, p, n)] = a - t * r;
        C[IDX(q, q, n)] = b + t * r;
        /* accumulate Q <- Q J */
        for (int k = 0; k < n; ++k) {
          double complex qkp = Q[IDX(k, p, n)];
          double complex qkq = Q[IDX(k, q, n)];
          Q[IDX(k, p, n)] = qkp * c + qkq * jqp;
          Q[IDX(k, q, n)] = qkp * jpq + qkq * c;
        }
      }
    }
    ++sweep;
    converged = off_norm(n, C) <= tol * fn;
  }
  for (int i = 0; i < n; ++i) mu[i] = creal(C[IDX(i, i, n)]);
  if (sweeps_out) *sweeps_out = sweep;
  return converged ? 0 : -3;
}

/* Sec. 2.3, Eq. eigenvaleq: V a = mu G a, solved without inverting G by the
 * standard reduction G = L L^T, C = L^{-1} V L^{-T} (Hermitian), C = Q M Q^H,
 * A = L^{-T} Q, so that A^H G A = Q^H Q = I (G-orthonormal eigenvectors). */
int orc_geneig(int n, const double complex* V, const double* G, double* mu,
               double complex* A, double tol, int max_sweeps, int* sweeps_out) {
  if (n <= 0 || !V || !mu || !A) return -1;
  size_t nn = (size_t)n * n;
  double* L = (double*)malloc(sizeof(double) * nn);
  double complex* X = (double complex*)malloc(sizeof(double complex) * nn);
  double complex* C = (double complex*)malloc(sizeof(double complex) * nn);
  double complex* Q = (double complex*)malloc(sizeof(double complex) * nn);
  double* mu_raw = (double*)malloc(sizeof(double) * n);
  int* order = (int*)malloc(sizeof(int) * n);
  int rc = 0;
  if (!L || !X || !C || !Q || !mu_raw || !order) { rc = -1; goto done; }

  if (G) {
    rc = orc_cholesky(n, G, L);
    if (rc) goto done;
  } else {
    memset(L, 0, sizeof(double) * nn);
    for (int i = 0; i < n; ++i) L[IDX(i, i, n)] = 1.0;
  }
  /* X = L^{-1} V by forward substitution, column by column */
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i < n; ++i) {
      double complex s = V[IDX(i, j, n)];
      for (int k = 0; k < i; ++k) s -= L[IDX(i, k, n)] * X[IDX(k, j, n)];
      X[IDX(i, j, n)] = s / L[IDX(i, i, n)];
    }
  }
  /* C = X L^{-T} = (L^{-1} X^H)^H: forward substitution on the rows of X */
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) {
      double complex s = X[IDX(i, j, n)];
      for (int k = 0; k < j; ++k) s -= C[IDX(i, k, n)] * L[IDX(j, k, n)];
      C[IDX(i, j, n)] = s / L[IDX(j, j, n)];
    }
  }
  /* remove the rounding-level anti-Hermitian part */
  for (int j = 0; j < n; ++j)
    for (int i = 0; i <= j; ++i) {
      double complex h = 0.5 * (C[IDX(i, j, n)] + conj(C[IDX(j, i, n)]));
      if (i == j) h = creal(h);
      C[IDX(i, j, n)] = h;
      C[IDX(j, i, n)] = conj(h);
    }

  rc = orc_jacobi_herm(n, C, mu_raw, Q, tol, max_sweeps, sweeps_out);
  if (rc) goto done;

  /* stable sort by descending eigenvalue (insertion sort on indices) */
  for (int i = 0; i < n; ++i) order[i] = i;
  for (int i = 1; i < n; ++i) {
    int key = order[i];
    int j = i - 1;
    while (j >= 0 && mu_raw[order[j]] < mu_raw[key]) {
      order[j + 1] = order[j];
      --j;
    }
    order[j + 1] = key;
  }
  /* A = L^{-T} Q by back substitution, in sorted column order */
  for (int e = 0; e < n; ++e) {
    int src = order[e];
    mu[e] = mu_raw[src];
    for (int i = n - 1; i >= 0; --i) {
      double complex s = Q[IDX(i, src, n)];
      for (int k = i + 1; k < n; ++k) s -= L[IDX(k, i, n)] * A[IDX(k, e, n)];
      A[IDX(i, e, n)] = s / L[IDX(i, i, n)];
    }
  }
done:
  free(L); free(X); free(C); free(Q); free(mu_raw); free(order);
  return rc;
}

/* Sec. 2.6 "Partitioning" and Alg. 1: an eigenpair joins the level whose
 * interval [lo, hi) holds its eigenvalue; eigenpairs outside every interval
 * are dropped. */
int orc_select_levels(int n_eig, const double* mu, int n_level,
                      const double* bounds, int* level_id) {
  if (n_eig < 0 || n_level <= 0 || !mu || !bounds || !level_id) return -1;
  for (int e = 0; e < n_eig; ++e) {
    level_id[e] = -1;
    for (int l = 0; l < n_level; ++l) {
      double lo = bounds[l], hi = bounds[n_level + l];
      if (lo <= mu[e] && mu[e] < hi) {
        level_id[e] = l;
        break;
      }
    }
  }
  return 0;
}

/* Sec. 2.4, Eq. standard_synthesis, with the per-pixel loop of Alg. 2 and the
 * interval accumulation of Alg. 1: for every pixel r the station phasors
 * exp(-j k <r, p_i>) are formed once (full FP64 argument, libm sin/cos) and
 * reused for every eigenvector. */
void orc_synth_levels(int64_t n_pix, const double* pix, int n_st,
                      const double* st_xyz, double wl, int n_eig,
                      const double complex* W, const double* d,
                      const int* level_id, int n_level, double* img) {
  const double k = 2.0 * M_PI / wl;
#pragma omp parallel
  {
    double complex* ph = (double complex*)malloc(sizeof(double complex) * (size_t)n_st);
#pragma omp for schedule(static)
    for (int64_t r = 0; r < n_pix; ++r) {
      double rx = pix[IDX(r, 0, n_pix)], ry = pix[IDX(r, 1, n_pix)], rz = pix[IDX(r, 2, n_pix)];
      for (int i = 0; i < n_st; ++i) {
        double arg = k * (rx * st_xyz[IDX(i, 0, n_st)] + ry * st_xyz[IDX(i, 1, n_st)] +
                          rz * st_xyz[IDX(i, 2, n_st)]);
        ph[i] = cos(arg) - I * sin(arg); /* exp(-j arg) */
      }
      for (int e = 0; e < n_eig; ++e) {
        int l = level_id[e];
        if (l < 0 || l >= n_level) continue;
        double complex z = 0.0;
        for (int i = 0; i < n_st; ++i) z += ph[i] * W[IDX(i, e, n_st)];
        double m2 = creal(z) * creal(z) + cimag(z) * cimag(z);
        img[IDX(r, l, n_pix)] += d[e] * m2;
      }
    }
    free(ph);
  }
}

/* One collect() step of Alg. 1. */
int orc_ss_step(int64_t n_pix, const double* pix, double wl, int n_level,
                const double* bounds, int n_eig, int filter, int gram_identity,
                int n_st, const double* st_xyz, const double complex* V,
                double* img, double* mu_out, int* level_out,
                double complex* W_out, double tol, int max_sweeps) {
  if (n_pix < 0 || !pix || !bounds || !st_xyz || !V || !img) return -1;
  if (n_st <= 0 || n_eig <= 0 || n_eig > n_st || n_level <= 0) return -1;
  if (filter != 0 && filter != 1) return -1;
  size_t nn = (size_t)n_st * n_st;
  double* G = NULL;
  double* mu = (double*)malloc(sizeof(double) * n_st);
  double complex* A = (double complex*)malloc(sizeof(double complex) * nn);
  double* d = (double*)malloc(sizeof(double) * n_eig);
  int* lev = (int*)malloc(sizeof(int) * n_eig);
  int rc = 0;
  if (!mu || !A || !d || !lev) { rc = -1; goto done; }
  if (!gram_identity) {
    G = (double*)malloc(sizeof(double) * nn);
    if (!G) { rc = -1; goto done; }
    rc = orc_gram(n_st, st_xyz, wl, G);
    if (rc) goto done;
  }
  rc = orc_geneig(n_st, V, G, mu, A, tol, max_sweeps, NULL);
  if (rc) goto done;
  /* truncation to the n_eig leading pairs (Sec. 2.6) is the first n_eig
   * columns of the descending decomposition; filters: LSQ d = mu, STD d = 1 */
  for (int e = 0; e < n_eig; ++e) d[e] = (filter == 0) ? mu[e] : 1.0;
  orc_select_levels(n_eig, mu, n_level, bounds, lev);
  orc_synth_levels(n_pix, pix, n_st, st_xyz, wl, n_eig, A, d, lev, n_level, img);
  if (mu_out) memcpy(mu_out, mu, sizeof(double) * n_eig);
  if (level_out) memcpy(level_out, lev, sizeof(int) * n_eig);
  if (W_out) memcpy(W_out, A, sizeof(double complex) * (size_t)n_st * n_eig);
done:
  free(G); free(mu); free(A); free(d); free(lev);
  return rc;
}

/* Gradient of the level-image loss (differentiation through the synthesis of
 * Eq. standard_synthesis with gains g, Sec. 2.1 and 2.4). With
 * R_l(r) = 2 (I_l(r) - T_l(r)) and W' = diag(conj g) W, the Wirtinger
 * derivatives give
 *   grad_W'[i,e] = 2 sum_r Phi(r,i) d_e R_{l(e)}(r) z_e(r),  Phi = exp(+j k<r,p_i>)
 *   grad_W[i,e]  = g_i grad_W'[i,e]
 *   grad_g[i]    = sum_t sum_e conj(grad_W'_t[i,e]) W_t[i,e].
 * First the forward images are formed, then the pixel sums above. */
int orc_grad(int64_t n_pix, const double* pix, double wl, int n_level,
             int n_t, int n_st, int n_eig, const double* st_xyz,
             const double complex* W, const double* d, const int* level_id,
             const double complex* g, const double* target, double* loss,
             double* img_out, double complex* grad_g, double complex* grad_W) {
  if (n_pix <= 0 || !pix || n_level <= 0 || n_t <= 0 || n_st <= 0 || n_eig <= 0) return -1;
  if (!st_xyz || !W || !d || !level_id || !g || !target || !loss) return -1;
  const double k = 2.0 * M_PI / wl;
  size_t nimg = (size_t)n_pix * n_level;
  size_t nw = (size_t)n_st * n_eig;
  double* img = (double*)calloc(nimg, sizeof(double));
  double complex* Wp = (double complex*)malloc(sizeof(double complex) * nw * n_t);
  double complex* gWp = (double complex*)calloc(nw * n_t, sizeof(double complex));
  int rc = 0;
  if (!img || !Wp || !gWp) { rc = -1; goto done; }
  for (int t = 0; t < n_t; ++t)
    for (int e = 0; e < n_eig; ++e)
      for (int i = 0; i < n_st; ++i)
        Wp[t * nw + IDX(i, e, n_st)] = conj(g[i]) * W[t * nw + IDX(i, e, n_st)];

  /* forward: I_l(r) */
#pragma omp parallel
  {
    double complex* ph = (double complex*)malloc(sizeof(double complex) * (size_t)n_st);
#pragma omp for schedule(static)
    for (int64_t r = 0; r < n_pix; ++r) {
      double rx = pix[IDX(r, 0, n_pix)], ry = pix[IDX(r, 1, n_pix)], rz = pix[IDX(r, 2, n_pix)];
      for (int t = 0; t < n_t; ++t) {
        const double* p = st_xyz + (size_t)t * n_st * 3;
        for (int i = 0; i < n_st; ++i) {
          double arg = k * (rx * p[IDX(i, 0, n_st)] + ry * p[IDX(i, 1, n_st)] + rz * p[IDX(i, 2, n_st)]);
          ph[i] = cos(arg) - I * sin(arg);
        }
        for (int e = 0; e < n_eig; ++e) {
          int l = level_id[t * n_eig + e];
          if (l < 0 || l >= n_level) continue;
          double complex z = 0.0;
          for (int i = 0; i < n_st; ++i) z += ph[i] * Wp[t * nw + IDX(i, e, n_st)];
          img[IDX(r, l, n_pix)] += d[t * n_eig + e] * (creal(z) * creal(z) + cimag(z) * cimag(z));
        }
      }
    }
    free(ph);
  }
  double L = 0.0;
  for (size_t q = 0; q < nimg; ++q) {
    double diff = img[q] - target[q];
    L += diff * diff;
  }
  *loss = L;

  /* backward: grad_W'[t,i,e] = 2 sum_r Phi(r,i) d_e R_l(r) z_e(r).
   * The pixel sum is split over threads into per-thread partial sums that are
   * added together afterwards (one at a time, under a lock). */
  if (grad_g || grad_W) {
#pragma omp parallel
    {
      double complex* ph = (double complex*)malloc(sizeof(double complex) * (size_t)n_st);
      double complex* part = (double complex*)calloc(nw * n_t, sizeof(double complex));
#pragma omp for schedule(static)
      for (int64_t r = 0; r < n_pix; ++r) {
        double rx = pix[IDX(r, 0, n_pix)], ry = pix[IDX(r, 1, n_pix)], rz = pix[IDX(r, 2, n_pix)];
        for (int t = 0; t < n_t; ++t) {
          const double* p = st_xyz + (size_t)t * n_st * 3;
          for (int i = 0; i < n_st; ++i) {
            double arg = k * (rx * p[IDX(i, 0, n_st)] + ry * p[IDX(i, 1, n_st)] + rz * p[IDX(i, 2, n_st)]);
            ph[i] = cos(arg) - I * sin(arg); /* conj(Phi(r,i)) */
          }
          for (int e = 0; e < n_eig; ++e) {
            int l = level_id[t * n_eig + e];
            if (l < 0 || l >= n_level) continue;
            double complex z = 0.0;
            for (int i = 0; i < n_st; ++i) z += ph[i] * Wp[t * nw + IDX(i, e, n_st)];
            double Rl = 2.0 * (img[IDX(r, l, n_pix)] - target[IDX(r, l, n_pix)]);
            double complex y = d[t * n_eig + e] * Rl * z;
            for (int i = 0; i < n_st; ++i)
              part[t * nw + IDX(i, e, n_st)] += 2.0 * conj(ph[i]) * y; /* Phi = conj(ph) */
          }
        }
      }
#pragma omp critical
      {
        for (size_t q = 0; q < nw * n_t; ++q) gWp[q] += part[q];
      }
      free(ph);
      free(part);
    }
    if (grad_W)
      for (int t = 0; t < n_t; ++t)
        for (int e = 0; e < n_eig; ++e)
          for (int i = 0; i < n_st; ++i)
            grad_W[t * nw + IDX(i, e, n_st)] = g[i] * gWp[t * nw + IDX(i, e, n_st)];
    if (grad_g)
      for (int i = 0; i < n_st; ++i) {
        double complex s = 0.0;
        for (int t = 0; t < n_t; ++t)
          for (int e = 0; e < n_eig; ++e)
            s += conj(gWp[t * nw + IDX(i, e, n_st)]) * W[t * nw + IDX(i, e, n_st)];
        grad_g[i] = s;
      }
  }
  if (img_out) memcpy(img_out, img, sizeof(double) * nimg);
done:
  free(img); free(Wp); free(gWp);
  return rc;
}
