// estimate.cu — the parameter estimation of Sec. 2.6 ("Energy Levels &
// Partitioning") on eigenvalues pooled from an observation: truncation to the
// leading eigenvectors that hold a given share of the energy, and level
// partitions by quantiles or by k-means clustering of the eigenvalues. Host
// code.
//
// k-means in one dimension has an exact optimum: the clusters of sorted values
// are contiguous runs, so dynamic programming over (cluster count, last index)
// with prefix sums of x and x^2 finds the partition of least within-cluster
// sum of squares, in O(k n log n) with the monotone split points (ties
// resolved towards the earliest start).
#include <math.h>

#include <algorithm>
#include <vector>

#include "bipp_internal.cuh"
#include "bipp_ss.h"

using namespace bipp;

extern "C" int bipp_ss_energy_neig(int32_t n, const double* mu_desc, double fraction, int32_t* n_eig) {
  if (n < 1 || !mu_desc || !n_eig || !(fraction > 0.0 && fraction <= 1.0))
    return set_global_error(BIPP_ERR_INVALID_ARG, "need n >= 1, mu_desc, n_eig and 0 < fraction <= 1");
  double total = 0.0;
  for (int i = 0; i < n; ++i) {
    if (!isfinite(mu_desc[i])) return set_global_error(BIPP_ERR_INVALID_ARG, "eigenvalues must be finite");
    if (i > 0 && mu_desc[i] > mu_desc[i - 1])
      return set_global_error(BIPP_ERR_INVALID_ARG, "eigenvalues must be in descending order");
    total += fmax(mu_desc[i], 0.0);
  }
  int k = 1;
  double acc = fmax(mu_desc[0], 0.0);
  while (k < n && acc < fraction * total) acc += fmax(mu_desc[k++], 0.0);
  *n_eig = k;
  return BIPP_OK;
}

extern "C" int bipp_ss_kmeans_bounds(int32_t n, const double* values, int32_t n_level, double* level_bounds) {
  if (n < 1 || !values || !level_bounds || n_level < 1 || n_level > n)
    return set_global_error(BIPP_ERR_INVALID_ARG, "need 1 <= n_level <= n, values and level_bounds");
  std::vector<double> x(values, values + n);
  for (double v : x)
    if (!isfinite(v)) return set_global_error(BIPP_ERR_INVALID_ARG, "values must be finite");
  std::sort(x.begin(), x.end());
  std::vector<double> s1(n + 1, 0.0), s2(n + 1, 0.0);
  for (int i = 0; i < n; ++i) {
    s1[i + 1] = s1[i] + x[i];
    s2[i + 1] = s2[i] + x[i] * x[i];
  }
  auto cost = [&](int i, int j) {  // sum of squares about the mean of x[i..j]
    const double m = (double)(j - i + 1), a = s1[j + 1] - s1[i];
    return (s2[j + 1] - s2[i]) - a * a / m;
  };
  const int K = n_level;
  // D[c][j]: least cost of c + 1 clusters over x[0..j]; B[c][j]: start of the last cluster.
  // The least-cost start is non-decreasing in j (the sum-of-squares cost obeys the
  // quadrangle inequality), so each row is filled by divide and conquer over j.
  std::vector<std::vector<double>> D(K, std::vector<double>(n, INFINITY));
  std::vector<std::vector<int>> B(K, std::vector<int>(n, 0));
  for (int jj = 0; jj < n; ++jj) D[0][jj] = cost(0, jj);
  struct Range {
    int jlo, jhi, ilo, ihi;
  };
  std::vector<Range> todo;
  for (int c = 1; c < K; ++c) {
    todo.clear();
    todo.push_back({c, n - 1, c, n - 1});
    while (!todo.empty()) {
      const Range r = todo.back();
      todo.pop_back();
      if (r.jlo > r.jhi) continue;
      const int mid = (r.jlo + r.jhi) / 2;
      double best = INFINITY;
      int arg = r.ilo;
      for (int i = r.ilo; i <= std::min(mid, r.ihi); ++i) {
        const double v = D[c - 1][i - 1] + cost(i, mid);
        if (v < best) {
          best = v;
          arg = i;
        }
      }
      D[c][mid] = best;
      B[c][mid] = arg;
      todo.push_back({r.jlo, mid - 1, r.ilo, arg});
      todo.push_back({mid + 1, r.jhi, arg, r.ihi});
    }
  }
  std::vector<int> start(K);  // first index of each cluster, ascending
  int j = n - 1;
  for (int c = K - 1; c >= 0; --c) {
    start[c] = (c == 0) ? 0 : B[c][j];
    j = start[c] - 1;
  }
  // level 0 = the highest cluster; edges halfway between neighbouring clusters
  for (int l = 0; l < K; ++l) {
    const int c = K - 1 - l;
    const double lo = (c == 0) ? -INFINITY : 0.5 * (x[start[c] - 1] + x[start[c]]);
    const double hi = (c == K - 1) ? INFINITY : 0.5 * (x[start[c + 1] - 1] + x[start[c + 1]]);
    level_bounds[l] = lo;
    level_bounds[K + l] = hi;
  }
  return BIPP_OK;
}

extern "C" int bipp_ss_quantile_bounds(int32_t n, const double* values, int32_t n_level, double* level_bounds) {
  if (n < 1 || !values || !level_bounds || n_level < 1 || n_level > n)
    return set_global_error(BIPP_ERR_INVALID_ARG, "need 1 <= n_level <= n, values and level_bounds");
  std::vector<double> x(values, values + n);
  for (double v : x)
    if (!isfinite(v)) return set_global_error(BIPP_ERR_INVALID_ARG, "values must be finite");
  std::sort(x.begin(), x.end());
  // inner edge q (1 <= q < n_level) sits between the sorted values k-1 and k,
  // k = q n / n_level rounded half to even and clamped to [1, n-1]
  std::vector<double> edge;
  for (int q = 1; q < n_level; ++q) {
    int k = (int)nearbyint((double)q * (double)n / (double)n_level);
    k = std::min(std::max(k, 1), n - 1);
    edge.push_back(0.5 * (x[k - 1] + x[k]));
  }
  std::sort(edge.begin(), edge.end());
  // level 0 holds the largest values: its interval is [edge_last, +inf)
  const int K = n_level;
  for (int l = 0; l < K; ++l) {
    const int c = K - 1 - l;  // interval index in ascending order
    level_bounds[l] = (c == 0) ? -INFINITY : edge[c - 1];
    level_bounds[K + l] = (c == K - 1) ? INFINITY : edge[c];
  }
  return BIPP_OK;
}
