// One-sided Jacobi SVD (Hestenes) of a dense real matrix, used once per handle to factorise the
// double-centred interaction V_c(x, R) = sum_k s_k u_k(x) w_k(R) (rank-k form of the matrix
// elements of the paper's Eq. W).  Columns are orthogonalised by plane rotations in round-robin
// order; the n/2 disjoint pairs of a round are independent and run in parallel (OpenMP).
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

namespace icwf {

// A: m x n column-major (m >= n), overwritten.  On return s (n, descending), U (m x n
// column-major, columns for s > 0), Vr (n x n column-major right singular vectors).
void jacobi_svd(int m, int n, std::vector<double>& A, std::vector<double>& s,
                std::vector<double>& U, std::vector<double>& Vr) {
  Vr.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Vr[(size_t)i * n + i] = 1.0;
  std::vector<double> nrm(n);
  const int np = (n + 1) / 2 * 2;           // even number of slots (one dummy if n is odd)
  std::vector<int> order(np);
  std::iota(order.begin(), order.end(), 0);
  const double tol = 1e-15;
  for (int sweep = 0; sweep < 60; ++sweep) {
    for (int c = 0; c < n; ++c) {
      const double* a = &A[(size_t)c * m];
      double t = 0.0;
      for (int i = 0; i < m; ++i) t += a[i] * a[i];
      nrm[c] = t;
    }
    long rotations = 0;
    for (int round = 0; round < np - 1; ++round) {
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : rotations)
      for (int k = 0; k < np / 2; ++k) {
        int p = order[k], q = order[np - 1 - k];
        if (p >= n || q >= n) continue;
        if (p > q) std::swap(p, q);
        double* ap = &A[(size_t)p * m];
        double* aq = &A[(size_t)q * m];
        const double alpha = nrm[p], beta = nrm[q];
        double gamma = 0.0;
        for (int i = 0; i < m; ++i) gamma += ap[i] * aq[i];
        if (alpha == 0.0 || beta == 0.0 || std::fabs(gamma) <= tol * std::sqrt(alpha * beta)) continue;
        const double zeta = (beta - alpha) / (2.0 * gamma);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = cs * t;
        for (int i = 0; i < m; ++i) {
          const double x = ap[i], y = aq[i];
          ap[i] = cs * x - sn * y;
          aq[i] = sn * x + cs * y;
        }
        double* vp = &Vr[(size_t)p * n];
        double* vq = &Vr[(size_t)q * n];
        for (int i = 0; i < n; ++i) {
          const double x = vp[i], y = vq[i];
          vp[i] = cs * x - sn * y;
          vq[i] = sn * x + cs * y;
        }
        nrm[p] = alpha - t * gamma;
        nrm[q] = beta + t * gamma;
        ++rotations;
      }
      // round-robin rotation of the slots (slot 0 fixed)
      const int last = order[np - 1];
      for (int k = np - 1; k > 1; --k) order[k] = order[k - 1];
      order[1] = last;
    }
    if (rotations == 0) break;
  }
  std::vector<double> sv(n);
  for (int c = 0; c < n; ++c) {
    const double* a = &A[(size_t)c * m];
    double t = 0.0;
    for (int i = 0; i < m; ++i) t += a[i] * a[i];
    sv[c] = std::sqrt(t);
  }
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return sv[x] > sv[y]; });
  s.resize(n);
  U.assign((size_t)m * n, 0.0);
  std::vector<double> V2((size_t)n * n);
  for (int k = 0; k < n; ++k) {
    const int c = idx[k];
    s[k] = sv[c];
    if (sv[c] > 0.0)
      for (int i = 0; i < m; ++i) U[(size_t)k * m + i] = A[(size_t)c * m + i] / sv[c];
    for (int i = 0; i < n; ++i) V2[(size_t)k * n + i] = Vr[(size_t)c * n + i];
  }
  Vr.swap(V2);
}

}  // namespace icwf
