// Dense symmetric eigensolver for the small projected matrix of the Krylov
// method (size m <= 256, FP64): Householder reduction to tridiagonal form,
// then implicit symmetric QR steps with the Wilkinson shift, accumulating
// the orthogonal transforms (Golub and Van Loan, Matrix Computations,
// Sec. 8.3).  Eigenvalues are returned ascending with their vectors.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "internal.h"

namespace sfairsc {

void host_symmetric_eig(int m, double* A, double* w) {
  // A: m x m column-major symmetric; on exit its columns are the eigenvectors.
  std::vector<double> Q((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) Q[(size_t)i * m + i] = 1.0;
  auto a = [&](int i, int j) -> double& { return A[(size_t)j * m + i]; };
  auto q = [&](int i, int j) -> double& { return Q[(size_t)j * m + i]; };

  // Householder: for column k, reflect x = A[k+1:, k] onto alpha e_1.
  std::vector<double> v(m), p(m), wv(m);
  for (int k = 0; k + 2 < m; ++k) {
    const int len = m - k - 1;
    double sig = 0.0;
    for (int i = 0; i < len; ++i) sig += a(k + 1 + i, k) * a(k + 1 + i, k);
    sig = std::sqrt(sig);
    if (sig == 0.0) continue;
    const double x0 = a(k + 1, k);
    const double alpha = x0 >= 0.0 ? -sig : sig;
    for (int i = 0; i < len; ++i) v[i] = a(k + 1 + i, k);
    v[0] -= alpha;
    double vv = 0.0;
    for (int i = 0; i < len; ++i) vv += v[i] * v[i];
    if (vv == 0.0) continue;
    const double beta = 2.0 / vv;
    // p = beta * A22 v
    for (int i = 0; i < len; ++i) {
      double s = 0.0;
      for (int j = 0; j < len; ++j) s += a(k + 1 + i, k + 1 + j) * v[j];
      p[i] = beta * s;
    }
    double vp = 0.0;
    for (int i = 0; i < len; ++i) vp += v[i] * p[i];
    const double K = 0.5 * beta * vp;
    for (int i = 0; i < len; ++i) wv[i] = p[i] - K * v[i];
    for (int j = 0; j < len; ++j)
      for (int i = 0; i < len; ++i) a(k + 1 + i, k + 1 + j) -= v[i] * wv[j] + wv[i] * v[j];
    a(k + 1, k) = alpha;
    a(k, k + 1) = alpha;
    for (int i = 1; i < len; ++i) {
      a(k + 1 + i, k) = 0.0;
      a(k, k + 1 + i) = 0.0;
    }
    // Q <- Q (I - beta v v^T) on columns k+1..m-1
    for (int r = 0; r < m; ++r) {
      double s = 0.0;
      for (int j = 0; j < len; ++j) s += q(r, k + 1 + j) * v[j];
      s *= beta;
      for (int j = 0; j < len; ++j) q(r, k + 1 + j) -= s * v[j];
    }
  }
  std::vector<double> d(m), e(std::max(m - 1, 1), 0.0);
  for (int i = 0; i < m; ++i) d[i] = a(i, i);
  for (int i = 0; i + 1 < m; ++i) e[i] = a(i + 1, i);

  // Implicit symmetric QR with Wilkinson shift on the unreduced trailing block.
  const double eps = std::numeric_limits<double>::epsilon();
  int hi = m - 1;
  int guard = 0;
  while (hi > 0 && guard < 60 * m) {
    if (std::fabs(e[hi - 1]) <= eps * (std::fabs(d[hi - 1]) + std::fabs(d[hi]))) {
      e[hi - 1] = 0.0;
      --hi;
      continue;
    }
    int lo = hi - 1;
    while (lo > 0 && std::fabs(e[lo - 1]) > eps * (std::fabs(d[lo - 1]) + std::fabs(d[lo]))) --lo;
    ++guard;
    const double dd = 0.5 * (d[hi - 1] - d[hi]);
    const double bb = e[hi - 1];
    const double den = dd + (dd >= 0.0 ? 1.0 : -1.0) * std::hypot(dd, bb);
    const double mu = d[hi] - (den != 0.0 ? bb * bb / den : 0.0);
    double x = d[lo] - mu, z = e[lo];
    for (int k = lo; k < hi; ++k) {
      const double r = std::hypot(x, z);
      double c = 1.0, s = 0.0;
      if (r != 0.0) {
        c = x / r;
        s = -z / r;
      }
      if (k > lo) e[k - 1] = c * e[k - 1] - s * z;
      const double ak = d[k], ak1 = d[k + 1], bk = e[k];
      d[k] = c * c * ak - 2.0 * c * s * bk + s * s * ak1;
      d[k + 1] = s * s * ak + 2.0 * c * s * bk + c * c * ak1;
      e[k] = c * s * (ak - ak1) + (c * c - s * s) * bk;
      if (k + 1 < hi) {
        z = -s * e[k + 1];
        e[k + 1] = c * e[k + 1];
        x = e[k];
      }
      for (int rr = 0; rr < m; ++rr) {
        const double qk = q(rr, k), qk1 = q(rr, k + 1);
        q(rr, k) = c * qk - s * qk1;
        q(rr, k + 1) = s * qk + c * qk1;
      }
    }
  }
  std::vector<int> order(m);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int i, int j) { return d[i] < d[j]; });
  for (int c = 0; c < m; ++c) {
    w[c] = d[order[c]];
    for (int r = 0; r < m; ++r) A[(size_t)c * m + r] = Q[(size_t)order[c] * m + r];
  }
}

}  // namespace sfairsc
