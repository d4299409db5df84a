// Dense symmetric eigensolver for the small projected matrix of the Krylov
// method (size m <= 256, FP64): Householder reduction to tridiagonal form,
// then implicit symmetric QR steps with the Wilkinson shift (Golub and Van
// Loan, Matrix Computations, Sec. 8.3).  Eigenvalues are returned ascending
// with their vectors.
//
// Neither the reduction's reflectors nor the QR rotations depend on the
// eigenvector matrix, so both are recorded and the vectors are formed
// afterwards row by row: row r of Q is e_r^T H_0 H_1 ... G_1 G_2 ..., the
// same operations on each row as accumulating Q transform by transform.
// Rows are independent, so ranges of rows go to a few host threads.
#include <algorithm>
#include <cmath>
#include <limits>
#include <numeric>
#include <thread>
#include <vector>

#include "internal.h"

namespace sfairsc {

namespace {

struct Rotation {
  int k;
  double c, s;  // (x_k, x_k+1) <- (c x_k - s x_k+1, s x_k + c x_k+1)
};

}  // namespace

bool host_symmetric_eig(int m, double* A, double* w, int max_sweeps) {
  // A: m x m column-major symmetric; on exit its columns are the eigenvectors.
  auto a = [&](int i, int j) -> double& { return A[(size_t)j * m + i]; };

  // Householder: for column k, reflect x = A[k+1:, k] onto alpha e_1.  The
  // reflector I - beta v v^T (v over rows k+1..m-1) is kept for the vectors.
  std::vector<double> refl((size_t)m * m, 0.0);  // v of step k at refl[k * m + k + 1 ..]
  std::vector<double> rbeta(m, 0.0);             // 0: no reflection at this step
  std::vector<double> p(m), wv(m);
  for (int k = 0; k + 2 < m; ++k) {
    const int len = m - k - 1;
    double sig = 0.0;
    for (int i = 0; i < len; ++i) sig += a(k + 1 + i, k) * a(k + 1 + i, k);
    sig = std::sqrt(sig);
    if (sig == 0.0) continue;
    const double x0 = a(k + 1, k);
    const double alpha = x0 >= 0.0 ? -sig : sig;
    double* v = &refl[(size_t)k * m + k + 1];
    for (int i = 0; i < len; ++i) v[i] = a(k + 1 + i, k);
    v[0] -= alpha;
    double vv = 0.0;
    for (int i = 0; i < len; ++i) vv += v[i] * v[i];
    if (vv == 0.0) continue;
    const double beta = 2.0 / vv;
    rbeta[k] = beta;
    // p = beta * A22 v, down the columns of A22
    for (int i = 0; i < len; ++i) p[i] = 0.0;
    for (int j = 0; j < len; ++j) {
      const double vj = v[j];
      const double* col = &A[(size_t)(k + 1 + j) * m + k + 1];
      for (int i = 0; i < len; ++i) p[i] += col[i] * vj;
    }
    for (int i = 0; i < len; ++i) p[i] *= beta;
    double vp = 0.0;
    for (int i = 0; i < len; ++i) vp += v[i] * p[i];
    const double K = 0.5 * beta * vp;
    for (int i = 0; i < len; ++i) wv[i] = p[i] - K * v[i];
    {
      const double* __restrict__ vr = v;
      const double* __restrict__ wr = wv.data();
      for (int j = 0; j < len; ++j) {
        double* __restrict__ colj = &A[(size_t)(k + 1 + j) * m + k + 1];
        const double vj = vr[j], wj = wr[j];
        for (int i = 0; i < len; ++i) colj[i] -= vr[i] * wj + wr[i] * vj;
      }
    }
    a(k + 1, k) = alpha;
    a(k, k + 1) = alpha;
    for (int i = 1; i < len; ++i) {
      a(k + 1 + i, k) = 0.0;
      a(k, k + 1 + i) = 0.0;
    }
  }
  std::vector<double> d(m), e(std::max(m - 1, 1), 0.0);
  for (int i = 0; i < m; ++i) d[i] = a(i, i);
  for (int i = 0; i + 1 < m; ++i) e[i] = a(i + 1, i);

  // Implicit symmetric QR with Wilkinson shift on the unreduced trailing block.
  const double eps = std::numeric_limits<double>::epsilon();
  std::vector<Rotation> rot;
  rot.reserve((size_t)8 * m * m);
  int hi = m - 1;
  int guard = 0;
  const int guard_limit = max_sweeps < 0 ? 60 * m : max_sweeps;
  while (hi > 0 && guard < guard_limit) {
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
      // entries of the projected matrix are far from the overflow range, so
      // the plain root serves (std::hypot's scaling dominated the loop)
      const double r = std::sqrt(x * x + z * z);
      double c = 1.0, s = 0.0;
      if (r != 0.0) {
        c = x / r;
        s = -z / r;
      }
      rot.push_back(Rotation{k, c, s});
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
    }
  }
  std::vector<int> order(m);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int i, int j) { return d[i] < d[j]; });
  std::vector<int> where(m);  // column of Q that lands in output column c
  for (int c = 0; c < m; ++c) {
    w[c] = d[order[c]];
    where[c] = order[c];
  }

  // Rows [r0, r1) of Q = I H_0 H_1 ... (rotations in order), written to A's columns in ascending
  // eigenvalue order (A is free: d and e hold T).  A thread's rows are held column by column
  // (x[j * W + t] = row r0 + t's entry j), so every reflector and rotation acts on a contiguous run
  // of W values and each thread reads the recorded transforms once.
  auto rows = [&](int r0, int r1) {
    const int W = r1 - r0;
    if (W <= 0) return;
    std::vector<double> x((size_t)m * W, 0.0), sbuf(W);
    for (int t = 0; t < W; ++t) x[(size_t)(r0 + t) * W + t] = 1.0;
    for (int k = 0; k + 2 < m; ++k) {
      const double beta = rbeta[k];
      if (beta == 0.0) continue;
      const double* v = &refl[(size_t)k * m + k + 1];
      const int len = m - k - 1;
      double* s = sbuf.data();
      for (int t = 0; t < W; ++t) s[t] = 0.0;
      for (int jj = 0; jj < len; ++jj) {
        const double* xj = &x[(size_t)(k + 1 + jj) * W];
        const double vj = v[jj];
        for (int t = 0; t < W; ++t) s[t] += xj[t] * vj;
      }
      for (int t = 0; t < W; ++t) s[t] *= beta;
      for (int jj = 0; jj < len; ++jj) {
        double* xj = &x[(size_t)(k + 1 + jj) * W];
        const double vj = v[jj];
        for (int t = 0; t < W; ++t) xj[t] -= s[t] * vj;
      }
    }
    for (const Rotation& g : rot) {
      double* x0 = &x[(size_t)g.k * W];
      double* x1 = x0 + W;
      const double c = g.c, sn = g.s;
      for (int t = 0; t < W; ++t) {
        const double a0 = x0[t], a1 = x1[t];
        x0[t] = c * a0 - sn * a1;
        x1[t] = sn * a0 + c * a1;
      }
    }
    for (int c = 0; c < m; ++c)
      for (int t = 0; t < W; ++t) A[(size_t)c * m + r0 + t] = x[(size_t)where[c] * W + t];
  };
  // one contiguous row range per thread, a few threads (more add start-up cost than they save at
  // m ~ 100)
  const unsigned hw = std::thread::hardware_concurrency();
  const int nt = m < 48 ? 1 : (int)std::min<unsigned>({4u, std::max(1u, hw / 2), (unsigned)((m + 7) / 8)});
  if (nt <= 1) {
    rows(0, m);
  } else {
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) pool.emplace_back(rows, t * m / nt, (t + 1) * m / nt);
    rows(0, m / nt);
    for (auto& th : pool) th.join();
  }
  return hi <= 0;
}

bool host_symmetric_eig_jacobi(int m, double* A, double* w) {
  // Cyclic Jacobi (Golub and Van Loan, Sec. 8.5): sweep over all (p, q) pairs,
  // zeroing a_pq by a plane rotation chosen with |angle| <= pi/4, until the
  // off-diagonal mass is below eps^2 of the total.  V accumulates the rotations.
  auto a = [&](int i, int j) -> double& { return A[(size_t)j * m + i]; };
  for (size_t i = 0; i < (size_t)m * m; ++i)
    if (!std::isfinite(A[i])) return false;
  std::vector<double> V((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) V[(size_t)i * m + i] = 1.0;
  const double eps = std::numeric_limits<double>::epsilon();
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int j = 0; j < m; ++j)
      for (int i = 0; i < m; ++i) {
        const double x = a(i, j) * a(i, j);
        tot += x;
        if (i != j) off += x;
      }
    if (off <= eps * eps * tot || off == 0.0) break;
    for (int p = 0; p < m - 1; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double apq = a(p, q);
        if (apq == 0.0) continue;
        // tan of the rotation angle: t = sign(tau) / (|tau| + sqrt(1 + tau^2)), tau = (a_qq - a_pp) / (2 a_pq)
        const double tau = (a(q, q) - a(p, p)) / (2.0 * apq);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < m; ++k) {  // columns p, q: A <- A J
          const double akp = a(k, p), akq = a(k, q);
          a(k, p) = c * akp - s * akq;
          a(k, q) = s * akp + c * akq;
        }
        for (int k = 0; k < m; ++k) {  // rows p, q: A <- J^T A
          const double apk = a(p, k), aqk = a(q, k);
          a(p, k) = c * apk - s * aqk;
          a(q, k) = s * apk + c * aqk;
        }
        for (int k = 0; k < m; ++k) {
          double* vp = &V[(size_t)p * m + k];
          double* vq = &V[(size_t)q * m + k];
          const double x = *vp, y = *vq;
          *vp = c * x - s * y;
          *vq = s * x + c * y;
        }
      }
  }
  std::vector<int> order(m);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int i, int j) { return a(i, i) < a(j, j); });
  std::vector<double> d(m);
  for (int i = 0; i < m; ++i) d[i] = a(i, i);
  for (int c = 0; c < m; ++c) {
    w[c] = d[order[c]];
    for (int k = 0; k < m; ++k) A[(size_t)c * m + k] = V[(size_t)order[c] * m + k];
  }
  return true;
}

}  // namespace sfairsc
