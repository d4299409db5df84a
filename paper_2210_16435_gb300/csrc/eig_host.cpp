// Dense symmetric eigensolver for the small projected matrix of the Krylov
// method (size m <= 256, FP64): Householder reduction to tridiagonal form,
// then implicit symmetric QR steps with the Wilkinson shift (Golub and Van
// Loan, Matrix Computations, Sec. 8.3).  Eigenvalues are returned ascending
// with their vectors.
//
// Neither the reduction's reflectors nor the QR rotations depend on the
// eigenvector matrix, so both are recorded and the vectors are formed row by
// row: row r of Q is e_r^T H_0 H_1 ... G_1 G_2 ..., the same operations on each
// row as accumulating Q transform by transform.  Rows are independent, so a few
// host threads each form a contiguous range of rows, and they start as soon as
// the reduction is done: while the calling thread runs the QR iteration, they
// apply its rotations in order as each QR step publishes them.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <limits>
#include <memory>
#include <numeric>
#include <stdexcept>
#include <thread>
#include <vector>

#include "internal.h"

namespace sfairsc {

namespace {

struct Rotation {
  int k;
  double c, s;  // (x_k, x_k+1) <- (c x_k - s x_k+1, s x_k + c x_k+1)
};

// The QR iteration's rotations in fixed-size chunks that never move.  One thread appends and
// publishes the count with release order; readers apply the published prefix (acquire order)
// while the iteration goes on.  finish() publishes the final count, then the end flag, so a
// reader that sees the flag and then reads the count has every rotation.
class RotationLog {
 public:
  static constexpr size_t kChunk = 1024;
  explicit RotationLog(size_t max_count) : chunks_(max_count / kChunk + 1) {}
  // false: max_count reached (cannot happen when max_count bounds the iteration's rotations)
  bool push(const Rotation& r) {
    const size_t c = size_ / kChunk;
    if (c >= chunks_.size()) return false;
    if (size_ % kChunk == 0) chunks_[c].reset(new Rotation[kChunk]);
    chunks_[c][size_ % kChunk] = r;
    ++size_;
    return true;
  }
  void publish() { count_.store(size_, std::memory_order_release); }
  void finish(bool ok) {
    ok_.store(ok, std::memory_order_relaxed);
    count_.store(size_, std::memory_order_release);
    ended_.store(true, std::memory_order_release);
  }
  bool ended() const { return ended_.load(std::memory_order_acquire); }
  size_t published() const { return count_.load(std::memory_order_acquire); }
  bool ok() const { return ok_.load(std::memory_order_relaxed); }
  const Rotation& operator[](size_t i) const { return chunks_[i / kChunk][i % kChunk]; }

 private:
  std::vector<std::unique_ptr<Rotation[]>> chunks_;
  size_t size_ = 0;
  std::atomic<size_t> count_{0};
  std::atomic<bool> ended_{false};
  std::atomic<bool> ok_{true};
};

}  // namespace

bool host_symmetric_eig(int m, double* A, double* w, int max_sweeps) {
  // A: m x m column-major symmetric; on exit its columns are the eigenvectors.
  auto a = [&](int i, int j) -> double& { return A[(size_t)j * m + i]; };

  // Householder: for column k, reflect x = A[k+1:, k] onto alpha e_1.  The
  // reflector I - beta v v^T (v over rows k+1..m-1) is kept for the vectors.
  // Only the lower triangle of the trailing block is read and updated.
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
    // p = beta * A22 v from the lower triangle of A22: column j's rows i > j add to p[i] and, by
    // symmetry, to p[j] (four partial sums for that dot product)
    for (int i = 0; i < len; ++i) p[i] = 0.0;
    {
      const double* __restrict__ vr = v;
      double* __restrict__ pr = p.data();
      for (int j = 0; j < len; ++j) {
        const double* __restrict__ col = &A[(size_t)(k + 1 + j) * m + k + 1];
        const double vj = vr[j];
        double s0 = col[j] * vj, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int i = j + 1;
        for (; i + 4 <= len; i += 4) {
          pr[i] += col[i] * vj;
          pr[i + 1] += col[i + 1] * vj;
          pr[i + 2] += col[i + 2] * vj;
          pr[i + 3] += col[i + 3] * vj;
          s0 += col[i] * vr[i];
          s1 += col[i + 1] * vr[i + 1];
          s2 += col[i + 2] * vr[i + 2];
          s3 += col[i + 3] * vr[i + 3];
        }
        for (; i < len; ++i) {
          pr[i] += col[i] * vj;
          s0 += col[i] * vr[i];
        }
        pr[j] += (s0 + s1) + (s2 + s3);
      }
    }
    for (int i = 0; i < len; ++i) p[i] *= beta;
    double vp = 0.0;
    for (int i = 0; i < len; ++i) vp += v[i] * p[i];
    const double K = 0.5 * beta * vp;
    for (int i = 0; i < len; ++i) wv[i] = p[i] - K * v[i];
    {
      const double* __restrict__ vr = v;
      const double* __restrict__ wr = wv.data();
      for (int j = 0; j < len; ++j) {  // A22 -= v w^T + w v^T, lower triangle
        double* __restrict__ colj = &A[(size_t)(k + 1 + j) * m + k + 1];
        const double vj = vr[j], wj = wr[j];
        for (int i = j; i < len; ++i) colj[i] -= vr[i] * wj + wr[i] * vj;
      }
    }
    a(k + 1, k) = alpha;
    for (int i = 1; i < len; ++i) a(k + 1 + i, k) = 0.0;
  }
  std::vector<double> d(m), e(std::max(m - 1, 1), 0.0);
  for (int i = 0; i < m; ++i) d[i] = a(i, i);
  for (int i = 0; i + 1 < m; ++i) e[i] = a(i + 1, i);

  const int guard_limit = max_sweeps < 0 ? 60 * m : max_sweeps;
  // each QR step records at most m - 1 rotations
  RotationLog rot((size_t)std::max(guard_limit, 0) * (size_t)std::max(m - 1, 0) + 1);
  std::vector<int> where(m);  // column of Q that lands in output column c (set before the log ends)

  // Rows [r0, r1) of Q = I H_0 H_1 ... (rotations in order), written to A's columns in ascending
  // eigenvalue order (A is free: d and e hold T).  A thread's rows are held column by column
  // (x[j * W + t] = row r0 + t's entry j), so every reflector and rotation acts on a contiguous run
  // of W values and each thread reads the recorded transforms once.  The rotations are taken as
  // the QR iteration publishes them.
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
    size_t done = 0;
    for (;;) {
      const bool ended = rot.ended();  // before the count: once ended, the count read next is final
      const size_t avail = rot.published();
      for (; done < avail; ++done) {
        const Rotation& g = rot[done];
        double* x0 = &x[(size_t)g.k * W];
        double* x1 = x0 + W;
        const double c = g.c, sn = g.s;
        for (int t = 0; t < W; ++t) {
          const double a0 = x0[t], a1 = x1[t];
          x0[t] = c * a0 - sn * a1;
          x1[t] = sn * a0 + c * a1;
        }
      }
      if (ended) break;
      std::this_thread::yield();  // the QR step in progress publishes its rotations when it ends
    }
    if (!rot.ok()) return;
    for (int c = 0; c < m; ++c)
      for (int t = 0; t < W; ++t) A[(size_t)c * m + r0 + t] = x[(size_t)where[c] * W + t];
  };
  // one contiguous row range per thread, a few threads (more add start-up cost than they save at
  // m ~ 100); they run during the QR iteration, which this thread does
  const unsigned hw = std::thread::hardware_concurrency();
  const int nt = m < 48 ? 1 : (int)std::min<unsigned>({4u, std::max(1u, hw / 2), (unsigned)((m + 7) / 8)});
  std::vector<std::thread> pool;
  try {
    if (nt > 1)
      for (int t = 0; t < nt; ++t) pool.emplace_back(rows, t * m / nt, (t + 1) * m / nt);
  } catch (...) {  // a thread could not start: the ones running stop without writing
    rot.finish(false);
    for (auto& th : pool) th.join();
    throw;
  }

  // Implicit symmetric QR with Wilkinson shift on the unreduced trailing block.
  int hi = m - 1;
  try {
    const double eps = std::numeric_limits<double>::epsilon();
    int guard = 0;
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
        if (!rot.push(Rotation{k, c, s})) throw std::length_error("rotation log");
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
      rot.publish();
    }
    std::vector<int> order(m);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int i, int j) { return d[i] < d[j]; });
    for (int c = 0; c < m; ++c) {
      w[c] = d[order[c]];
      where[c] = order[c];
    }
  } catch (...) {
    rot.finish(false);  // the row threads stop without writing
    for (auto& th : pool) th.join();
    throw;
  }
  rot.finish(true);
  if (nt > 1) {
    for (auto& th : pool) th.join();
  } else {
    rows(0, m);
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
