// Kernels of the eigenvector-level backward pass: the gradient of a loss on H
// (and on the eigenvalues) with respect to the edge weights.
//
// For the generalized eigenvectors h_i of the fair problem (Algorithm 2's
// pencil, H^T D H = I, simple eigenvalues), first-order perturbation gives
// v_i = sum_{j != i} h_j (h_j^T gbar_i) / (lambda_i - lambda_j) and, per
// undirected weight w_ab,
//   dloss/dw_ab = sum_i (v_ia - v_ib)(h_ia - h_ib) - lambda_i (v_ia h_ia + v_ib h_ib)
//                       - c_i (h_ia^2 + h_ib^2) / 2,   c_i = gbar_i^T h_i.
// In the normalized coordinates x = D^{1/2} h (eigenvectors of L_n^sigma in
// null(C^T)), v_i = D^{-1/2} z_i with z_i = sum_{j != i} x_j x_j^T b_i / (lambda_i
// - lambda_j), b_i = P D^{-1/2} gbar_i.  The j <= k terms are formed from the
// computed X; the rest is -(A - lambda_i I)^{-1} applied to b_i with the
// computed eigenvectors projected out, where A - lambda_i I is positive
// definite (its eigenvalues there are lambda_j - lambda_i, j > k): conjugate
// gradients, k systems at once, on the FP64 operator.
//
// The kernels here: column-major block helpers (scaled transposes, Gram
// blocks X^T Y, small right products X C, column dots, CG updates) and the
// vertex pass that prepares the SDDMM over W's pattern.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace sfairsc {

// out[r + i n] = G[r k + i] * s[r] (divide: / s[r]); row-major n x k to column-major, scaled per row
__global__ void rows_to_cols_scaled_kernel(int n, int k, const double* __restrict__ G, const double* __restrict__ s,
                                           int divide, double* out) {
  const int64_t total = (int64_t)n * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / k, i = e % k;
    out[r + i * (int64_t)n] = divide ? G[e] / s[r] : G[e] * s[r];
  }
}

void launch_rows_to_cols_scaled(int n, int k, const double* G, const double* s, int divide, double* out,
                                cudaStream_t st) {
  rows_to_cols_scaled_kernel<<<1024, 256, 0, st>>>(n, k, G, s, divide, out);
  check_cuda(cudaGetLastError(), "rows to cols launch");
}

// partial[b][i k2 + j] = sum over block b's rows of X[r + i n] Y[r + j n]; 64-row tiles staged in
// shared memory (k1 + k2 columns), thread q owns the entries q, q + 256, ... (k1 k2 <= 64 * 64).
__global__ void __launch_bounds__(256) col_gram_kernel(int n, int k1, const double* __restrict__ X, int k2,
                                                       const double* __restrict__ Y, double* partial) {
  extern __shared__ double tile[];  // 64 x (k1 + k2), row-major
  const int w = k1 + k2, nq = k1 * k2;
  double acc[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) acc[j] = 0.0;
  for (int t0 = blockIdx.x * 64; t0 < n; t0 += gridDim.x * 64) {
    const int rows = min(64, n - t0);
    __syncthreads();
    for (int e = threadIdx.x; e < 64 * w; e += blockDim.x) {
      const int c = e / 64, rr = e % 64;  // column-major reads: consecutive threads, consecutive rows
      double v = 0.0;
      if (rr < rows) v = c < k1 ? X[(size_t)t0 + rr + (size_t)c * n] : Y[(size_t)t0 + rr + (size_t)(c - k1) * n];
      tile[rr * w + c] = v;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int q = threadIdx.x + j * blockDim.x;
      if (q < nq) {
        const int i = q / k2, jj = q % k2;
        double s = 0.0;
        for (int rr = 0; rr < rows; ++rr) s = fma(tile[rr * w + i], tile[rr * w + k1 + jj], s);
        acc[j] += s;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int q = threadIdx.x + j * blockDim.x;
    if (q < nq) partial[(size_t)blockIdx.x * nq + q] = acc[j];
  }
}

void launch_col_gram(int n, int k1, const double* X, int k2, const double* Y, double* partial, int nblocks,
                     cudaStream_t s) {
  if (k1 * k2 > 16 * 256 || k1 + k2 > 128) fail(SFAIRSC_ERR_UNSUPPORTED, "Gram block too wide");
  const size_t smem = sizeof(double) * 64 * (k1 + k2);
  check_cuda(cudaFuncSetAttribute(col_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "attr");
  col_gram_kernel<<<nblocks, 256, smem, s>>>(n, k1, X, k2, Y, partial);
  check_cuda(cudaGetLastError(), "col gram launch");
}

// out[:, j] = beta out[:, j] + sum_i X[:, i] C[i k2 + j] (column-major n x k1 times k1 x k2);
// 64-row tiles of X staged in shared memory, C in shared memory.
__global__ void __launch_bounds__(256) col_gemm_kernel(int n, int k1, const double* __restrict__ X, int k2,
                                                       const double* __restrict__ C, double beta, double* out) {
  extern __shared__ double sm[];
  double* Cs = sm;               // k1 x k2
  double* Xs = sm + k1 * k2;     // 64 x k1, row-major
  for (int e = threadIdx.x; e < k1 * k2; e += blockDim.x) Cs[e] = C[e];
  for (int t0 = blockIdx.x * 64; t0 < n; t0 += gridDim.x * 64) {
    const int rows = min(64, n - t0);
    __syncthreads();
    for (int e = threadIdx.x; e < 64 * k1; e += blockDim.x) {
      const int c = e / 64, rr = e % 64;
      Xs[rr * k1 + c] = rr < rows ? X[(size_t)t0 + rr + (size_t)c * n] : 0.0;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 64 * k2; e += blockDim.x) {
      const int j = e / 64, rr = e % 64;
      if (rr >= rows) continue;
      double s = 0.0;
      for (int i = 0; i < k1; ++i) s = fma(Xs[rr * k1 + i], Cs[i * k2 + j], s);
      double* o = out + (size_t)t0 + rr + (size_t)j * n;
      *o = beta == 0.0 ? s : fma(beta, *o, s);
    }
  }
}

void launch_col_gemm(int n, int k1, const double* X, int k2, const double* C, double beta, double* out,
                     cudaStream_t s) {
  const size_t smem = sizeof(double) * ((size_t)k1 * k2 + 64 * (size_t)k1);
  if (smem > 200 * 1024) fail(SFAIRSC_ERR_UNSUPPORTED, "too many columns for the vector gradient");
  check_cuda(cudaFuncSetAttribute(col_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "attr");
  const int nb = std::max(1, std::min(1024, (n + 63) / 64));
  col_gemm_kernel<<<nb, 256, smem, s>>>(n, k1, X, k2, C, beta, out);
  check_cuda(cudaGetLastError(), "col gemm launch");
}

// partial[b][i] = sum over block b's rows of A[r + i n] B[r + i n] (warp per column)
__global__ void col_dots_kernel(int n, int k, const double* __restrict__ A, const double* __restrict__ B,
                                double* partial) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int per = (n + gridDim.x - 1) / gridDim.x;
  const int r0 = blockIdx.x * per, r1 = min(n, r0 + per);
  for (int i = warp; i < k; i += nw) {
    double s = 0.0;
    for (int r = r0 + lane; r < r1; r += 32) s = fma(A[(size_t)r + (size_t)i * n], B[(size_t)r + (size_t)i * n], s);
    s = warp_allsum(s);
    if (lane == 0) partial[(size_t)blockIdx.x * k + i] = s;
  }
}

void launch_col_dots(int n, int k, const double* A, const double* B, double* partial, int nblocks, cudaStream_t s) {
  col_dots_kernel<<<nblocks, 256, 0, s>>>(n, k, A, B, partial);
  check_cuda(cudaGetLastError(), "col dots launch");
}

// Q[:, i] -= shift[i] P[:, i]
__global__ void col_shift_kernel(int n, int k, double* Q, const double* __restrict__ P, const double* __restrict__ shift) {
  const int64_t total = (int64_t)n * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    Q[e] = fma(-shift[e / n], P[e], Q[e]);
}

// Y[:, i] += alpha[i] P[:, i];  R[:, i] -= alpha[i] Q[:, i]
__global__ void cg_update_kernel(int n, int k, double* Y, double* R, const double* __restrict__ P,
                                 const double* __restrict__ Q, const double* __restrict__ alpha) {
  const int64_t total = (int64_t)n * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const double a = alpha[e / n];
    Y[e] = fma(a, P[e], Y[e]);
    R[e] = fma(-a, Q[e], R[e]);
  }
}

// P[:, i] = R[:, i] + beta[i] P[:, i]
__global__ void cg_direction_kernel(int n, int k, double* P, const double* __restrict__ R,
                                    const double* __restrict__ beta) {
  const int64_t total = (int64_t)n * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    P[e] = fma(beta[e / n], P[e], R[e]);
}

void launch_col_shift(int n, int k, double* Q, const double* P, const double* shift, cudaStream_t s) {
  col_shift_kernel<<<1024, 256, 0, s>>>(n, k, Q, P, shift);
  check_cuda(cudaGetLastError(), "col shift launch");
}
void launch_cg_update(int n, int k, double* Y, double* R, const double* P, const double* Q, const double* alpha,
                      cudaStream_t s) {
  cg_update_kernel<<<1024, 256, 0, s>>>(n, k, Y, R, P, Q, alpha);
  check_cuda(cudaGetLastError(), "cg update launch");
}
void launch_cg_direction(int n, int k, double* P, const double* R, const double* beta, cudaStream_t s) {
  cg_direction_kernel<<<1024, 256, 0, s>>>(n, k, P, R, beta);
  check_cuda(cudaGetLastError(), "cg direction launch");
}

// Vertex pass of the vector backward: with H (row-major n x k), Zc (column-major n x k, the z_i in
// the normalized coordinates) and dinv = D^{-1/2}, form v = D^{-1/2} z and per vertex a
//   Gp row  [h_a, v_a]              (gathered at the other end of each entry),
//   Qp row  [(v_a + 2 glam .* h_a) / 2, h_a / 2],
//   A_a  =  sum_i (1 - lambda_i) (v_ia + glam_i h_ia) h_ia - c_i h_ia^2 / 2,
// so that the SDDMM's (A_a + A_b - 2 Qp_a . Gp_b) / 2 is the per-entry gradient.  Rows padded to kp.
__global__ void vector_vertex_kernel(int n, int k, int kp, const double* __restrict__ H, const double* __restrict__ Zc,
                                     const double* __restrict__ dinv, const double* __restrict__ lam,
                                     const double* __restrict__ glam, const double* __restrict__ cvec, double* A,
                                     double* Qp, double* Gp) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const double di = dinv[r];
  double a = 0.0;
  double* q = Qp + (size_t)r * kp;
  double* g = Gp + (size_t)r * kp;
  for (int i = 0; i < k; ++i) {
    const double hv = H[(size_t)r * k + i];
    const double vv = di * Zc[(size_t)r + (size_t)i * n];
    const double gl = glam ? glam[i] : 0.0;
    a = fma((1.0 - lam[i]) * (vv + gl * hv), hv, a);
    a = fma(-0.5 * cvec[i] * hv, hv, a);
    g[i] = hv;
    g[k + i] = vv;
    q[i] = 0.5 * vv + gl * hv;
    q[k + i] = 0.5 * hv;
  }
  for (int i = 2 * k; i < kp; ++i) {
    g[i] = 0.0;
    q[i] = 0.0;
  }
  A[r] = a;
}

void launch_vector_vertex(int n, int k, int kp, const double* H, const double* Zc, const double* dinv,
                          const double* lam, const double* glam, const double* cvec, double* A, double* Qp, double* Gp,
                          cudaStream_t s) {
  vector_vertex_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, k, kp, H, Zc, dinv, lam, glam, cvec, A, Qp, Gp);
  check_cuda(cudaGetLastError(), "vector vertex launch");
}

}  // namespace sfairsc
