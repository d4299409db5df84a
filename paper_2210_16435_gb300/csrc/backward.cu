// Backward pass of the eigenvalue sum (the differentiation form):
//   f = sum_i gbar_i lambda_i,
//   d lambda_i / d w_ab = (h_ai - h_bi)^2 - lambda_i (h_ai^2 + h_bi^2)
// for the undirected weight w_ab = w_ba.  The eigenvalues are those of the
// pencil (Z^T L Z, Z^T D Z) of Algorithm 2, whose Z spans null(F^T) and does
// not depend on W; with H^T D H = I first-order perturbation gives
// d lambda = h^T (dL - lambda dD) h.  Each stored entry (a, b) gets half.
// Expanded per entry:  A_a + A_b - 2 sum_i gbar_i h_ai h_bi  with
// A_v = sum_i gbar_i (1 - lambda_i) h_vi^2, so one k-term dot per entry (SDDMM).
#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"

namespace sfairsc {

__global__ void vertex_term_kernel(int n, int k, const double* __restrict__ H, const double* __restrict__ lam,
                                   const double* __restrict__ gbar, double* A) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  double s = 0.0;
  for (int i = 0; i < k; ++i) {
    const double hv = H[(size_t)v * k + i];
    s = fma(gbar[i] * (1.0 - lam[i]), hv * hv, s);
  }
  A[v] = s;
}

template <typename MT>
__device__ __forceinline__ double log_weight(MT w);
template <>
__device__ __forceinline__ double log_weight<double>(double w) { return log(w); }
template <>
__device__ __forceinline__ double log_weight<float>(float w) { return (double)logf(w); }
template <>
__device__ __forceinline__ double log_weight<__nv_bfloat16>(__nv_bfloat16 w) { return (double)logf(__bfloat162float(w)); }

// Warp per row: q_a = gbar .* h_a in shared memory, lanes over the row's entries.
template <typename MT>
__global__ void sddmm_kernel(int n, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                             const MT* __restrict__ val, int k, const double* __restrict__ H,
                             const double* __restrict__ gbar, const double* __restrict__ A, double* grad,
                             double bandwidth, double* partial) {
  extern __shared__ double qs[];  // nwarps * k
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double* q = qs + warp * k;
  double gs = 0.0;
  for (int a = blockIdx.x * nw + warp; a < n; a += gridDim.x * nw) {
    for (int i = lane; i < k; i += 32) q[i] = gbar[i] * H[(size_t)a * k + i];
    __syncwarp();
    const double Aa = A[a];
    for (int e = row_ptr[a] + lane; e < row_ptr[a + 1]; e += 32) {
      const int b = col[e];
      const double* hb = H + (size_t)b * k;
      double dot = 0.0;
      for (int i = 0; i < k; ++i) dot = fma(q[i], hb[i], dot);
      const double g = 0.5 * (Aa + A[b] - 2.0 * dot);
      grad[e] = g;
      if (bandwidth > 0.0) {
        const double w = to_f64(val[e]);
        gs += g * w * (-2.0 * log_weight<MT>(val[e])) / bandwidth;
      }
    }
    __syncwarp();
  }
  gs = warp_allsum(gs);
  if (lane == 0) red[warp] = gs;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w];
    partial[blockIdx.x] = s;
  }
}

void launch_backward(int n, const int32_t* row_ptr, const int32_t* col, const void* val, int val_dtype, int k,
                     const double* H, const double* lam, const double* gbar, double* grad, double bandwidth,
                     double* partial, int nblocks, double* A, cudaStream_t s) {
  vertex_term_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, k, H, lam, gbar, A);
  const int T = 256;
  const size_t smem = sizeof(double) * (T / 32) * k;
  switch (val_dtype) {
    case SFAIRSC_F64:
      sddmm_kernel<double><<<nblocks, T, smem, s>>>(n, row_ptr, col, (const double*)val, k, H, gbar, A, grad, bandwidth, partial);
      break;
    case SFAIRSC_F32:
      sddmm_kernel<float><<<nblocks, T, smem, s>>>(n, row_ptr, col, (const float*)val, k, H, gbar, A, grad, bandwidth, partial);
      break;
    default:
      sddmm_kernel<__nv_bfloat16><<<nblocks, T, smem, s>>>(n, row_ptr, col, (const __nv_bfloat16*)val, k, H, gbar, A,
                                                           grad, bandwidth, partial);
  }
  check_cuda(cudaGetLastError(), "backward launch");
}

}  // namespace sfairsc
