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

// One pass over the vertices: A_v and a copy of H with rows padded to KP
// doubles (a multiple of 4: each row starts on a 32-byte sector and the SDDMM
// gathers it as KP / 2 independent 16-byte loads).
// normalized = 0 (L = D - W, H^T H = I): d lambda / d w_ab = (h_a - h_b)^2, so the lambda term drops.
__global__ void vertex_term_kernel(int n, int k, int kp, const double* __restrict__ H, const double* __restrict__ lam,
                                   const double* __restrict__ gbar, int normalized, double* A, double* Hp) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  double s = 0.0;
  for (int i = 0; i < k; ++i) {
    const double hv = H[(size_t)v * k + i];
    s = fma(gbar[i] * (1.0 - (normalized ? lam[i] : 0.0)), hv * hv, s);
    Hp[(size_t)v * kp + i] = hv;
  }
  for (int i = k; i < kp; ++i) Hp[(size_t)v * kp + i] = 0.0;
  A[v] = s;
}

// w (-2 ln w): the bandwidth term's per-entry factor (dw/ds = w (-2 ln w) / s, the 1/s applied once
// to the sum on the host).  FP32 weights in FP32 (relative error about 1e-7 per entry), FP64 in FP64.
template <typename MT>
__device__ __forceinline__ double bandwidth_factor(MT w);
template <>
__device__ __forceinline__ double bandwidth_factor<double>(double w) { return -2.0 * w * log(w); }
template <>
__device__ __forceinline__ double bandwidth_factor<float>(float w) { return (double)(-2.f * w * logf(w)); }
template <>
__device__ __forceinline__ double bandwidth_factor<__nv_bfloat16>(__nv_bfloat16 w) {
  const float x = __bfloat162float(w);
  return (double)(-2.f * x * logf(x));
}

// Warp per row a: every lane holds q_a = gbar .* h_a (KP doubles, from the
// padded copy), and each lane takes one stored entry (a, b) at a time: the
// KP / 2 loads of row b are issued together, then one dot product.
// grad[e] = (A_a + A_b - 2 q_a . h_b) / 2.  KP = 0: any padded width kp.
template <typename MT, int KP>
__global__ void __launch_bounds__(256) sddmm_kernel(int n, const int32_t* __restrict__ row_ptr,
                                                    const int32_t* __restrict__ col, const MT* __restrict__ val,
                                                    int k, int kp_rt, const double* __restrict__ Hp,
                                                    const double* __restrict__ gbar, const double* __restrict__ A,
                                                    double* grad, double bandwidth, double* partial,
                                                    const double* __restrict__ Qp) {
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int kp = KP > 0 ? KP : kp_rt;
  double gs = 0.0;
  for (int a = blockIdx.x * nw + warp; a < n; a += gridDim.x * nw) {
    const int e0 = __ldg(row_ptr + a), e1 = __ldg(row_ptr + a + 1);
    const double Aa = A[a];
    const double* ha = Hp + (size_t)a * kp;
    if constexpr (KP > 0) {
      double q[KP];
      if (Qp) {  // precomputed left rows (the eigenvector-level backward)
#pragma unroll
        for (int i = 0; i < KP; i += 2) {
          const double2 x = __ldg(reinterpret_cast<const double2*>(Qp + (size_t)a * KP + i));
          q[i] = x.x;
          q[i + 1] = x.y;
        }
      } else {
#pragma unroll
        for (int i = 0; i < KP; i += 2) {
          const double2 x = __ldg(reinterpret_cast<const double2*>(ha + i));  // padding columns are zero
          q[i] = i < k ? x.x * gbar[i] : 0.0;                                   // gbar has k entries
          q[i + 1] = i + 1 < k ? x.y * gbar[i + 1] : 0.0;
        }
      }
      for (int e = e0 + lane; e < e1; e += 32) {
        const int b = __ldg(col + e);
        const double2* hb = reinterpret_cast<const double2*>(Hp + (size_t)b * KP);
        double2 y[KP / 2];
#pragma unroll
        for (int i = 0; i < KP / 2; ++i) y[i] = __ldg(hb + i);
        double dot = 0.0;
#pragma unroll
        for (int i = 0; i < KP / 2; ++i) {
          dot = fma(q[2 * i], y[i].x, dot);
          dot = fma(q[2 * i + 1], y[i].y, dot);
        }
        const double g = 0.5 * (Aa + __ldg(A + b) - 2.0 * dot);
        grad[e] = g;
        if (bandwidth > 0.0) gs = fma(g, bandwidth_factor<MT>(val[e]), gs);
      }
    } else {
      for (int e = e0 + lane; e < e1; e += 32) {
        const int b = __ldg(col + e);
        const double* hb = Hp + (size_t)b * kp;
        double dot = 0.0;
        if (Qp)
          for (int i = 0; i < kp; ++i) dot = fma(Qp[(size_t)a * kp + i], hb[i], dot);
        else
          for (int i = 0; i < k; ++i) dot = fma(gbar[i] * ha[i], hb[i], dot);
        const double g = 0.5 * (Aa + __ldg(A + b) - 2.0 * dot);
        grad[e] = g;
        if (bandwidth > 0.0) gs = fma(g, bandwidth_factor<MT>(val[e]), gs);
      }
    }
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

template <typename MT>
static void sddmm_launch(int nblocks, int n, const int32_t* row_ptr, const int32_t* col, const void* val, int k, int kp,
                         const double* Hp, const double* gbar, const double* A, double* grad, double bandwidth,
                         double* partial, const double* Qp, cudaStream_t s) {
  const MT* v = static_cast<const MT*>(val);
  switch (kp) {
    case 4: sddmm_kernel<MT, 4><<<nblocks, 256, 0, s>>>(n, row_ptr, col, v, k, kp, Hp, gbar, A, grad, bandwidth, partial, Qp); break;
    case 8: sddmm_kernel<MT, 8><<<nblocks, 256, 0, s>>>(n, row_ptr, col, v, k, kp, Hp, gbar, A, grad, bandwidth, partial, Qp); break;
    case 12: sddmm_kernel<MT, 12><<<nblocks, 256, 0, s>>>(n, row_ptr, col, v, k, kp, Hp, gbar, A, grad, bandwidth, partial, Qp); break;
    case 16: sddmm_kernel<MT, 16><<<nblocks, 256, 0, s>>>(n, row_ptr, col, v, k, kp, Hp, gbar, A, grad, bandwidth, partial, Qp); break;
    case 20: sddmm_kernel<MT, 20><<<nblocks, 256, 0, s>>>(n, row_ptr, col, v, k, kp, Hp, gbar, A, grad, bandwidth, partial, Qp); break;
    case 24: sddmm_kernel<MT, 24><<<nblocks, 256, 0, s>>>(n, row_ptr, col, v, k, kp, Hp, gbar, A, grad, bandwidth, partial, Qp); break;
    default: sddmm_kernel<MT, 0><<<nblocks, 256, 0, s>>>(n, row_ptr, col, v, k, kp, Hp, gbar, A, grad, bandwidth, partial, Qp);
  }
}

int backward_padded_width(int k) { return (k + 3) / 4 * 4; }

void launch_backward(int n, const int32_t* row_ptr, const int32_t* col, const void* val, int val_dtype, int k,
                     const double* H, const double* lam, const double* gbar, double* grad, double bandwidth,
                     double* partial, int nblocks, double* A, double* Hp, int normalized, cudaStream_t s) {
  const int kp = backward_padded_width(k);
  vertex_term_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, k, kp, H, lam, gbar, normalized, A, Hp);
  switch (val_dtype) {
    case SFAIRSC_F64:
      sddmm_launch<double>(nblocks, n, row_ptr, col, val, k, kp, Hp, gbar, A, grad, bandwidth, partial, nullptr, s);
      break;
    case SFAIRSC_F32:
      sddmm_launch<float>(nblocks, n, row_ptr, col, val, k, kp, Hp, gbar, A, grad, bandwidth, partial, nullptr, s);
      break;
    default:
      sddmm_launch<__nv_bfloat16>(nblocks, n, row_ptr, col, val, k, kp, Hp, gbar, A, grad, bandwidth, partial, nullptr, s);
  }
  check_cuda(cudaGetLastError(), "backward launch");
}

// The SDDMM over W's pattern with precomputed left rows Qp and gathered rows Gp (n x kp each) and
// vertex terms A: grad[e] = (A_a + A_b - 2 Qp_a . Gp_b) / 2, plus the bandwidth partial sums.
void launch_sddmm_rows(int n, const int32_t* row_ptr, const int32_t* col, const void* val, int val_dtype, int kp,
                       const double* Qp, const double* Gp, const double* A, double* grad, double bandwidth,
                       double* partial, int nblocks, cudaStream_t s) {
  switch (val_dtype) {
    case SFAIRSC_F64:
      sddmm_launch<double>(nblocks, n, row_ptr, col, val, kp, kp, Gp, nullptr, A, grad, bandwidth, partial, Qp, s);
      break;
    case SFAIRSC_F32:
      sddmm_launch<float>(nblocks, n, row_ptr, col, val, kp, kp, Gp, nullptr, A, grad, bandwidth, partial, Qp, s);
      break;
    default:
      sddmm_launch<__nv_bfloat16>(nblocks, n, row_ptr, col, val, kp, kp, Gp, nullptr, A, grad, bandwidth, partial, Qp,
                                  s);
  }
  check_cuda(cudaGetLastError(), "sddmm launch");
}

}  // namespace sfairsc
