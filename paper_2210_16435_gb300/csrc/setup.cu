// Setup pass of Algorithm 3 (steps 1-2): input validation, degrees
// d_i = sum_j w_ij (Sec. 2.1), D^{-1/2}, group sizes |V_s| and
// S_s = sum_{i in V_s} 1/d_i (from which C^T C follows in closed form),
// sigma = ||L_n||_1 (App. C), and the nnz-balanced row partition that the
// cooperative kernels share.
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace sfairsc {

enum : unsigned {
  kBadRowPtr = 1u << 0,
  kBadCol = 1u << 1,
  kSelfLoop = 1u << 2,
  kNegWeight = 1u << 3,
  kNonFinite = 1u << 4,
  kBadLabel = 1u << 5,
  kAsymmetric = 1u << 6,
  kUnsorted = 1u << 7,
  kIsolated = 1u << 8,
};

template <typename MT>
__global__ void validate_kernel(int n, int64_t nnz, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                const MT* __restrict__ val, const int32_t* __restrict__ labels, int h, int symm,
                                unsigned* flags) {
  unsigned f = 0;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r == 0) {
    if (row_ptr[0] != 0 || (int64_t)row_ptr[n] != nnz) f |= kBadRowPtr;
  }
  if (r < n) {
    const int64_t e0 = row_ptr[r], e1 = row_ptr[r + 1];
    if (e1 < e0 || e0 < 0 || e1 > nnz) f |= kBadRowPtr;
    const int64_t lo = max((int64_t)0, e0), hi = min(nnz, e1);
    int prev = -1;
    for (int64_t e = lo; e < hi; ++e) {
      const int c = col[e];
      const double w = to_f64(val[e]);
      if (c < 0 || c >= n) {
        f |= kBadCol;
        continue;
      }
      if (c == r) f |= kSelfLoop;
      if (!(w == w) || w - w != 0.0) f |= kNonFinite;
      else if (w < 0.0) f |= kNegWeight;
      if (symm) {
        if (c <= prev) f |= kUnsorted;
        prev = c;
        // binary search r in row c
        int64_t a = max((int64_t)0, (int64_t)row_ptr[c]), b = min(nnz, (int64_t)row_ptr[c + 1]);
        bool found = false;
        while (a < b) {
          const int64_t m = (a + b) >> 1;
          const int cm = col[m];
          if (cm == r) {
            found = to_f64(val[m]) == w;
            break;
          }
          if (cm < r) a = m + 1;
          else b = m;
        }
        if (!found) f |= kAsymmetric;
      }
    }
    const int g = labels[r];
    if (g < 0 || g >= h) f |= kBadLabel;
  }
  if (f) atomicOr(flags, f);
}

void launch_validate(int n, int64_t nnz, const int32_t* row_ptr, const int32_t* col, const void* val, int val_dtype,
                     const int32_t* labels, int h, int check_symmetry, unsigned* flags, cudaStream_t s) {
  const int T = 256;
  const int G = (n + T - 1) / T;
  switch (val_dtype) {
    case SFAIRSC_F64:
      validate_kernel<double><<<G, T, 0, s>>>(n, nnz, row_ptr, col, (const double*)val, labels, h, check_symmetry, flags);
      break;
    case SFAIRSC_F32:
      validate_kernel<float><<<G, T, 0, s>>>(n, nnz, row_ptr, col, (const float*)val, labels, h, check_symmetry, flags);
      break;
    default:
      validate_kernel<__nv_bfloat16><<<G, T, 0, s>>>(n, nnz, row_ptr, col, (const __nv_bfloat16*)val, labels, h,
                                                    check_symmetry, flags);
  }
  check_cuda(cudaGetLastError(), "validate launch");
}

// One thread per row: degree in FP64, labels to uint8, D^{-1/2}; per-block
// group sums of (1, 1/d_i) (or (1, 1) unnormalized) in fixed lane/warp order.
template <typename MT>
__global__ void degree_kernel(int n, const int32_t* __restrict__ row_ptr, const MT* __restrict__ val,
                              const int32_t* __restrict__ labels_in, uint8_t* lab, double* deg, double* dinv64,
                              float* dinv32, double* blocksums, int h, int normalized, unsigned* flags) {
  __shared__ double red[32 * 2 * kMaxGroups];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = r < n;
  double x[2] = {0.0, 0.0};
  int g = 0;
  if (valid) {
    double d = 0.0;
    for (int e = row_ptr[r]; e < row_ptr[r + 1]; ++e) d += to_f64(val[e]);
    g = labels_in[r];
    lab[r] = (uint8_t)g;
    deg[r] = d;
    const double di = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
    dinv64[r] = di;
    dinv32[r] = (float)di;
    if (!(d > 0.0)) atomicOr(flags, kIsolated);
    x[0] = 1.0;
    x[1] = normalized ? (d > 0.0 ? 1.0 / d : 0.0) : 1.0;
  }
  double acc[2] = {0.0, 0.0};
  for (int s = 0; s < h; ++s) {
    const bool mine = valid && g == s;
    if (__ballot_sync(0xffffffffu, mine) == 0u) continue;
    for (int v = 0; v < 2; ++v) {
      const double t = warp_allsum(mine ? x[v] : 0.0);
      if (lane == s) acc[v] += t;
    }
  }
  if (lane < h) {
    red[warp * 2 * h + lane * 2 + 0] = acc[0];
    red[warp * 2 * h + lane * 2 + 1] = acc[1];
  }
  __syncthreads();
  for (int p = threadIdx.x; p < 2 * h; p += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < nwarps; ++w) s += red[w * 2 * h + p];
    blocksums[(size_t)blockIdx.x * 2 * h + p] = s;
  }
}

int degrees_blocks(int n) { return (n + 255) / 256; }

void launch_degrees(int n, const int32_t* row_ptr, const void* val, int val_dtype, const int32_t* labels_in,
                    uint8_t* lab, double* deg, double* dinv64, float* dinv32, double* blocksums, int nblocks, int h,
                    int normalized, unsigned* flags, cudaStream_t s) {
  const int T = 256;
  switch (val_dtype) {
    case SFAIRSC_F64:
      degree_kernel<double><<<nblocks, T, 0, s>>>(n, row_ptr, (const double*)val, labels_in, lab, deg, dinv64, dinv32,
                                                  blocksums, h, normalized, flags);
      break;
    case SFAIRSC_F32:
      degree_kernel<float><<<nblocks, T, 0, s>>>(n, row_ptr, (const float*)val, labels_in, lab, deg, dinv64, dinv32,
                                                 blocksums, h, normalized, flags);
      break;
    default:
      degree_kernel<__nv_bfloat16><<<nblocks, T, 0, s>>>(n, row_ptr, (const __nv_bfloat16*)val, labels_in, lab, deg,
                                                         dinv64, dinv32, blocksums, h, normalized, flags);
  }
  check_cuda(cudaGetLastError(), "degree launch");
}

// ||L_n||_1 = max_j (1 + d_j^{-1/2} sum_i w_ij d_i^{-1/2}) since w_jj = 0 and W = W^T;
// ||D - W||_1 = max_j 2 d_j for the unnormalized extension.  Per-block maxima.
template <typename MT>
__global__ void sigma_kernel(int n, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                             const MT* __restrict__ val, const double* __restrict__ dinv, const double* __restrict__ deg,
                             int normalized, double* blockmax) {
  __shared__ double red[32];
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  double m = 0.0;
  if (r < n) {
    if (normalized) {
      double s = 0.0;
      for (int e = row_ptr[r]; e < row_ptr[r + 1]; ++e) s += to_f64(val[e]) * dinv[col[e]];
      m = 1.0 + dinv[r] * s;
    } else {
      m = 2.0 * deg[r];
    }
  }
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = red[w] > b ? red[w] : b;
    blockmax[blockIdx.x] = b;
  }
}

void launch_sigma_rows(int n, const int32_t* row_ptr, const int32_t* col, const void* val, int val_dtype,
                       const double* dinv64, const double* deg, int normalized, double* blockmax, int nblocks,
                       cudaStream_t s) {
  const int T = 256;
  switch (val_dtype) {
    case SFAIRSC_F64:
      sigma_kernel<double><<<nblocks, T, 0, s>>>(n, row_ptr, col, (const double*)val, dinv64, deg, normalized, blockmax);
      break;
    case SFAIRSC_F32:
      sigma_kernel<float><<<nblocks, T, 0, s>>>(n, row_ptr, col, (const float*)val, dinv64, deg, normalized, blockmax);
      break;
    default:
      sigma_kernel<__nv_bfloat16><<<nblocks, T, 0, s>>>(n, row_ptr, col, (const __nv_bfloat16*)val, dinv64, deg,
                                                        normalized, blockmax);
  }
  check_cuda(cudaGetLastError(), "sigma launch");
}

// cta_rows[t] = first row r with row_ptr[r] + wgt * r >= t * total / grid.
__global__ void row_partition_kernel(int n, const int32_t* __restrict__ row_ptr, int grid, int wgt, int32_t* cta_rows) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t > grid) return;
  const long long total = (long long)row_ptr[n] + (long long)wgt * n;
  const long long target = total * t / grid;
  int lo = 0, hi = n;
  while (lo < hi) {
    const int m = (lo + hi) >> 1;
    if ((long long)row_ptr[m] + (long long)wgt * m >= target) hi = m;
    else lo = m + 1;
  }
  cta_rows[t] = (t == 0) ? 0 : (t == grid ? n : lo);
}

void launch_row_partition(int n, const int32_t* row_ptr, int grid, int row_weight, int32_t* cta_rows, cudaStream_t s) {
  row_partition_kernel<<<(grid + 1 + 255) / 256, 256, 0, s>>>(n, row_ptr, grid, row_weight, cta_rows);
  check_cuda(cudaGetLastError(), "row partition launch");
}

}  // namespace sfairsc

namespace sfairsc {

// C^T C for a dense constraint matrix (C = D^{-1/2} F, or F for the unnormalized extension):
// partial[b][s * p + t] = sum over block b's rows of F_rs F_rt / d_r.  Rows are staged 64 at a
// time (scaled by d_r^{-1/2}); thread q owns the entries q, q + 256, ... (p * p <= 961).
__global__ void dense_ctc_kernel(int n, int p, const double* __restrict__ F, const double* __restrict__ deg,
                                 int normalized, double* partial) {
  extern __shared__ double tile[];  // 64 x p
  const int npair = p * p;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int t0 = blockIdx.x * 64; t0 < n; t0 += gridDim.x * 64) {
    const int rows = min(64, n - t0);
    __syncthreads();
    for (int e = threadIdx.x; e < 64 * p; e += blockDim.x) {
      const int rr = e / p, s = e % p;
      double v = 0.0;
      if (rr < rows) {
        const int r = t0 + rr;
        v = F[(size_t)r * p + s];
        if (normalized) v /= sqrt(deg[r]);
      }
      tile[e] = v;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int q = threadIdx.x + j * blockDim.x;
      if (q < npair) {
        const int s = q / p, t = q % p;
        double sacc = 0.0;
        for (int rr = 0; rr < rows; ++rr) sacc = fma(tile[rr * p + s], tile[rr * p + t], sacc);
        acc[j] += sacc;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int q = threadIdx.x + j * blockDim.x;
    if (q < npair) partial[(size_t)blockIdx.x * npair + q] = acc[j];
  }
}

void launch_dense_ctc(int n, int p, const double* F, const double* deg, int normalized, double* partial, int nblocks,
                      cudaStream_t s) {
  dense_ctc_kernel<<<nblocks, 256, sizeof(double) * 64 * p, s>>>(n, p, F, deg, normalized, partial);
  check_cuda(cudaGetLastError(), "dense C^T C launch");
}

// partial[b][s * k + i] = sum over block b's rows of F_rs H_ri (F^T H, the fairness residual of a
// dense constraint matrix); thread q owns the entries q, q + 256, ...
__global__ void dense_fth_kernel(int n, int p, int k, const double* __restrict__ F, const double* __restrict__ H,
                                 double* partial) {
  const int per = (n + gridDim.x - 1) / gridDim.x;
  const int r0 = blockIdx.x * per, r1 = min(n, r0 + per);
  for (int q = threadIdx.x; q < p * k; q += blockDim.x) {
    const int s = q / k, i = q % k;
    double acc = 0.0;
    for (int r = r0; r < r1; ++r) acc = fma(F[(size_t)r * p + s], H[(size_t)r * k + i], acc);
    partial[(size_t)blockIdx.x * p * k + q] = acc;
  }
}

void launch_dense_fth(int n, int p, int k, const double* F, const double* H, double* partial, int nblocks,
                      cudaStream_t s) {
  dense_fth_kernel<<<nblocks, 256, 0, s>>>(n, p, k, F, H, partial);
  check_cuda(cudaGetLastError(), "dense F^T H launch");
}

__global__ void f64_to_f32_rows_kernel(int64_t count, const double* in, float* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

void launch_f64_to_f32(int64_t count, const double* in, float* out, cudaStream_t s) {
  f64_to_f32_rows_kernel<<<1024, 256, 0, s>>>(count, in, out);
  check_cuda(cudaGetLastError(), "conversion launch");
}


// The small solve of the operator applied to each unit vector: column t of the map is the
// coefficient vector of tot = e_t (forward and backward substitution with the factor L of C^T C,
// then, for labels, the shift by z . y that expresses C a through the group coefficients).
void fill_group_map(double* P, int h, bool dense) {
  const int p = h - 1;
  std::vector<double> y((size_t)std::max(p, 1));
  for (int t = 0; t < h; ++t) {
    const double sum = dense ? 0.0 : 1.0;  // sum of the unit vector's entries
    for (int s = 0; s < p; ++s) {
      double r = (s == t ? 1.0 : 0.0) - (dense ? 0.0 : P[kPZ + s] * sum);
      for (int q = 0; q < s; ++q) r -= P[kPL + s * kLStride + q] * y[q];
      y[s] = r * P[kPLinv + s];
    }
    for (int s = p - 1; s >= 0; --s) {
      double r = y[s];
      for (int q = s + 1; q < p; ++q) r -= P[kPL + q * kLStride + s] * y[q];
      y[s] = r * P[kPLinv + s];
    }
    double za = 0.0;
    if (!dense)
      for (int s = 0; s < p; ++s) za += P[kPZ + s] * y[s];
    for (int s = 0; s < p; ++s) P[kPG + s * h + t] = y[s] - za;
    P[kPG + p * h + t] = -za;
  }
}


template <typename MT>
__global__ void kmat_kernel(int n, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                            const MT* __restrict__ val, const uint8_t* __restrict__ lab, const double* __restrict__ Fd,
                            int p, int kpad, const double* __restrict__ dinv, const double* __restrict__ deg,
                            int normalized, double* K64, float* K32) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  double M[kMaxGroups];
  for (int t = 0; t < kpad; ++t) M[t] = 0.0;
  for (int e = row_ptr[c]; e < row_ptr[c + 1]; ++e) {
    const int r = col[e];
    const double w = to_f64(val[e]) * (normalized ? dinv[r] * dinv[r] : 1.0);
    if (Fd) {
      for (int t = 0; t < p; ++t) M[t] += w * Fd[(size_t)r * p + t];
    } else {
      M[lab[r]] += w;
    }
  }
  const size_t pn = (size_t)n * 4;
  for (int t = 0; t < kpad; ++t) {
    const double f = Fd ? (t < p ? Fd[(size_t)c * p + t] : 0.0) : (t == (int)lab[c] ? 1.0 : 0.0);
    const double kv = normalized ? dinv[c] * (f - M[t]) : deg[c] * f - M[t];
    const size_t at = (size_t)(t >> 2) * pn + (size_t)c * 4 + (t & 3);
    if (K64) K64[at] = kv;
    if (K32) K32[at] = (float)kv;
  }
}

void launch_kmat(int n, const int32_t* row_ptr, const int32_t* col, const void* val, int val_dtype, const uint8_t* lab,
                 const double* Fd, int p, int h, const double* dinv64, const double* deg, int normalized,
                 double* K64, float* K32, cudaStream_t s) {
  const int kpad = (h + 3) & ~3;
  if (kpad > kMaxGroups) fail(SFAIRSC_ERR_UNSUPPORTED, "more than 32 constraint columns");
  const int grid = (n + 255) / 256;
  switch (val_dtype) {
    case SFAIRSC_F64:
      kmat_kernel<double><<<grid, 256, 0, s>>>(n, row_ptr, col, static_cast<const double*>(val), lab, Fd, p, kpad,
                                                dinv64, deg, normalized, K64, K32);
      break;
    case SFAIRSC_F32:
      kmat_kernel<float><<<grid, 256, 0, s>>>(n, row_ptr, col, static_cast<const float*>(val), lab, Fd, p, kpad,
                                               dinv64, deg, normalized, K64, K32);
      break;
    default:
      kmat_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(n, row_ptr, col, static_cast<const __nv_bfloat16*>(val), lab,
                                                       Fd, p, kpad, dinv64, deg, normalized, K64, K32);
  }
  check_cuda(cudaGetLastError(), "kmat launch");
}

}  // namespace sfairsc
