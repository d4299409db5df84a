// Krylov-subspace kernels of the restarted block Lanczos (Algorithm 3 step 3):
// CGS2 orthogonalisation of a new block against the basis, Cholesky-QR of the
// block, thick restart V <- V Y, and the final FP64 checks / embedding.
//
// The basis V is stored as ldv/4 panels of 4 columns, each an n x 4
// row-major array (panel p = columns 4p..4p+3), so a run of rows of one
// panel is contiguous.
#include "common.cuh"
#include "internal.h"

namespace sfairsc {

// ---------------------------------------------------------------- thick restart / Ritz vectors
// OUT[r, 0:K] = V[r, 0:m] Y[:, 0:K] for a 64-row tile: the tile of V (read
// panel by panel, 1 KB contiguous per panel) is held transposed in shared
// memory (stride 68), Y (row-major, so each CTA's copy is a coalesced read) in
// 64-column chunks, and each of the 256 threads accumulates a 4 x 4 block
// (rows 4*tr.., columns 4*tc..) from two 16-byte shared loads per inner step.
// The restart stores each row's 4 columns as one 16-byte write into their
// panel; the FP64 Ritz output (column-major) goes through a shared-memory
// tile so that each column is written as one 64-row run.
constexpr int kTR = 64;       // rows per CTA
constexpr int kTS = kTR + 4;  // transposed stride (keeps 16-byte alignment)

template <typename VT>
__device__ __forceinline__ void lds4(const VT* p, VT (&x)[4]) {
  if constexpr (sizeof(VT) == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
  } else {
    const double2 a = reinterpret_cast<const double2*>(p)[0];
    const double2 b = reinterpret_cast<const double2*>(p)[1];
    x[0] = a.x; x[1] = a.y; x[2] = b.x; x[3] = b.y;
  }
}

// mode 0: in place into V[:, 0:K] (+ carry V[:, m:m+B] to V[:, K:K+B] and Q);
// mode 1: into X (column-major n x K, FP64).
template <typename VT, int MODE>
__global__ void __launch_bounds__(256) tile_gemm_kernel(int n, VT* V, int64_t ldv, int m, int K, int B,
                                                        const VT* __restrict__ Y, VT* Q, double* X,
                                                        const double* __restrict__ E) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int width = m + B;
  VT* Vt = reinterpret_cast<VT*>(sm);  // width x kTS (transposed tile)
  VT* Ys = Vt + (size_t)width * kTS;   // m x 64
  const int t = threadIdx.x, tr = t >> 4, tc = t & 15;
  const int rbase = blockIdx.x * kTR;
  const int rows = min(kTR, n - rbase);
  const size_t pn = (size_t)n * 4;
  const int width4 = (width + 3) & ~3;
  // the tile: unit u = (panel u / kTR, row u % kTR), one row of a panel; a
  // thread issues all its loads before its shared-memory stores
  {
    constexpr int UN = 8;
    const int total = (width4 / 4) * kTR;
    for (int u0 = t; u0 < total; u0 += 256 * UN) {
      VT v[UN][4];
#pragma unroll
      for (int q = 0; q < UN; ++q) {
        const int u = u0 + q * 256, p = u / kTR, rr = u % kTR;
        if (u < total && rr < rows) lds4(V + p * pn + (size_t)(rbase + rr) * 4, v[q]);
        else v[q][0] = v[q][1] = v[q][2] = v[q][3] = VT(0);
      }
#pragma unroll
      for (int q = 0; q < UN; ++q) {
        const int u = u0 + q * 256, p = u / kTR, rr = u % kTR;
        if (u < total)
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (4 * p + e < width) Vt[(size_t)(4 * p + e) * kTS + rr] = v[q][e];
      }
    }
  }
  for (int k0 = 0; k0 < K; k0 += 64) {
    const int kc = min(64, K - k0);
    __syncthreads();
    if (sizeof(VT) == 4 && (K & 3) == 0) {
      // 16-byte pieces (c, 4 kk4): the whole chunk in one round of loads
      constexpr int UN = 8;
      const int nq = m * 16;
      for (int i0 = t; i0 < nq; i0 += 256 * UN) {
        float4 y[UN];
#pragma unroll
        for (int q = 0; q < UN; ++q) {
          const int i = i0 + q * 256, c = i >> 4, kk = (i & 15) * 4;
          y[q] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (i < nq && kk < kc) y[q] = *reinterpret_cast<const float4*>(Y + (size_t)c * K + k0 + kk);  // kc % 4 == 0
        }
#pragma unroll
        for (int q = 0; q < UN; ++q) {
          const int i = i0 + q * 256;
          if (i < nq) *reinterpret_cast<float4*>(Ys + (size_t)(i >> 4) * 64 + (i & 15) * 4) = y[q];
        }
      }
    } else {
      constexpr int UN = 8;
      for (int i0 = t; i0 < m * 64; i0 += 256 * UN) {
        VT y[UN];
#pragma unroll
        for (int q = 0; q < UN; ++q) {
          const int i = i0 + q * 256, c = i >> 6, kk = i & 63;
          y[q] = i < m * 64 && kk < kc ? Y[(size_t)c * K + k0 + kk] : VT(0);
        }
#pragma unroll
        for (int q = 0; q < UN; ++q)
          if (i0 + q * 256 < m * 64) Ys[i0 + q * 256] = y[q];
      }
    }
    __syncthreads();
    VT acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = VT(0);
    for (int c = 0; c < m; ++c) {
      VT va[4], yb[4];
      lds4(Vt + (size_t)c * kTS + 4 * tr, va);
      lds4(Ys + (size_t)c * 64 + 4 * tc, yb);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(va[i], yb[j], acc[i][j]);
    }
    if (MODE == 0) {
      // columns k0 + 4 tc .. + 3 form panel (k0 + 4 tc) / 4 (k0 is a multiple of 64)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int rr = 4 * tr + i;
        if (rr >= rows) continue;
        const int r = rbase + rr;
        VT* dst = V + ((k0 + 4 * tc) >> 2) * pn + (size_t)r * 4;
        if (4 * tc + 4 <= kc) {
          if constexpr (sizeof(VT) == 4) {
            *reinterpret_cast<float4*>(dst) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
          } else {
            reinterpret_cast<double2*>(dst)[0] = make_double2(acc[i][0], acc[i][1]);
            reinterpret_cast<double2*>(dst)[1] = make_double2(acc[i][2], acc[i][3]);
          }
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (4 * tc + j < kc) dst[j] = acc[i][j];
        }
      }
    } else {
      // through shared memory (the Y chunk's space, after every thread is done with it)
      double* Xs = reinterpret_cast<double*>(Ys);  // 64 columns x (kTR + 1)
      __syncthreads();
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) Xs[(size_t)(4 * tc + j) * (kTR + 1) + 4 * tr + i] = (double)acc[i][j];
      __syncthreads();
      for (int e = t; e < kc * kTR; e += blockDim.x) {
        const int col = e / kTR, rr = e % kTR;
        if (rr < rows) X[(size_t)(rbase + rr) + (size_t)(k0 + col) * n] = Xs[(size_t)col * (kTR + 1) + rr];
      }
    }
  }
  if (MODE == 0) {
    __syncthreads();
    VT* Es = Ys;  // the Y chunk's space is free now: E (m x B) in the basis precision
    if (E)
      for (int i = t; i < m * B; i += blockDim.x) Es[i] = (VT)E[i];
    __syncthreads();
    for (int i = t; i < rows * B; i += blockDim.x) {
      const int rr = i / B, v = i % B;
      VT x = Vt[(size_t)(m + v) * kTS + rr];
      if (E) {  // the carried block's pending second projection: x -= V[r, 0:m] E[:, v]
        VT d = VT(0);
        for (int c = 0; c < m; ++c) d = fma(Vt[(size_t)c * kTS + rr], Es[c * B + v], d);
        x -= d;
      }
      V[((K + v) >> 2) * pn + (size_t)(rbase + rr) * 4 + ((K + v) & 3)] = x;
      Q[(size_t)(rbase + rr) * 4 + v] = x;
    }
  }
}

template <typename VT, int MODE>
static void tile_gemm_launch(int n, VT* V, int64_t ldv, int m, int K, int B, const VT* Y, VT* Q, double* X,
                             const double* E, cudaStream_t s) {
  size_t smem = sizeof(VT) * ((size_t)(m + B) * kTS + (size_t)m * 64);
  if (MODE == 1)  // the Y chunk's space also holds the 64 x (kTR + 1) FP64 output tile
    smem = std::max(smem, sizeof(VT) * (size_t)(m + B) * kTS + sizeof(double) * 64 * (kTR + 1));
  if (smem > 227 * 1024) fail(SFAIRSC_ERR_UNSUPPORTED, "Krylov basis too wide for the restart tile in this precision");
  auto kern = tile_gemm_kernel<VT, MODE>;
  check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "tile gemm smem");
  kern<<<(n + kTR - 1) / kTR, 256, smem, s>>>(n, V, ldv, m, K, B, Y, Q, X, E);
  check_cuda(cudaGetLastError(), "tile gemm launch");
}

void launch_restart(VecType vt, int n, void* V, int64_t ldv, int m, int K, int B, const void* Y, void* Q,
                    const double* E, cudaStream_t s) {
  if (vt == VecType::F64)
    tile_gemm_launch<double, 0>(n, (double*)V, ldv, m, K, B, (const double*)Y, (double*)Q, nullptr, E, s);
  else tile_gemm_launch<float, 0>(n, (float*)V, ldv, m, K, B, (const float*)Y, (float*)Q, nullptr, E, s);
}

void launch_ritz(VecType vt, int n, const void* V, int64_t ldv, int m, int k, const void* Y, double* X64,
                 cudaStream_t s) {
  if (vt == VecType::F64)
    tile_gemm_launch<double, 1>(n, (double*)V, ldv, m, k, 0, (const double*)Y, nullptr, X64, nullptr, s);
  else tile_gemm_launch<float, 1>(n, (float*)V, ldv, m, k, 0, (const float*)Y, nullptr, X64, nullptr, s);
}

__global__ void column_resid_kernel(int n, int k, const double* __restrict__ X, const double* __restrict__ AX,
                                    const double* __restrict__ lam, double* partial) {
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int per = (n + gridDim.x - 1) / gridDim.x;
  const int lo = blockIdx.x * per, hi = min(n, lo + per);
  for (int c = 0; c < k; ++c) {
    double s = 0.0;
    const double l = lam[c];
    for (int r = lo + threadIdx.x; r < hi; r += blockDim.x) {
      const double t = AX[(size_t)c * n + r] - l * X[(size_t)c * n + r];
      s = fma(t, t, s);
    }
    s = warp_allsum(s);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < nw; ++w) t += red[w];
      partial[(size_t)blockIdx.x * k + c] = t;
    }
    __syncthreads();
  }
}

void launch_column_resid(int n, int k, const double* X, const double* AX, const double* lam, double* partial,
                         int nblocks, cudaStream_t s) {
  column_resid_kernel<<<nblocks, 256, 0, s>>>(n, k, X, AX, lam, partial);
  check_cuda(cudaGetLastError(), "column resid launch");
}

// ---------------------------------------------------------------- start block
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <typename VT>
__global__ void random_block_kernel(int n, VT* V, int64_t ldv, int B, uint64_t seed) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  for (int v = 0; v < B; ++v) {
    const uint64_t z = mix64(seed + ((uint64_t)r * 4 + v + 1) * 0x9E3779B97F4A7C15ull);
    V[(size_t)r * ldv + v] = (VT)((double)(z >> 11) * 0x1.0p-53 - 0.5);
  }
}

void launch_random_block(VecType vt, int n, void* V, int64_t ldv, int B, uint64_t seed, cudaStream_t s) {
  const int grid = (n + 255) / 256;
  if (vt == VecType::F64) random_block_kernel<double><<<grid, 256, 0, s>>>(n, (double*)V, ldv, B, seed);
  else random_block_kernel<float><<<grid, 256, 0, s>>>(n, (float*)V, ldv, B, seed);
  check_cuda(cudaGetLastError(), "random block launch");
}

template <typename VT>
__global__ void to_f64_kernel(int n, const VT* V, int64_t ldv, int k, double* X) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  for (int c = 0; c < k; ++c) X[(size_t)r + (size_t)c * n] = (double)V[(size_t)(c >> 2) * n * 4 + (size_t)r * 4 + (c & 3)];
}

void launch_to_f64(VecType vt, int n, const void* V, int64_t ldv, int k, double* X, cudaStream_t s) {
  const int grid = (n + 255) / 256;
  if (vt == VecType::F64) to_f64_kernel<double><<<grid, 256, 0, s>>>(n, (const double*)V, ldv, k, X);
  else to_f64_kernel<float><<<grid, 256, 0, s>>>(n, (const float*)V, ldv, k, X);
  check_cuda(cudaGetLastError(), "to_f64 launch");
}

// ---------------------------------------------------------------- FP64 final checks
// Per block and column c: (<x, Ax>, <x, x>, <Ax, Ax>) in FP64, fixed reduction order.
__global__ void column_stats_kernel(int n, int k, const double* __restrict__ X, const double* __restrict__ AX,
                                    double* partial) {
  __shared__ double red[3 * 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int per = (n + gridDim.x - 1) / gridDim.x;
  const int lo = blockIdx.x * per, hi = min(n, lo + per);
  for (int c = 0; c < k; ++c) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    const double* x = X + (size_t)c * n;
    const double* y = AX + (size_t)c * n;
    for (int r = lo + threadIdx.x; r < hi; r += blockDim.x) {
      const double xv = x[r], yv = y[r];
      s0 = fma(xv, yv, s0);
      s1 = fma(xv, xv, s1);
      s2 = fma(yv, yv, s2);
    }
    s0 = warp_allsum(s0);
    s1 = warp_allsum(s1);
    s2 = warp_allsum(s2);
    if (lane == 0) {
      red[warp * 3 + 0] = s0;
      red[warp * 3 + 1] = s1;
      red[warp * 3 + 2] = s2;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += red[w * 3 + threadIdx.x];
      partial[((size_t)blockIdx.x * k + c) * 3 + threadIdx.x] = s;
    }
    __syncthreads();
  }
}

void launch_column_stats(int n, int k, const double* X, const double* AX, const double* lam, double* partial,
                         int nblocks, double* out, cudaStream_t s) {
  (void)lam;
  (void)out;
  column_stats_kernel<<<nblocks, 256, 0, s>>>(n, k, X, AX, partial);
  check_cuda(cudaGetLastError(), "column stats launch");
}

__global__ void scale_columns_kernel(int n, int k, double* X, const double* __restrict__ scale) {
  const int64_t N = (int64_t)n * k;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    X[i] *= scale[i / n];
}

void launch_scale_columns(int n, int k, double* X, const double* scale, cudaStream_t s) {
  scale_columns_kernel<<<1024, 256, 0, s>>>(n, k, X, scale);
  check_cuda(cudaGetLastError(), "scale columns launch");
}

// ---------------------------------------------------------------- embedding
// colkey[c] = max |x_c| (as ordered bits), colkey[k + c] = lowest row attaining it.
__global__ void colmax_kernel(int n, int k, const double* __restrict__ X, unsigned long long* colkey) {
  const int c = blockIdx.y;
  unsigned long long best = 0;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(X[(size_t)c * n + r]));
    best = b > best ? b : best;
  }
  best = warp_max(best);
  if ((threadIdx.x & 31) == 0) atomicMax(colkey + c, best);
}

__global__ void colargmax_kernel(int n, int k, const double* __restrict__ X, unsigned long long* colkey) {
  const int c = blockIdx.y;
  const unsigned long long best = colkey[c];
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(X[(size_t)c * n + r]));
    if (b == best) atomicMin(colkey + k + c, (unsigned long long)r);
  }
}

// H = sign_c D^{-1/2} X through a shared tile of 32 rows: X is read a column at a time (32
// consecutive doubles per column) and H written a row block at a time (32 k consecutive doubles),
// both coalesced.
constexpr int kEmbRows = 32;
__global__ void __launch_bounds__(256) embed_kernel(int n, int k, const double* __restrict__ X,
                                                    const double* __restrict__ dinv, int normalized,
                                                    const unsigned long long* colkey, double* H) {
  extern __shared__ double tile[];  // kEmbRows x (k + 1), plus k signs
  double* sg = tile + kEmbRows * (k + 1);
  const int r0 = blockIdx.x * kEmbRows;
  const int rows = min(kEmbRows, n - r0);
  for (int c = threadIdx.x; c < k; c += blockDim.x) sg[c] = X[(size_t)c * n + colkey[k + c]] < 0.0 ? -1.0 : 1.0;
  for (int e = threadIdx.x; e < kEmbRows * k; e += blockDim.x) {
    const int c = e / kEmbRows, rr = e % kEmbRows;
    if (rr < rows) tile[rr * (k + 1) + c] = X[(size_t)c * n + r0 + rr];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < rows * k; e += blockDim.x) {
    const int rr = e / k, c = e % k;
    const double sc = normalized ? dinv[r0 + rr] : 1.0;
    H[(size_t)(r0 + rr) * k + c] = sg[c] * sc * tile[rr * (k + 1) + c];
  }
}

__global__ void init_colkey_kernel(int k, unsigned long long* colkey) {
  const int c = threadIdx.x + blockIdx.x * blockDim.x;
  if (c < k) {
    colkey[c] = 0ull;
    colkey[k + c] = ~0ull;
  }
}

void launch_embed(int n, int k, const double* X, const double* dinv64, int normalized, double* H,
                  unsigned long long* colkey, cudaStream_t s) {
  init_colkey_kernel<<<(k + 255) / 256, 256, 0, s>>>(k, colkey);
  dim3 g(min(152 * 2, (n + 255) / 256), k);
  colmax_kernel<<<g, 256, 0, s>>>(n, k, X, colkey);
  colargmax_kernel<<<g, 256, 0, s>>>(n, k, X, colkey);
  const size_t smem = sizeof(double) * ((size_t)kEmbRows * (k + 1) + k);
  if (smem > 48 * 1024)
    check_cuda(cudaFuncSetAttribute(embed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "embed smem");
  embed_kernel<<<(n + kEmbRows - 1) / kEmbRows, 256, smem, s>>>(n, k, X, dinv64, normalized, colkey, H);
  check_cuda(cudaGetLastError(), "embed launch");
}

// ---------------------------------------------------------------- diagnostics
// Per CTA: group sums of the columns of H (h x k, for max |F^T H|) and the
// upper triangle of H^T D H = X^T X (for max |H^T D H - I|), over 64-row
// tiles.  AT = float accumulates each tile in FP32 and carries it in FP64.
template <typename AT>
__global__ void __launch_bounds__(256) diagnostics_kernel(int n, int k, int h, const double* __restrict__ H,
                                                          const double* __restrict__ deg,
                                                          const uint8_t* __restrict__ lab, double* partial) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double* gs = reinterpret_cast<double*>(smraw);       // h * k
  AT* Xs = reinterpret_cast<AT*>(gs + (size_t)h * k);  // 64 x (k + 1)
  const int P = h * k + k * k;
  const int ks = k + 1;
  for (int i = threadIdx.x; i < h * k; i += blockDim.x) gs[i] = 0.0;
  constexpr int MP = 9;  // pairs per thread (k <= 64 -> at most 2080 pairs / 256 threads)
  double tot[MP];
  int pi[MP], pj[MP];
  const int npairs = k * (k + 1) / 2;
  for (int q = 0; q < MP; ++q) {
    tot[q] = 0.0;
    const int p = threadIdx.x + q * blockDim.x;
    int i = 0, rem = p;
    while (i < k && rem >= k - i) {
      rem -= k - i;
      ++i;
    }
    pi[q] = p < npairs ? i : -1;
    pj[q] = p < npairs ? i + rem : -1;
  }
  __syncthreads();
  __shared__ double sqd[64];  // sqrt(d_r) of the tile's rows: one FP64 root per row, not per entry
  __shared__ int labs[64];
  for (int t0 = blockIdx.x * 64; t0 < n; t0 += gridDim.x * 64) {
    const int rows = min(64, n - t0);
    if (threadIdx.x < 64) {
      const int r = t0 + threadIdx.x;
      sqd[threadIdx.x] = (int)threadIdx.x < rows ? sqrt(deg[r]) : 0.0;
      labs[threadIdx.x] = (int)threadIdx.x < rows ? (int)lab[r] : 0;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 64 * k; e += blockDim.x) {
      const int rr = e / k, c = e % k;
      const double v = rr < rows ? H[(size_t)(t0 + rr) * k + c] * sqd[rr] : 0.0;
      Xs[rr * ks + c] = (AT)v;
    }
    // F^T H group sums: thread c owns column c (no atomics; rows in order, so reproducible)
    if ((int)threadIdx.x < k)
      for (int rr = 0; rr < rows; ++rr) gs[labs[rr] * k + threadIdx.x] += H[(size_t)(t0 + rr) * k + threadIdx.x];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < MP; ++q) {
      if (pi[q] < 0) continue;
      AT s = AT(0);
      for (int rr = 0; rr < rows; ++rr) s = fma(Xs[rr * ks + pi[q]], Xs[rr * ks + pj[q]], s);
      tot[q] += (double)s;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < h * k; i += blockDim.x) partial[(size_t)blockIdx.x * P + i] = gs[i];
  for (int q = 0; q < MP; ++q)
    if (pi[q] >= 0) partial[(size_t)blockIdx.x * P + h * k + pi[q] * k + pj[q]] = tot[q];
}

void launch_diagnostics(int n, int k, int h, const double* H, const double* deg, const uint8_t* lab,
                        const double* params, double* partial, int nblocks, double* out, cudaStream_t s, bool fp64) {
  (void)params;
  (void)out;
  if (k > 64) fail(SFAIRSC_ERR_UNSUPPORTED, "diagnostics support k <= 64");
  const size_t P = (size_t)h * k + (size_t)k * k;
  check_cuda(cudaMemsetAsync(partial, 0, sizeof(double) * P * nblocks, s), "memset");
  if (fp64) {
    const size_t smem = sizeof(double) * ((size_t)h * k + 64 * (size_t)(k + 1));
    check_cuda(cudaFuncSetAttribute(diagnostics_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "attr");
    diagnostics_kernel<double><<<nblocks, 256, smem, s>>>(n, k, h, H, deg, lab, partial);
  } else {
    const size_t smem = sizeof(double) * (size_t)h * k + sizeof(float) * 64 * (size_t)(k + 1);
    check_cuda(cudaFuncSetAttribute(diagnostics_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "attr");
    diagnostics_kernel<float><<<nblocks, 256, smem, s>>>(n, k, h, H, deg, lab, partial);
  }
  check_cuda(cudaGetLastError(), "diagnostics launch");
}

}  // namespace sfairsc
