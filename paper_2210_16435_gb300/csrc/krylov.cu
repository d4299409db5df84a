// Krylov-subspace kernels of the restarted block Lanczos (Algorithm 3 step 3):
// CGS2 orthogonalisation of a new block against the basis, Cholesky-QR of the
// block, thick restart V <- V Y, and the final FP64 checks / embedding.
//
// The basis V is ROW-major (n x ldv): a warp reads one row of up to 256
// basis coefficients as 32-lane coalesced lines, each lane owning a column.
// Inner products V^T u accumulate in FP64 (FP64 path) or in compensated
// FP32 pairs (Dot2, mixed path), and are reduced across CTAs in a fixed
// order, so every run is bitwise reproducible.
#include "common.cuh"
#include "internal.h"

namespace sfairsc {

template <typename VT>
struct Acc;
template <>
struct Acc<float> {
  Dot2 d;
  __device__ __forceinline__ void add(float a, float b) { d.add_prod(a, b); }
  __device__ __forceinline__ double value() const { return d.value(); }
};
template <>
struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ double value() const { return s; }
};

template <typename VT>
struct OrthArgs {
  int n;
  int64_t ldv;
  VT* V;
  VT* U;  // row-major n x 4
  VT* Q;  // row-major n x 4, copy of the new block
  double* H;
  int ldh;
  double* partial;
  double* coef;
  const int32_t* __restrict__ cta_rows;
  GridBarrier bar;
  unsigned* err;
  int* brk_step;
  int J, j;
};

template <typename VT, int B>
__device__ __forceinline__ void load_u(const VT* U, int r, VT (&u)[B]) {
#pragma unroll
  for (int v = 0; v < B; ++v) u[v] = U[(size_t)r * 4 + v];
}

// Per-CTA column partials: acc[g][v] of every warp -> partial[cta][c*B+v] (c < J), fixed warp order.
template <typename VT, int B, int MAXG>
__device__ __forceinline__ void store_columns(Acc<VT> (&acc)[MAXG][B], int G, int J, double* red, double* partial,
                                              int stride) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
#pragma unroll
  for (int g = 0; g < MAXG; ++g) {
    if (g >= G) break;
#pragma unroll
    for (int v = 0; v < B; ++v) red[(warp * 32 + lane) * B + v] = acc[g][v].value();
    __syncthreads();
    for (int t = threadIdx.x; t < 32 * B; t += blockDim.x) {
      const int c = g * 32 + t / B;
      double s = 0.0;
      for (int w = 0; w < nwarps; ++w) s += red[w * 32 * B + t];
      if (c < J) partial[(size_t)blockIdx.x * stride + (size_t)g * 32 * B + t] = s;
    }
    __syncthreads();
  }
}

// CTA b owns pairs p = b, b + grid, ...; it sums partial[i][p] over all CTAs i
// in a fixed order and writes out[p].  Returns after a __syncthreads.
__device__ __forceinline__ void reduce_owned(const double* partial, int stride, int P, double* out, double* scratch) {
  const int nct = gridDim.x;
  const int Q = P > (int)blockIdx.x ? (P - (int)blockIdx.x + nct - 1) / nct : 0;
  if (Q == 0) {
    __syncthreads();
    return;
  }
  const int T = blockDim.x;
  const int nchunk = max(1, min(nct, T / Q));
  const int t = threadIdx.x, q = t % Q, c = t / Q;
  const int p = blockIdx.x + q * nct;
  if (c < nchunk) {
    const int lo = (int)((long long)c * nct / nchunk), hi = (int)((long long)(c + 1) * nct / nchunk);
    double s = 0.0;
    for (int i = lo; i < hi; ++i) s += __ldcg(partial + (size_t)i * stride + p);
    scratch[c * Q + q] = s;
  }
  __syncthreads();
  if (t < Q) {
    double s = 0.0;
    for (int cc = 0; cc < nchunk; ++cc) s += scratch[cc * Q + t];
    out[blockIdx.x + t * nct] = s;
  }
  __syncthreads();
}

template <typename VT, int B, int MAXG>
__global__ void __launch_bounds__(512, 1) orth_kernel(OrthArgs<VT> a) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  double* red = reinterpret_cast<double*>(sm);     // nwarps * 32 * B
  double* scratch = red + nwarps * 32 * B;         // blockDim.x
  VT* coef_s = reinterpret_cast<VT*>(scratch + blockDim.x);  // MAXG * 32 * B
  __shared__ double gram_s[16], R1[16], R2[16], unorm[4];
  __shared__ int brk;

  const int r0 = a.cta_rows[blockIdx.x], r1 = a.cta_rows[blockIdx.x + 1];
  const int J = a.J, G = (J + 31) / 32, P = J * B;
  const int stride = MAXG * 32 * B + 16;  // per-CTA partial stride (doubles)
  const VT* V = a.V;
  VT* U = a.U;
  if (threadIdx.x == 0) brk = 0;

  auto load_coef = [&]() {
    for (int i = threadIdx.x; i < MAXG * 32 * B; i += blockDim.x)
      coef_s[i] = i < P ? (VT)__ldcg(a.coef + i) : VT(0);
    __syncthreads();
  };

  if (J > 0) {
    // ---------------- pass 1: c1 = V[:, 0:J]^T U and the input norms
    {
      Acc<VT> acc[MAXG][B];
      Acc<VT> nacc;
      for (int r = r0 + warp; r < r1; r += nwarps) {
        VT u[B];
        load_u<VT, B>(U, r, u);
        const VT* row = V + (size_t)r * a.ldv;
#pragma unroll
        for (int g = 0; g < MAXG; ++g) {
          const int c = g * 32 + lane;
          const VT x = (g < G && c < J) ? row[c] : VT(0);
#pragma unroll
          for (int v = 0; v < B; ++v) acc[g][v].add(x, u[v]);
        }
        VT uu = VT(0);
#pragma unroll
        for (int v = 0; v < B; ++v) uu = lane == v ? u[v] : uu;
        nacc.add(uu, uu);
      }
      store_columns<VT, B, MAXG>(acc, G, J, red, a.partial, stride);
      // input norms (lanes v < B of every warp)
      const double nv = nacc.value();
      if (lane < B) red[warp * B + lane] = nv;
      __syncthreads();
      if (threadIdx.x < B) {
        double s = 0.0;
        for (int w = 0; w < nwarps; ++w) s += red[w * B + threadIdx.x];
        a.partial[(size_t)blockIdx.x * stride + MAXG * 32 * B + threadIdx.x] = s;
      }
      __syncthreads();
    }
    if (!grid_sync(a.bar, a.err)) return;
    reduce_owned(a.partial, stride, P, a.coef, scratch);
    if (a.j >= 0) {
      for (int p = blockIdx.x; p < P; p += gridDim.x) a.H[(size_t)(p / B) + (size_t)a.ldh * (a.j + p % B)] = a.coef[p];
    }
    if (!grid_sync(a.bar, a.err)) return;
    load_coef();
    if (threadIdx.x < B) {
      double s = 0.0;
      for (int i = 0; i < (int)gridDim.x; ++i) s += __ldcg(a.partial + (size_t)i * stride + MAXG * 32 * B + threadIdx.x);
      unorm[threadIdx.x] = s;
    }
    __syncthreads();

    // ---------------- pass 2: u -= V c1; c2 = V^T u
    {
      Acc<VT> acc[MAXG][B];
      for (int r = r0 + warp; r < r1; r += nwarps) {
        VT u[B];
        load_u<VT, B>(U, r, u);
        const VT* row = V + (size_t)r * a.ldv;
        VT x[MAXG];
        VT d[B];
#pragma unroll
        for (int v = 0; v < B; ++v) d[v] = VT(0);
#pragma unroll
        for (int g = 0; g < MAXG; ++g) {
          const int c = g * 32 + lane;
          x[g] = (g < G && c < J) ? row[c] : VT(0);
#pragma unroll
          for (int v = 0; v < B; ++v) d[v] = fma(x[g], coef_s[(g * 32 + lane) * B + v], d[v]);
        }
#pragma unroll
        for (int v = 0; v < B; ++v) u[v] -= warp_allsum(d[v]);
        __syncwarp();
        if (lane == 0) {
#pragma unroll
          for (int v = 0; v < B; ++v) U[(size_t)r * 4 + v] = u[v];
        }
#pragma unroll
        for (int g = 0; g < MAXG; ++g)
#pragma unroll
          for (int v = 0; v < B; ++v) acc[g][v].add(x[g], u[v]);
      }
      store_columns<VT, B, MAXG>(acc, G, J, red, a.partial, stride);
    }
    if (!grid_sync(a.bar, a.err)) return;
    reduce_owned(a.partial, stride, P, a.coef, scratch);
    if (a.j >= 0) {
      for (int p = blockIdx.x; p < P; p += gridDim.x) a.H[(size_t)(p / B) + (size_t)a.ldh * (a.j + p % B)] += a.coef[p];
    }
    if (!grid_sync(a.bar, a.err)) return;
    load_coef();
  } else {
    if (threadIdx.x < B) unorm[threadIdx.x] = 0.0;
    __syncthreads();
  }

  // ---------------- pass 3: u -= V c2 (if J > 0); Gram = U^T U
  {
    Acc<VT> gacc;
    for (int r = r0 + warp; r < r1; r += nwarps) {
      VT u[B];
      load_u<VT, B>(U, r, u);
      if (J > 0) {
        const VT* row = V + (size_t)r * a.ldv;
        VT d[B];
#pragma unroll
        for (int v = 0; v < B; ++v) d[v] = VT(0);
#pragma unroll
        for (int g = 0; g < MAXG; ++g) {
          const int c = g * 32 + lane;
          const VT x = (g < G && c < J) ? row[c] : VT(0);
#pragma unroll
          for (int v = 0; v < B; ++v) d[v] = fma(x, coef_s[(g * 32 + lane) * B + v], d[v]);
        }
#pragma unroll
        for (int v = 0; v < B; ++v) u[v] -= warp_allsum(d[v]);
        __syncwarp();
        if (lane == 0) {
#pragma unroll
          for (int v = 0; v < B; ++v) U[(size_t)r * 4 + v] = u[v];
        }
      }
      VT ua = VT(0), ub = VT(0);
#pragma unroll
      for (int v = 0; v < B; ++v)
#pragma unroll
        for (int q = 0; q < B; ++q)
          if (lane == v * B + q) {
            ua = u[v];
            ub = u[q];
          }
      gacc.add(ua, ub);
    }
    const double gv = gacc.value();
    if (lane < B * B) red[warp * 16 + lane] = gv;
    __syncthreads();
    if (threadIdx.x < B * B) {
      double s = 0.0;
      for (int w = 0; w < nwarps; ++w) s += red[w * 16 + threadIdx.x];
      a.partial[(size_t)blockIdx.x * stride + threadIdx.x] = s;
    }
  }
  if (!grid_sync(a.bar, a.err)) return;
  // Gram in gram_s (row-major B x B) = R^T R with R upper triangular.  A
  // column whose remaining norm vanishes (relative to its input norm) marks a
  // breakdown: its row of R is zero (recorded in H) and Rdiv keeps a unit
  // divisor so no value overflows; the host discards that block.
  __shared__ double Rdiv1[16], Rdiv2[16];
  auto cholesky = [&](double* R, double* Rdiv) {
    if (threadIdx.x == 0) {
      for (int i = 0; i < B * B; ++i) R[i] = Rdiv[i] = 0.0;
      for (int c = 0; c < B; ++c) {
        double dsum = gram_s[c * B + c];
        for (int q = 0; q < c; ++q) dsum -= R[q * B + c] * R[q * B + c];
        const double ref = unorm[c] > 0.0 ? unorm[c] : gram_s[c * B + c];
        const double floor_rel = sizeof(VT) == 8 ? 1e-24 : 1e-10;
        if (!(dsum > floor_rel * ref) || !(dsum > 0.0)) {
          brk = 1;
          R[c * B + c] = dsum > 0.0 ? sqrt(dsum) : 0.0;
          Rdiv[c * B + c] = 1.0;
          continue;
        }
        const double rc = sqrt(dsum);
        R[c * B + c] = rc;
        Rdiv[c * B + c] = rc;
        for (int q = c + 1; q < B; ++q) {
          double s = gram_s[c * B + q];
          for (int p = 0; p < c; ++p) s -= R[p * B + c] * R[p * B + q];
          R[c * B + q] = s / rc;
          Rdiv[c * B + q] = s / rc;
        }
      }
    }
    __syncthreads();
  };
  if (threadIdx.x < B * B) {
    double s = 0.0;
    for (int i = 0; i < (int)gridDim.x; ++i) s += __ldcg(a.partial + (size_t)i * stride + threadIdx.x);
    gram_s[threadIdx.x] = s;
  }
  __syncthreads();
  cholesky(R1, Rdiv1);

  // Row-wise triangular solve x R = u (R upper): x_v = (u_v - sum_{q<v} x_q R_qv) / R_vv.
  auto tri = [&](const double* R, VT (&u)[B]) {
#pragma unroll
    for (int v = 0; v < B; ++v) {
      VT s = u[v];
#pragma unroll
      for (int q = 0; q < v; ++q) s -= u[q] * (VT)R[q * B + v];
      u[v] = s / (VT)R[v * B + v];
    }
  };

  if (B > 1) {
    // ---------------- pass 4: U <- U R1^{-1}, Gram again (Cholesky-QR twice)
    __syncthreads();
    Acc<VT> g2[B][B];
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
      VT u[B];
      load_u<VT, B>(U, r, u);
      tri(Rdiv1, u);
#pragma unroll
      for (int v = 0; v < B; ++v) U[(size_t)r * 4 + v] = u[v];
#pragma unroll
      for (int v = 0; v < B; ++v)
#pragma unroll
        for (int q = 0; q < B; ++q) g2[v][q].add(u[v], u[q]);
    }
#pragma unroll
    for (int v = 0; v < B; ++v)
#pragma unroll
      for (int q = 0; q < B; ++q) {
        const double s = warp_allsum(g2[v][q].value());
        if (lane == 0) red[warp * 16 + v * B + q] = s;
      }
    __syncthreads();
    if (threadIdx.x < B * B) {
      double s = 0.0;
      for (int w = 0; w < nwarps; ++w) s += red[w * 16 + threadIdx.x];
      a.partial[(size_t)blockIdx.x * stride + 16 + threadIdx.x] = s;
    }
    if (!grid_sync(a.bar, a.err)) return;
    if (threadIdx.x < B * B) {
      double s = 0.0;
      for (int i = 0; i < (int)gridDim.x; ++i) s += __ldcg(a.partial + (size_t)i * stride + 16 + threadIdx.x);
      gram_s[threadIdx.x] = s;
    }
    if (threadIdx.x < B) unorm[threadIdx.x] = 0.0;
    __syncthreads();
    cholesky(R2, Rdiv2);
  } else {
    if (threadIdx.x == 0) {
      R2[0] = 1.0;
      Rdiv2[0] = 1.0;
    }
    __syncthreads();
  }

  // ---------------- pass 5: V[:, J:J+B] = U R^{-1}; H[J:J+B, j:j+B] = R2 R1
  for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    VT u[B];
    load_u<VT, B>(U, r, u);
    if (B > 1) tri(Rdiv2, u);
    else u[0] = u[0] / (VT)Rdiv1[0];
#pragma unroll
    for (int v = 0; v < B; ++v) {
      a.V[(size_t)r * a.ldv + J + v] = u[v];
      a.Q[(size_t)r * 4 + v] = u[v];
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (brk) {
      atomicOr(a.err, kErrBreakdown);
      atomicMin(a.brk_step, a.j);
    }
    if (a.j >= 0) {
      for (int q = 0; q < B; ++q)
        for (int v = 0; v < B; ++v) {
          double s = 0.0;
          if (B > 1) {
            for (int p = 0; p < B; ++p) s += R2[q * B + p] * R1[p * B + v];
          } else {
            s = R1[0];
          }
          a.H[(size_t)(J + q) + (size_t)a.ldh * (a.j + v)] = q <= v ? s : 0.0;
        }
    }
  }
}

static size_t orth_smem(int threads, int B, int MAXG, size_t vs) {
  return sizeof(double) * ((size_t)(threads / 32) * 32 * B + threads) + vs * MAXG * 32 * B + 64;
}

template <typename VT, int B, int MAXG>
static void orth_launch_t(const OrthPlan& p, int J, int j, cudaStream_t s) {
  OrthArgs<VT> a;
  a.n = p.n;
  a.ldv = p.ldv;
  a.V = static_cast<VT*>(p.V);
  a.U = static_cast<VT*>(p.U);
  a.Q = static_cast<VT*>(p.Q);
  a.H = p.H;
  a.ldh = p.ldh;
  a.partial = p.partial;
  a.coef = p.coef;
  a.cta_rows = p.cta_rows;
  a.bar = GridBarrier{p.barrier, p.barrier + 1};
  a.err = p.err;
  a.brk_step = p.brk_step;
  a.J = J;
  a.j = j;
  const size_t smem = orth_smem(p.threads, B, MAXG, sizeof(VT));
  auto kern = orth_kernel<VT, B, MAXG>;
  check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "orth smem attr");
  void* args[] = {&a};
  check_cuda(cudaLaunchCooperativeKernel((void*)kern, dim3(p.grid), dim3(p.threads), args, smem, s),
             "orth cooperative launch");
}

template <typename VT, int B>
static void orth_launch_b(const OrthPlan& p, int J, int j, cudaStream_t s) {
  if (J <= 128) orth_launch_t<VT, B, 4>(p, J, j, s);
  else orth_launch_t<VT, B, 8>(p, J, j, s);
}

void launch_orth(const OrthPlan& p, VecType vt, int J, int j, int B, cudaStream_t s) {
  if (J > 256) fail(SFAIRSC_ERR_UNSUPPORTED, "Krylov basis larger than 256 columns");
  if (vt == VecType::F64) {
    if (B == 1) orth_launch_b<double, 1>(p, J, j, s);
    else if (B == 2) orth_launch_b<double, 2>(p, J, j, s);
    else orth_launch_b<double, 4>(p, J, j, s);
  } else {
    if (B == 1) orth_launch_b<float, 1>(p, J, j, s);
    else if (B == 2) orth_launch_b<float, 2>(p, J, j, s);
    else orth_launch_b<float, 4>(p, J, j, s);
  }
}

template <typename VT, int B, int MAXG>
static int orth_grid_t(int threads) {
  auto kern = orth_kernel<VT, B, MAXG>;
  const size_t smem = orth_smem(threads, B, MAXG, sizeof(VT));
  check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "orth smem attr");
  int per_sm = 0, dev = 0, sms = 0;
  check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem), "orth occupancy");
  check_cuda(cudaGetDevice(&dev), "get device");
  check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "sm count");
  return per_sm * sms;
}

int orth_max_grid(VecType vt, int B, int threads) {
  int g = 1 << 30;
  auto upd = [&](int x) { g = x < g ? x : g; };
  if (vt == VecType::F64) {
    if (B == 1) { upd(orth_grid_t<double, 1, 4>(threads)); upd(orth_grid_t<double, 1, 8>(threads)); }
    else if (B == 2) { upd(orth_grid_t<double, 2, 4>(threads)); upd(orth_grid_t<double, 2, 8>(threads)); }
    else { upd(orth_grid_t<double, 4, 4>(threads)); upd(orth_grid_t<double, 4, 8>(threads)); }
  } else {
    if (B == 1) { upd(orth_grid_t<float, 1, 4>(threads)); upd(orth_grid_t<float, 1, 8>(threads)); }
    else if (B == 2) { upd(orth_grid_t<float, 2, 4>(threads)); upd(orth_grid_t<float, 2, 8>(threads)); }
    else { upd(orth_grid_t<float, 4, 4>(threads)); upd(orth_grid_t<float, 4, 8>(threads)); }
  }
  return g;
}

// ---------------------------------------------------------------- thick restart
// V[r, 0:K] = V[r, 0:m] Y for a 32-row tile held in shared memory (in place),
// then V[r, K:K+B] = V[r, m:m+B] (the residual block carried over).
template <typename VT>
__global__ void __launch_bounds__(1024) restart_kernel(int n, VT* V, int64_t ldv, int m, int K, int B,
                                                       const double* __restrict__ Y, VT* Q) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int width = m + B;
  VT* Vs = reinterpret_cast<VT*>(sm);  // 32 x width
  VT* Ys = Vs + 32 * width;            // m x 64
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rbase = blockIdx.x * 32;
  const int rows = min(32, n - rbase);
  for (int i = threadIdx.x; i < rows * width; i += blockDim.x) {
    const int rr = i / width, c = i % width;
    Vs[rr * width + c] = V[(size_t)(rbase + rr) * ldv + c];
  }
  for (int k0 = 0; k0 < K; k0 += 64) {
    const int kc = min(64, K - k0);
    __syncthreads();
    for (int i = threadIdx.x; i < m * 64; i += blockDim.x) {
      const int c = i / 64, kk = i % 64;
      Ys[i] = kk < kc ? (VT)Y[(size_t)c + (size_t)(k0 + kk) * m] : VT(0);
    }
    __syncthreads();
    if (warp < rows) {
      VT acc0 = VT(0), acc1 = VT(0);
      const VT* vr = Vs + warp * width;
      for (int c = 0; c < m; ++c) {
        const VT x = vr[c];
        acc0 = fma(x, Ys[c * 64 + lane], acc0);
        acc1 = fma(x, Ys[c * 64 + 32 + lane], acc1);
      }
      VT* out = V + (size_t)(rbase + warp) * ldv + k0;
      if (lane < kc) out[lane] = acc0;
      if (32 + lane < kc) out[32 + lane] = acc1;
    }
  }
  __syncthreads();
  if (warp < rows && lane < B) {
    const VT x = Vs[warp * width + m + lane];
    V[(size_t)(rbase + warp) * ldv + K + lane] = x;
    Q[(size_t)(rbase + warp) * 4 + lane] = x;
  }
}

void launch_restart(VecType vt, int n, void* V, int64_t ldv, int m, int K, int B, const double* Y, void* Q,
                    cudaStream_t s) {
  const int grid = (n + 31) / 32;
  if (vt == VecType::F64) {
    const size_t smem = sizeof(double) * (32 * (size_t)(m + B) + (size_t)m * 64);
    check_cuda(cudaFuncSetAttribute(restart_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
               "restart smem");
    restart_kernel<double><<<grid, 1024, smem, s>>>(n, (double*)V, ldv, m, K, B, Y, (double*)Q);
  } else {
    const size_t smem = sizeof(float) * (32 * (size_t)(m + B) + (size_t)m * 64);
    check_cuda(cudaFuncSetAttribute(restart_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
               "restart smem");
    restart_kernel<float><<<grid, 1024, smem, s>>>(n, (float*)V, ldv, m, K, B, Y, (float*)Q);
  }
  check_cuda(cudaGetLastError(), "restart launch");
}

// X64[r + c n] = sum_q V[r, q] Y[q, c]: a 32-row tile of V in shared memory,
// warp per row, lanes over output columns.  V is not modified.
template <typename VT>
__global__ void __launch_bounds__(1024) ritz_kernel(int n, const VT* V, int64_t ldv, int m, int k,
                                                   const double* __restrict__ Y, double* X) {
  extern __shared__ __align__(16) unsigned char sm[];
  VT* Vs = reinterpret_cast<VT*>(sm);  // 32 x m
  VT* Ys = Vs + 32 * m;                // m x 64
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rbase = blockIdx.x * 32;
  const int rows = min(32, n - rbase);
  for (int i = threadIdx.x; i < rows * m; i += blockDim.x) {
    const int rr = i / m, c = i % m;
    Vs[rr * m + c] = V[(size_t)(rbase + rr) * ldv + c];
  }
  for (int k0 = 0; k0 < k; k0 += 64) {
    const int kc = min(64, k - k0);
    __syncthreads();
    for (int i = threadIdx.x; i < m * 64; i += blockDim.x) {
      const int c = i / 64, kk = i % 64;
      Ys[i] = kk < kc ? (VT)Y[(size_t)c + (size_t)(k0 + kk) * m] : VT(0);
    }
    __syncthreads();
    if (warp < rows) {
      VT acc0 = VT(0), acc1 = VT(0);
      const VT* vr = Vs + warp * m;
      for (int c = 0; c < m; ++c) {
        const VT x = vr[c];
        acc0 = fma(x, Ys[c * 64 + lane], acc0);
        acc1 = fma(x, Ys[c * 64 + 32 + lane], acc1);
      }
      const int r = rbase + warp;
      if (lane < kc) X[(size_t)r + (size_t)(k0 + lane) * n] = (double)acc0;
      if (32 + lane < kc) X[(size_t)r + (size_t)(k0 + 32 + lane) * n] = (double)acc1;
    }
  }
}

void launch_ritz(VecType vt, int n, const void* V, int64_t ldv, int m, int k, const double* Y, double* X64,
                 cudaStream_t s) {
  const int grid = (n + 31) / 32;
  if (vt == VecType::F64) {
    const size_t smem = sizeof(double) * (32 * (size_t)m + (size_t)m * 64);
    check_cuda(cudaFuncSetAttribute(ritz_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "ritz smem");
    ritz_kernel<double><<<grid, 1024, smem, s>>>(n, (const double*)V, ldv, m, k, Y, X64);
  } else {
    const size_t smem = sizeof(float) * (32 * (size_t)m + (size_t)m * 64);
    check_cuda(cudaFuncSetAttribute(ritz_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "ritz smem");
    ritz_kernel<float><<<grid, 1024, smem, s>>>(n, (const float*)V, ldv, m, k, Y, X64);
  }
  check_cuda(cudaGetLastError(), "ritz launch");
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
  for (int c = 0; c < k; ++c) X[(size_t)r + (size_t)c * n] = (double)V[(size_t)r * ldv + c];
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

__global__ void embed_kernel(int n, int k, const double* __restrict__ X, const double* __restrict__ dinv,
                             int normalized, const unsigned long long* colkey, double* H) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const double sc = normalized ? dinv[r] : 1.0;
  for (int c = 0; c < k; ++c) {
    const double piv = X[(size_t)c * n + colkey[k + c]];
    const double sg = piv < 0.0 ? -1.0 : 1.0;
    H[(size_t)r * k + c] = sg * sc * X[(size_t)c * n + r];
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
  embed_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, k, X, dinv64, normalized, colkey, H);
  check_cuda(cudaGetLastError(), "embed launch");
}

// ---------------------------------------------------------------- diagnostics
// Per block: group sums of H columns (h x k) and the k x k Gram of H^T D H.
__global__ void diagnostics_kernel(int n, int k, int h, const double* __restrict__ H, const double* __restrict__ deg,
                                   const uint8_t* __restrict__ lab, double* partial) {
  extern __shared__ double acc[];  // h*k + k*k
  const int P = h * k + k * k;
  for (int i = threadIdx.x; i < P; i += blockDim.x) acc[i] = 0.0;
  __syncthreads();
  const int per = (n + gridDim.x - 1) / gridDim.x;
  const int lo = blockIdx.x * per, hi = min(n, lo + per);
  // group sums: one thread per (row)
  for (int r = lo + threadIdx.x; r < hi; r += blockDim.x) {
    const int g = lab[r];
    for (int c = 0; c < k; ++c) atomicAdd(&acc[g * k + c], H[(size_t)r * k + c]);
  }
  // Gram: threads over pairs, loop over rows
  for (int p = threadIdx.x; p < k * k; p += blockDim.x) {
    const int c1 = p / k, c2 = p % k;
    if (c2 < c1) continue;
    double s = 0.0;
    for (int r = lo; r < hi; ++r) s = fma(deg[r] * H[(size_t)r * k + c1], H[(size_t)r * k + c2], s);
    acc[h * k + p] += s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < P; i += blockDim.x) partial[(size_t)blockIdx.x * P + i] = acc[i];
}

void launch_diagnostics(int n, int k, int h, const double* H, const double* deg, const uint8_t* lab,
                        const double* params, double* partial, int nblocks, double* out, cudaStream_t s) {
  (void)params;
  (void)out;
  const size_t smem = sizeof(double) * ((size_t)h * k + (size_t)k * k);
  check_cuda(cudaFuncSetAttribute(diagnostics_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
             "diagnostics smem");
  diagnostics_kernel<<<nblocks, 256, smem, s>>>(n, k, h, H, deg, lab, partial);
  check_cuda(cudaGetLastError(), "diagnostics launch");
}

}  // namespace sfairsc
