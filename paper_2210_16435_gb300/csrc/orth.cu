// Block Gram-Schmidt step of the restarted block Lanczos (Algorithm 3 step 3):
// orthogonalise the new block U = L_n^sigma Q against V[:, 0:J], record the
// coefficients in the projected matrix H, orthonormalise the block
// (Cholesky QR) and append it to the basis.
//
// Classical Gram-Schmidt with the DGKS refinement test of ARPACK (the
// eigensolver behind the paper's eigs): the sweep that applies the first
// projection also forms the second coefficients and the Gram matrix; a third
// sweep applies the second projection only when some column kept less than
// 1/sqrt(2) of its norm.  So a launch reads V twice, or three times.
//
// One cooperative launch; each CTA owns a contiguous row range of the
// ROW-major basis (n x ldv).  Rows stream through a ring of shared-memory
// stages filled by the bulk-copy (TMA) engine (cp.async.bulk + mbarrier),
// so the bytes in flight do not occupy registers.  Lane l of a warp owns
// columns 4l..4l+3 (+128 per chunk).  Inner products accumulate per lane in
// FP32 over windows of 32 rows and are carried in FP64 per warp, then summed
// over warps and CTAs in a fixed order (bitwise reproducible); the FP64
// path accumulates in FP64 throughout.  Every mbarrier wait is bounded.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "internal.h"

namespace sfairsc {

// 2-D tiled bulk copy of a box {Jc columns, rows} of V into shared memory.
__device__ __forceinline__ void tensor_g2s_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

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
  int* sweeps;
  int J, j;
};

template <typename VT, int NC>
struct OrthShape {
  static constexpr int kThreads = 512;
  static constexpr int kWarps = kThreads / 32;
  static constexpr int kRowsPerWarp = (sizeof(VT) == 4 ? 4 : 2) / NC;
  static constexpr int kGroupRows = kWarps * kRowsPerWarp;  // rows per ring stage
  static constexpr int kCols = 128 * NC;                     // columns one warp covers
  static constexpr int kStages = NC == 1 ? 3 : 2;  // ring + per-warp sums stay under 227 KB
  static constexpr size_t kStageElems = (size_t)kGroupRows * kCols + (size_t)kGroupRows * 4;  // V box + U rows
};

template <typename VT>
__device__ __forceinline__ void lds_row4(const VT* p, VT (&x)[4]) {
  if constexpr (sizeof(VT) == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
  } else {
    const double2 a = reinterpret_cast<const double2*>(p)[0];
    const double2 b = reinterpret_cast<const double2*>(p)[1];
    x[0] = a.x; x[1] = a.y; x[2] = b.x; x[3] = b.y;
  }
}

template <typename VT, int B>
__device__ __forceinline__ void load_u(const VT* U, int r, VT (&u)[B]) {
  if constexpr (sizeof(VT) == 4 && B == 4) {
    const float4 v = *reinterpret_cast<const float4*>(U + (size_t)r * 4);
    u[0] = v.x; u[1] = v.y; u[2] = v.z; u[3] = v.w;
  } else {
#pragma unroll
    for (int v = 0; v < B; ++v) u[v] = U[(size_t)r * 4 + v];
  }
}

// CTA b owns pairs p = b, b + grid, ...; sums partial[i][p] over CTAs i in
// a fixed order and writes out[p].  Ends with __syncthreads.
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

// All CTAs: out[t] = sum over CTAs of partial[i][off + t], t < cnt (fixed order).
__device__ __forceinline__ void reduce_all(const double* partial, int stride, int off, int cnt, double* out) {
  if ((int)threadIdx.x < cnt) {
    double s = 0.0;
    for (int i = 0; i < (int)gridDim.x; ++i) s += __ldcg(partial + (size_t)i * stride + off + threadIdx.x);
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

constexpr int kWindow = 64;

template <typename VT, int B, int NC>
__global__ void __launch_bounds__(512, 1) orth_kernel(OrthArgs<VT> a, const __grid_constant__ CUtensorMap vmap) {
  using S = OrthShape<VT, NC>;
  extern __shared__ __align__(128) unsigned char smraw[];
  unsigned char* sm = smraw + ((128u - (smem_u32(smraw) & 127u)) & 127u);  // 128-byte aligned stages
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int CW = S::kCols;
  VT* ring = reinterpret_cast<VT*>(sm);                                                   // stages
  double* tot = reinterpret_cast<double*>(sm + sizeof(VT) * S::kStages * S::kStageElems);  // warps x CW x B
  double* scratch = tot + (size_t)S::kWarps * CW * B;                                     // 512
  __shared__ __align__(8) uint64_t full[S::kStages], empty[S::kStages];
  __shared__ double gram_s[16], R1[16], R2[16], Rd1[16], Rd2[16], unorm[4];
  __shared__ int brk, again, abort_flag;

  const int r0 = a.cta_rows[blockIdx.x], r1 = a.cta_rows[blockIdx.x + 1];
  const int J = a.J, P = J * B;
  const int Jc = (J + 3) & ~3;
  const int kNorm = CW * B, kGram = kNorm + 4, kGram2 = kGram + 16, stride = kGram2 + 16;
  VT* U = a.U;
  if (threadIdx.x == 0) {
    brk = 0;
    for (int s = 0; s < S::kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], S::kWarps);
    }
    mbar_fence_init();
  }
  __syncthreads();
  long seq = 0;  // ring groups issued so far (same value in every thread)

  auto colof = [&](int q, int i) { return 128 * q + 4 * lane + i; };

  // Stream the CTA's rows of V[:, 0:Jc] through the ring; consume(r, row_in_smem) per row.
  auto stream = [&](auto&& consume) -> bool {
    const int ngroups = (r1 - r0 + S::kGroupRows - 1) / S::kGroupRows;
    const unsigned rowbytes = (unsigned)(Jc * sizeof(VT));
    auto issue = [&](int g) {
      // one tiled copy of rows rg..rg+kGroupRows-1, columns 0..Jc-1 (rows past n read as zero),
      // and one linear copy of the same rows of U (clipped at n)
      const int s = (int)((seq + g) % S::kStages);
      const int rg = r0 + g * S::kGroupRows;
      const int nu = min(S::kGroupRows, a.n - rg);
      const unsigned ubytes = (unsigned)(nu * 4 * sizeof(VT));
      VT* st = ring + (size_t)s * S::kStageElems;
      mbar_arrive_expect_tx(&full[s], (unsigned)S::kGroupRows * rowbytes + ubytes);
      tensor_g2s_2d(st, &vmap, 0, rg, &full[s]);
      bulk_g2s(st + (size_t)S::kGroupRows * S::kCols, U + (size_t)rg * 4, ubytes, &full[s]);
    };
    if (threadIdx.x == 0) {
      fence_proxy_async();
      for (int g = 0; g < min(S::kStages, ngroups); ++g) issue(g);
    }
    if (threadIdx.x == 0) abort_flag = 0;
    __syncthreads();
    int g = 0;
    for (; g < ngroups; ++g) {
      const long q = seq + g;
      const int s = (int)(q % S::kStages);
      const unsigned par = (unsigned)((q / S::kStages) & 1);
      if (!mbar_wait(&full[s], par, a.err)) atomicExch(&abort_flag, 1);
      if (*(volatile int*)&abort_flag) break;
      const VT* stage = ring + (size_t)s * S::kStageElems;
      const int rw = r0 + g * S::kGroupRows + warp * S::kRowsPerWarp;
      consume(rw, stage + (size_t)warp * S::kRowsPerWarp * Jc,
              stage + (size_t)S::kGroupRows * S::kCols + (size_t)warp * S::kRowsPerWarp * 4);
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
      if (threadIdx.x == 0 && g + S::kStages < ngroups) {
        if (mbar_wait(&empty[s], par, a.err)) {
          fence_proxy_async();
          issue(g + S::kStages);
        } else {
          atomicExch(&abort_flag, 1);
        }
      }
    }
    __syncthreads();
    if (abort_flag) {
      // drain: wait (bounded) for every copy this CTA issued before returning
      if (threadIdx.x == 0) {
        for (int gg = 0; gg < ngroups; ++gg) {
          const long q = seq + gg;
          if (!mbar_try_wait(&full[(int)(q % S::kStages)], (unsigned)((q / S::kStages) & 1)))
            mbar_wait(&full[(int)(q % S::kStages)], (unsigned)((q / S::kStages) & 1), a.err, 100000000ull);
        }
      }
      __syncthreads();
      return false;
    }
    seq += ngroups;
    __syncthreads();
    return true;
  };

  auto zero_tot = [&]() {
    for (int i = lane; i < CW * B; i += 32) tot[(size_t)warp * CW * B + i] = 0.0;
    __syncwarp();
  };
  // CTA partial of the column sums (columns < J), warps in order.
  auto store_tot = [&]() {
    __syncthreads();
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
      double s = 0.0;
      for (int w = 0; w < S::kWarps; ++w) s += tot[(size_t)w * CW * B + p];
      a.partial[(size_t)blockIdx.x * stride + p] = s;
    }
  };
  auto store_small = [&](double val, int cnt, int off) {
    // lanes t < cnt of every warp hold val; CTA sum to partial[off + t]
    __syncthreads();
    if (lane < cnt) scratch[warp * 16 + lane] = val;
    __syncthreads();
    if ((int)threadIdx.x < cnt) {
      double s = 0.0;
      for (int w = 0; w < S::kWarps; ++w) s += scratch[w * 16 + threadIdx.x];
      a.partial[(size_t)blockIdx.x * stride + off + threadIdx.x] = s;
    }
  };

  // sweep kinds: 0 = coefficients (+ input norms); 1 = update with a.coef, then
  // next coefficients and Gram; 2 = update with a.coef, then Gram only.
  auto sweep = [&](int kind) -> bool {
    VT cr[NC][4][B];
#pragma unroll
    for (int q = 0; q < NC; ++q)
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int v = 0; v < B; ++v) {
          const int c = colof(q, i);
          cr[q][i][v] = (kind > 0 && c < J) ? (VT)__ldcg(a.coef + (size_t)c * B + v) : VT(0);
        }
    if (kind < 2) zero_tot();
    VT win[NC][4][B];
#pragma unroll
    for (int q = 0; q < NC; ++q)
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int v = 0; v < B; ++v) win[q][i][v] = VT(0);
    double side = 0.0;  // lanes < B: input norms (kind 0); lanes < B*B: Gram (kinds 1, 2)
    VT sidew = VT(0);   // its FP32 window
    int cnt = 0;
    auto flush = [&]() {
      side += (double)sidew;
      sidew = VT(0);
      if (kind == 2) return;
#pragma unroll
      for (int q = 0; q < NC; ++q)
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int v = 0; v < B; ++v) {
            tot[((size_t)warp * CW + colof(q, i)) * B + v] += (double)win[q][i][v];
            win[q][i][v] = VT(0);
          }
    };
    const bool ok = stream([&](int rw, const VT* rows, const VT* us) {
      constexpr int R = S::kRowsPerWarp;
      VT x[R][NC][4];
      VT u[R][B];
      bool live[R];
#pragma unroll
      for (int t = 0; t < R; ++t) {
        live[t] = rw + t < r1;
#pragma unroll
        for (int q = 0; q < NC; ++q) {
          if (colof(q, 0) < Jc) {
            lds_row4(rows + (size_t)t * Jc + colof(q, 0), x[t][q]);
#pragma unroll
            for (int i = 0; i < 4; ++i)
              if (colof(q, i) >= J || !live[t]) x[t][q][i] = VT(0);
          } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) x[t][q][i] = VT(0);
          }
        }
#pragma unroll
        for (int v = 0; v < B; ++v) u[t][v] = live[t] ? us[t * 4 + v] : VT(0);
      }
      if (kind > 0) {
        VT d[R][B];
#pragma unroll
        for (int t = 0; t < R; ++t)
#pragma unroll
          for (int v = 0; v < B; ++v) d[t][v] = VT(0);
#pragma unroll
        for (int t = 0; t < R; ++t)
#pragma unroll
          for (int q = 0; q < NC; ++q)
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
              for (int v = 0; v < B; ++v) d[t][v] = fma(x[t][q][i], cr[q][i][v], d[t][v]);
        // interleaved butterfly reductions of all R x B partial dots
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
          for (int t = 0; t < R; ++t)
#pragma unroll
            for (int v = 0; v < B; ++v) d[t][v] += __shfl_xor_sync(0xffffffffu, d[t][v], o);
#pragma unroll
        for (int t = 0; t < R; ++t) {
#pragma unroll
          for (int v = 0; v < B; ++v) u[t][v] -= d[t][v];
          if (lane == 0 && live[t]) {
#pragma unroll
            for (int v = 0; v < B; ++v) U[(size_t)(rw + t) * 4 + v] = u[t][v];
          }
          VT ua = VT(0), ub = VT(0);
#pragma unroll
          for (int v = 0; v < B; ++v)
#pragma unroll
            for (int w2 = 0; w2 < B; ++w2)
              if (lane == v * B + w2) {
                ua = u[t][v];
                ub = u[t][w2];
              }
          sidew = fma(ua, ub, sidew);
        }
      } else {
#pragma unroll
        for (int t = 0; t < R; ++t) {
          VT uu = VT(0);
#pragma unroll
          for (int v = 0; v < B; ++v) uu = lane == v ? u[t][v] : uu;
          sidew = fma(uu, uu, sidew);
        }
      }
      if (kind < 2) {
#pragma unroll
        for (int t = 0; t < R; ++t)
#pragma unroll
          for (int q = 0; q < NC; ++q)
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
              for (int v = 0; v < B; ++v) win[q][i][v] = fma(x[t][q][i], u[t][v], win[q][i][v]);
      }
      cnt += R;
      if (cnt >= kWindow) {
        flush();
        cnt = 0;
      }
    });
    if (!ok) return false;
    flush();
    if (kind < 2) store_tot();
    if (kind == 0) store_small(side, B, kNorm);
    else store_small(side, B * B, kGram);
    return true;
  };

  // Thread-per-row Gram of U (B x B) to partial[off..], optionally after U <- U R1^{-1}.
  auto gram_rows = [&](int off, bool apply_r1) {
    double gacc[B][B];
#pragma unroll
    for (int v = 0; v < B; ++v)
#pragma unroll
      for (int w2 = 0; w2 < B; ++w2) gacc[v][w2] = 0.0;
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
      VT u[B];
      load_u<VT, B>(U, r, u);
      if (apply_r1) {
#pragma unroll
        for (int v = 0; v < B; ++v) {
          VT s = u[v];
#pragma unroll
          for (int q = 0; q < v; ++q) s -= u[q] * (VT)Rd1[q * B + v];
          u[v] = s / (VT)Rd1[v * B + v];
        }
#pragma unroll
        for (int v = 0; v < B; ++v) U[(size_t)r * 4 + v] = u[v];
      }
#pragma unroll
      for (int v = 0; v < B; ++v)
#pragma unroll
        for (int w2 = 0; w2 < B; ++w2) gacc[v][w2] = fma((double)u[v], (double)u[w2], gacc[v][w2]);
    }
    __syncthreads();
#pragma unroll
    for (int v = 0; v < B; ++v)
#pragma unroll
      for (int w2 = 0; w2 < B; ++w2) {
        const double s = warp_allsum(gacc[v][w2]);
        if (lane == 0) scratch[warp * 16 + v * B + w2] = s;
      }
    __syncthreads();
    if (threadIdx.x < B * B) {
      double s = 0.0;
      for (int w = 0; w < S::kWarps; ++w) s += scratch[w * 16 + threadIdx.x];
      a.partial[(size_t)blockIdx.x * stride + off + threadIdx.x] = s;
    }
  };

  // Cholesky of gram_s = R^T R (R upper).  A column whose remaining norm
  // vanishes relative to its input norm marks a breakdown: its row of R is
  // zero (as recorded in H) and Rd keeps a unit divisor.
  auto cholesky = [&](double* R, double* Rd) {
    if (threadIdx.x == 0) {
      for (int i = 0; i < B * B; ++i) R[i] = Rd[i] = 0.0;
      for (int c = 0; c < B; ++c) {
        double dsum = gram_s[c * B + c];
        for (int q = 0; q < c; ++q) dsum -= R[q * B + c] * R[q * B + c];
        const double ref = unorm[c] > 0.0 ? unorm[c] : gram_s[c * B + c];
        const double floor_rel = sizeof(VT) == 8 ? 1e-24 : 1e-10;
        if (!(dsum > floor_rel * ref) || !(dsum > 0.0)) {
          brk = 1;
          R[c * B + c] = dsum > 0.0 ? sqrt(dsum) : 0.0;
          Rd[c * B + c] = 1.0;
          continue;
        }
        const double rc = sqrt(dsum);
        R[c * B + c] = rc;
        Rd[c * B + c] = rc;
        for (int q = c + 1; q < B; ++q) {
          double s = gram_s[c * B + q];
          for (int p = 0; p < c; ++p) s -= R[p * B + c] * R[p * B + q];
          R[c * B + q] = s / rc;
          Rd[c * B + q] = s / rc;
        }
      }
    }
    __syncthreads();
  };

  int sweeps = 0;
  if (J > 0) {
    // sweep 1: c1 = V^T U and the input norms
    if (!sweep(0)) return;
    ++sweeps;
    if (!grid_sync(a.bar, a.err)) return;
    reduce_owned(a.partial, stride, P, a.coef, scratch);
    if (a.j >= 0)
      for (int p = blockIdx.x; p < P; p += gridDim.x) a.H[(size_t)(p / B) + (size_t)a.ldh * (a.j + p % B)] = a.coef[p];
    reduce_all(a.partial, stride, kNorm, B, unorm);
    if (!grid_sync(a.bar, a.err)) return;
    // sweep 2: U -= V c1; c2 = V^T U; Gram
    if (!sweep(1)) return;
    ++sweeps;
    if (!grid_sync(a.bar, a.err)) return;
    reduce_all(a.partial, stride, kGram, B * B, gram_s);
    if (threadIdx.x == 0) {
      again = 0;
      for (int v = 0; v < B; ++v)
        if (gram_s[v * B + v] < 0.5 * unorm[v]) again = 1;  // DGKS: kept less than 1/sqrt(2) of the norm
    }
    __syncthreads();
    if (again) {
      reduce_owned(a.partial, stride, P, a.coef, scratch);
      if (a.j >= 0)
        for (int p = blockIdx.x; p < P; p += gridDim.x) a.H[(size_t)(p / B) + (size_t)a.ldh * (a.j + p % B)] += a.coef[p];
      if (!grid_sync(a.bar, a.err)) return;
      // sweep 3: U -= V c2; Gram
      if (!sweep(2)) return;
      ++sweeps;
      if (!grid_sync(a.bar, a.err)) return;
      reduce_all(a.partial, stride, kGram, B * B, gram_s);
    }
  } else {
    if (threadIdx.x < B) unorm[threadIdx.x] = 0.0;
    gram_rows(kGram, false);
    if (!grid_sync(a.bar, a.err)) return;
    reduce_all(a.partial, stride, kGram, B * B, gram_s);
  }
  cholesky(R1, Rd1);

  if (B > 1) {
    // Cholesky QR a second time: U <- U R1^{-1}, Gram again
    gram_rows(kGram2, true);
    if (!grid_sync(a.bar, a.err)) return;
    reduce_all(a.partial, stride, kGram2, B * B, gram_s);
    if (threadIdx.x < B) unorm[threadIdx.x] = 0.0;
    __syncthreads();
    cholesky(R2, Rd2);
  } else {
    if (threadIdx.x == 0) {
      R2[0] = 1.0;
      Rd2[0] = 1.0;
    }
    __syncthreads();
  }

  // V[:, J:J+B] = U R^{-1} and its copy Q
  for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    VT u[B];
    load_u<VT, B>(U, r, u);
    if (B > 1) {
#pragma unroll
      for (int v = 0; v < B; ++v) {
        VT s = u[v];
#pragma unroll
        for (int q = 0; q < v; ++q) s -= u[q] * (VT)Rd2[q * B + v];
        u[v] = s / (VT)Rd2[v * B + v];
      }
    } else {
      u[0] = u[0] / (VT)Rd1[0];
    }
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
    atomicAdd(a.sweeps, sweeps);
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

template <typename VT, int B, int NC>
static size_t orth_smem() {
  using S = OrthShape<VT, NC>;
  return sizeof(VT) * S::kStages * S::kStageElems + sizeof(double) * ((size_t)S::kWarps * S::kCols * B + 512) + 256;
}

// Tensor map of the basis V (row-major n x ldv) with a box of Jc columns x rows.
static void make_vmap(CUtensorMap* map, bool f64, void* V, int n, int64_t ldv, int Jc, int rows) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    check_cuda(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q),
               "driver entry point cuTensorMapEncodeTiled");
    if (!fn || q != cudaDriverEntryPointSuccess) fail(SFAIRSC_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const size_t vs = f64 ? 8 : 4;
  const cuuint64_t dims[2] = {(cuuint64_t)ldv, (cuuint64_t)n};
  const cuuint64_t strides[1] = {(cuuint64_t)(ldv * vs)};
  const cuuint32_t box[2] = {(cuuint32_t)Jc, (cuuint32_t)rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(map, f64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, V, dims,
                            strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) fail(SFAIRSC_ERR_CUDA, "cuTensorMapEncodeTiled failed for the basis");
}

template <typename VT, int B, int NC>
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
  a.sweeps = p.sweeps;
  a.J = J;
  a.j = j;
  const size_t smem = orth_smem<VT, B, NC>();
  auto kern = orth_kernel<VT, B, NC>;
  check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "orth smem attr");
  alignas(64) CUtensorMap vmap;
  const int Jc = (J + 3) & ~3;
  make_vmap(&vmap, sizeof(VT) == 8, p.V, p.n, p.ldv, Jc > 0 ? Jc : 4, OrthShape<VT, NC>::kGroupRows);
  void* args[] = {&a, &vmap};
  check_cuda(cudaLaunchCooperativeKernel((void*)kern, dim3(p.grid), dim3(OrthShape<VT, NC>::kThreads), args, smem, s),
             "orth cooperative launch");
}

template <typename VT, int B>
static void orth_launch_b(const OrthPlan& p, int J, int j, cudaStream_t s) {
  if (J <= 128) orth_launch_t<VT, B, 1>(p, J, j, s);
  else orth_launch_t<VT, B, 2>(p, J, j, s);
}

void launch_orth(const OrthPlan& p, VecType vt, int J, int j, int B, cudaStream_t s) {
  if (J > 256) fail(SFAIRSC_ERR_UNSUPPORTED, "Krylov basis larger than 256 columns");
  if (p.ldv % 4 != 0) fail(SFAIRSC_ERR_UNSUPPORTED, "basis leading dimension must be a multiple of 4");
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

template <typename VT, int B, int NC>
static int orth_grid_t() {
  auto kern = orth_kernel<VT, B, NC>;
  const size_t smem = orth_smem<VT, B, NC>();
  check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "orth smem attr");
  int per_sm = 0, dev = 0, sms = 0;
  check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, OrthShape<VT, NC>::kThreads, smem),
             "orth occupancy");
  check_cuda(cudaGetDevice(&dev), "get device");
  check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "sm count");
  return per_sm * sms;
}

int orth_max_grid(VecType vt, int B, int threads) {
  (void)threads;
  int g = 1 << 30;
  auto upd = [&](int x) { g = x < g ? x : g; };
  if (vt == VecType::F64) {
    if (B == 1) { upd(orth_grid_t<double, 1, 1>()); upd(orth_grid_t<double, 1, 2>()); }
    else if (B == 2) { upd(orth_grid_t<double, 2, 1>()); upd(orth_grid_t<double, 2, 2>()); }
    else { upd(orth_grid_t<double, 4, 1>()); upd(orth_grid_t<double, 4, 2>()); }
  } else {
    if (B == 1) { upd(orth_grid_t<float, 1, 1>()); upd(orth_grid_t<float, 1, 2>()); }
    else if (B == 2) { upd(orth_grid_t<float, 2, 1>()); upd(orth_grid_t<float, 2, 2>()); }
    else { upd(orth_grid_t<float, 4, 1>()); upd(orth_grid_t<float, 4, 2>()); }
  }
  return g;
}

}  // namespace sfairsc
