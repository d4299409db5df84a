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
// One cooperative launch; each CTA owns a contiguous row range.  The basis
// is stored as 4-column panels (panel p holds columns 4p..4p+3 as an n x 4
// row-major array), so 32 consecutive rows of a panel are one contiguous
// 16-byte-per-row run.  A warp takes 32-row blocks in two phases:
//   phase A, one lane per row: load the row's panels (coalesced 512-byte
//     warp loads), subtract V c (coefficients broadcast from shared memory),
//     store the row, add its Gram entries;
//   phase B, LPR lanes per row, lane p holding panel p: add the row's
//     products to the new coefficients V^T u (the panels come back from L1/L2).
// FP32 path: inner products in FP32 windows carried by TwoSum and combined
// over lanes by a TwoSum tree, then in FP64 over warps and CTAs in a fixed
// order (bitwise reproducible).  FP64 path: FP64 throughout.
#include "common.cuh"
#include "internal.h"

namespace sfairsc {

namespace {

constexpr int kOT = 512;  // threads per CTA
constexpr int kOW = kOT / 32;
constexpr int kCoefMax = 256 * 4;  // J * B
constexpr int kNormOff = kCoefMax, kGramOff = kCoefMax + 4, kGram2Off = kCoefMax + 20, kStride = kCoefMax + 36;
// per-warp partials: coefficients + 16 extras (J <= 128 columns when NC = 1)
template <int NC>
constexpr int red_stride() {
  return (NC == 1 ? 128 * 4 : kCoefMax) + 16;
}

// Accumulator: a window in VT plus a carry (TwoSum pair for FP32, plain FP64 for FP64).
template <typename VT>
struct Acc;
template <>
struct Acc<float> {
  float w;
  Comp32 k;
  __device__ __forceinline__ void zero() {
    w = 0.f;
    k.zero();
  }
  __device__ __forceinline__ void fma_(float x, float y) { w = fmaf(x, y, w); }
  __device__ __forceinline__ void flush() {
    k.add(w);
    w = 0.f;
  }
  __device__ __forceinline__ void reduce(int from) {
    flush();
    k.reduce(from);
  }
  __device__ __forceinline__ double value() const { return k.value(); }
};
template <>
struct Acc<double> {
  double w;
  __device__ __forceinline__ void zero() { w = 0.0; }
  __device__ __forceinline__ void fma_(double x, double y) { w = fma(x, y, w); }
  __device__ __forceinline__ void flush() {}
  __device__ __forceinline__ void reduce(int from) {
    for (int o = from; o < 32; o <<= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
  }
  __device__ __forceinline__ double value() const { return w; }
};

template <typename VT>
__device__ __forceinline__ void ld4(const VT* p, VT (&x)[4]) {
  if constexpr (sizeof(VT) == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    x[0] = v.x;
    x[1] = v.y;
    x[2] = v.z;
    x[3] = v.w;
  } else {
    const double2 a = reinterpret_cast<const double2*>(p)[0];
    const double2 b = reinterpret_cast<const double2*>(p)[1];
    x[0] = a.x;
    x[1] = a.y;
    x[2] = b.x;
    x[3] = b.y;
  }
}
template <typename VT>
__device__ __forceinline__ void st4(VT* p, const VT (&x)[4]) {
  if constexpr (sizeof(VT) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
  } else {
    reinterpret_cast<double2*>(p)[0] = make_double2(x[0], x[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(x[2], x[3]);
  }
}

__device__ __forceinline__ int lanes_for(int np) {
  return np <= 1 ? 1 : np <= 2 ? 2 : np <= 4 ? 4 : np <= 8 ? 8 : np <= 16 ? 16 : 32;
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

}  // namespace

template <typename VT>
struct OrthArgs {
  int n;
  VT* V;  // panels of n x 4
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

// Shared memory: coefficients (kCoefMax VT), per-warp partials (kOW x
// red_stride doubles), reduction scratch (1024 doubles), per-warp updated rows
// (kOW x 32 x 4 VT).  Kept small so that L1 holds the panels phase B re-reads.
template <typename VT, int NC>
constexpr size_t orth_smem_bytes() {
  return sizeof(VT) * kCoefMax + sizeof(double) * ((size_t)kOW * red_stride<NC>() + 1024) + sizeof(VT) * kOW * 32 * 4 +
         256;
}

template <typename VT, int B, int NC>
__global__ void __launch_bounds__(kOT, 1) orth_kernel(OrthArgs<VT> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  VT* cfs = reinterpret_cast<VT*>(smraw);                                  // coefficients c*B + v
  constexpr int kRed = red_stride<NC>();
  constexpr int kXo = kRed - 16;                                           // extras offset
  double* red = reinterpret_cast<double*>(smraw + sizeof(VT) * kCoefMax);  // kOW x kRed
  double* scratch = red + (size_t)kOW * kRed;                              // 1024
  VT* uws = reinterpret_cast<VT*>(scratch + 1024);                         // kOW x 32 x 4
  __shared__ double gram_s[16], R1[16], R2[16], Rd1[16], Rd2[16], unorm[4];
  __shared__ int brk, again;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r0 = a.cta_rows[blockIdx.x], r1 = a.cta_rows[blockIdx.x + 1];
  const int J = a.J, P = J * B;
  const int np = (J + 3) / 4;  // panels holding columns 0..J-1
  const size_t pn = (size_t)a.n * 4;
  constexpr int NG = B * (B + 1) / 2;  // unique Gram entries
  constexpr int NA = NG > B ? NG : B;
  VT* U = a.U;
  VT* uw = uws + (size_t)warp * 32 * 4;
  if (threadIdx.x == 0) brk = 0;
  __syncthreads();

  // sweep kinds: 0 = coefficients + input norms; 1 = update with a.coef, then the
  // next coefficients and the Gram matrix; 2 = update with a.coef, then the Gram matrix.
  auto sweep = [&](int kind) {
    const bool upd = kind >= 1, want_c = kind <= 1;
    if (upd) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) cfs[i] = (VT)__ldcg(a.coef + i);
      __syncthreads();
    }
    const int LPR = NC == 1 ? lanes_for(np) : 32;
    const int RPW = 32 / LPR;
    const int p0 = lane & (LPR - 1), ri = lane / LPR;
    Acc<VT> acc[NC][4][B];
    Acc<VT> ga[NA];
#pragma unroll
    for (int q = 0; q < NC; ++q)
#pragma unroll
      for (int jj = 0; jj < 4; ++jj)
#pragma unroll
        for (int v = 0; v < B; ++v) acc[q][jj][v].zero();
#pragma unroll
    for (int e = 0; e < NA; ++e) ga[e].zero();
    int nb = 0;
    for (int rb = r0 + warp * 32; rb < r1; rb += kOW * 32) {
      // ---- phase A: lane = row
      const int r = rb + lane;
      VT u[4] = {VT(0), VT(0), VT(0), VT(0)};
      if (r < r1) {
        ld4(U + (size_t)r * 4, u);
        if (upd) {
          VT d[B];
#pragma unroll
          for (int v = 0; v < B; ++v) d[v] = VT(0);
          const int nfull = J >> 2;  // panels whose 4 columns are all < J
#pragma unroll 8
          for (int pp = 0; pp < nfull; ++pp) {
            VT x[4];
            ld4(a.V + pp * pn + (size_t)r * 4, x);
#pragma unroll
            for (int jj = 0; jj < 4; ++jj)
#pragma unroll
              for (int v = 0; v < B; ++v) d[v] = fma(x[jj], cfs[(4 * pp + jj) * B + v], d[v]);
          }
          if (nfull < np) {
            VT x[4];
            ld4(a.V + nfull * pn + (size_t)r * 4, x);
            for (int jj = 0; jj < (J & 3); ++jj)
#pragma unroll
              for (int v = 0; v < B; ++v) d[v] = fma(x[jj], cfs[(4 * nfull + jj) * B + v], d[v]);
          }
#pragma unroll
          for (int v = 0; v < B; ++v) u[v] -= d[v];
          st4(U + (size_t)r * 4, u);
        } else {
          for (int pp = 0; pp < np; ++pp) asm volatile("prefetch.global.L1 [%0];" ::"l"(a.V + pp * pn + (size_t)r * 4));
        }
      }
      if (kind == 0) {
#pragma unroll
        for (int v = 0; v < B; ++v) ga[v].fma_(u[v], u[v]);
      } else {
        int e = 0;
#pragma unroll
        for (int v = 0; v < B; ++v)
#pragma unroll
          for (int w2 = v; w2 < B; ++w2) ga[e++].fma_(u[v], u[w2]);
      }
      if (want_c) st4(uw + lane * 4, u);
      __syncwarp();
      // ---- phase B: LPR lanes per row, lane p0 (+32 q) holding panel p0 (+32 q)
      if (want_c) {
        const int nrow = min(32, r1 - rb);
        for (int s0 = 0; s0 < LPR; s0 += 4) {
          // four rows' loads in flight before their products
          VT xs[4][NC][4], us[4][4];
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int i = ri + RPW * (s0 + t);
            const bool in = s0 + t < LPR && i < nrow;
            if (in) ld4(uw + i * 4, us[t]);
            else us[t][0] = us[t][1] = us[t][2] = us[t][3] = VT(0);
#pragma unroll
            for (int q = 0; q < NC; ++q) {
              const int pp = p0 + 32 * q;
              if (in && pp < np) {
                ld4(a.V + pp * pn + (size_t)(rb + i) * 4, xs[t][q]);
                if (4 * pp + 4 > J)
#pragma unroll
                  for (int jj = 0; jj < 4; ++jj)
                    if (4 * pp + jj >= J) xs[t][q][jj] = VT(0);
              } else {
                xs[t][q][0] = xs[t][q][1] = xs[t][q][2] = xs[t][q][3] = VT(0);
              }
            }
          }
#pragma unroll
          for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int q = 0; q < NC; ++q)
#pragma unroll
              for (int jj = 0; jj < 4; ++jj)
#pragma unroll
                for (int v = 0; v < B; ++v) acc[q][jj][v].fma_(xs[t][q][jj], us[t][v]);
        }
      }
      __syncwarp();
      if (++nb == 4) {
#pragma unroll
        for (int q = 0; q < NC; ++q)
#pragma unroll
          for (int jj = 0; jj < 4; ++jj)
#pragma unroll
            for (int v = 0; v < B; ++v) acc[q][jj][v].flush();
#pragma unroll
        for (int e = 0; e < NA; ++e) ga[e].flush();
        nb = 0;
      }
    }
    // ---- combine over the warp's lanes, then over warps into this CTA's partial
#pragma unroll
    for (int q = 0; q < NC; ++q)
#pragma unroll
      for (int jj = 0; jj < 4; ++jj)
#pragma unroll
        for (int v = 0; v < B; ++v) acc[q][jj][v].reduce(LPR);
#pragma unroll
    for (int e = 0; e < NA; ++e) ga[e].reduce(1);
    double* rw = red + (size_t)warp * kRed;
    if (want_c && ri == 0)
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        const int pp = p0 + 32 * q;
        if (pp < np)
#pragma unroll
          for (int jj = 0; jj < 4; ++jj)
            if (4 * pp + jj < J)
#pragma unroll
              for (int v = 0; v < B; ++v) rw[(4 * pp + jj) * B + v] = acc[q][jj][v].value();
      }
    if (lane == 0) {
      if (kind == 0) {
#pragma unroll
        for (int v = 0; v < B; ++v) rw[kXo + v] = ga[v].value();
      } else {
        int e = 0;
#pragma unroll
        for (int v = 0; v < B; ++v)
#pragma unroll
          for (int w2 = v; w2 < B; ++w2) {
            const double g = ga[e++].value();
            rw[kXo + v * B + w2] = g;
            rw[kXo + w2 * B + v] = g;
          }
      }
    }
    __syncthreads();
    if (want_c)
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < kOW; ++w) s += red[(size_t)w * kRed + i];
        a.partial[(size_t)blockIdx.x * kStride + i] = s;
      }
    const int ne = kind == 0 ? B : B * B;
    if ((int)threadIdx.x < ne) {
      double s = 0.0;
      for (int w = 0; w < kOW; ++w) s += red[(size_t)w * kRed + kXo + threadIdx.x];
      a.partial[(size_t)blockIdx.x * kStride + (kind == 0 ? kNormOff : kGramOff) + threadIdx.x] = s;
    }
  };

  // Thread-per-row Gram of U (B x B) to partial[off..], optionally after U <- U R1^{-1}.
  auto gram_rows = [&](int off, bool apply_r1) {
    Acc<VT> g[NG];
#pragma unroll
    for (int e = 0; e < NG; ++e) g[e].zero();
    int nb = 0;
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
      VT u[4];
      ld4(U + (size_t)r * 4, u);
      if (apply_r1) {
#pragma unroll
        for (int v = 0; v < B; ++v) {
          VT s = u[v];
#pragma unroll
          for (int q = 0; q < v; ++q) s -= u[q] * (VT)Rd1[q * B + v];
          u[v] = s / (VT)Rd1[v * B + v];
        }
        st4(U + (size_t)r * 4, u);
      }
      int e = 0;
#pragma unroll
      for (int v = 0; v < B; ++v)
#pragma unroll
        for (int w2 = v; w2 < B; ++w2) g[e++].fma_(u[v], u[w2]);
      if (++nb == 16) {
#pragma unroll
        for (int ee = 0; ee < NG; ++ee) g[ee].flush();
        nb = 0;
      }
    }
#pragma unroll
    for (int e = 0; e < NG; ++e) g[e].reduce(1);
    __syncthreads();
    if (lane == 0) {
      int e = 0;
#pragma unroll
      for (int v = 0; v < B; ++v)
#pragma unroll
        for (int w2 = v; w2 < B; ++w2) {
          const double x = g[e++].value();
          scratch[warp * 16 + v * B + w2] = x;
          scratch[warp * 16 + w2 * B + v] = x;
        }
    }
    __syncthreads();
    if ((int)threadIdx.x < B * B) {
      double s = 0.0;
      for (int w = 0; w < kOW; ++w) s += scratch[w * 16 + threadIdx.x];
      a.partial[(size_t)blockIdx.x * kStride + off + threadIdx.x] = s;
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
    sweep(0);
    ++sweeps;
    if (!grid_sync(a.bar, a.err)) return;
    reduce_owned(a.partial, kStride, P, a.coef, scratch);
    if (a.j >= 0)
      for (int p = blockIdx.x; p < P; p += gridDim.x) a.H[(size_t)(p / B) + (size_t)a.ldh * (a.j + p % B)] = a.coef[p];
    reduce_all(a.partial, kStride, kNormOff, B, unorm);
    if (!grid_sync(a.bar, a.err)) return;
    // sweep 2: U -= V c1; c2 = V^T U; Gram
    sweep(1);
    ++sweeps;
    if (!grid_sync(a.bar, a.err)) return;
    reduce_all(a.partial, kStride, kGramOff, B * B, gram_s);
    if (threadIdx.x == 0) {
      again = 0;
      for (int v = 0; v < B; ++v)
        if (gram_s[v * B + v] < 0.5 * unorm[v]) again = 1;  // DGKS: kept less than 1/sqrt(2) of the norm
    }
    __syncthreads();
    if (again) {
      reduce_owned(a.partial, kStride, P, a.coef, scratch);
      if (a.j >= 0)
        for (int p = blockIdx.x; p < P; p += gridDim.x) a.H[(size_t)(p / B) + (size_t)a.ldh * (a.j + p % B)] += a.coef[p];
      if (!grid_sync(a.bar, a.err)) return;
      // sweep 3: U -= V c2; Gram
      sweep(2);
      ++sweeps;
      if (!grid_sync(a.bar, a.err)) return;
      reduce_all(a.partial, kStride, kGramOff, B * B, gram_s);
    }
  } else {
    if (threadIdx.x < B) unorm[threadIdx.x] = 0.0;
    gram_rows(kGramOff, false);
    if (!grid_sync(a.bar, a.err)) return;
    reduce_all(a.partial, kStride, kGramOff, B * B, gram_s);
  }
  cholesky(R1, Rd1);

  if (B > 1) {
    // Cholesky QR a second time: U <- U R1^{-1}, Gram again
    gram_rows(kGram2Off, true);
    if (!grid_sync(a.bar, a.err)) return;
    reduce_all(a.partial, kStride, kGram2Off, B * B, gram_s);
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

  // V[:, J:J+B] = U R^{-1} (inside panel J/4: J % 4 + B <= 4) and its copy Q
  VT* Vp = a.V + (size_t)(J / 4) * pn;
  const int c0 = J & 3;
  for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    VT u[4];
    ld4(U + (size_t)r * 4, u);
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
      Vp[(size_t)r * 4 + c0 + v] = u[v];
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
static void orth_launch_t(const OrthPlan& p, int J, int j, cudaStream_t s) {
  OrthArgs<VT> a;
  a.n = p.n;
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
  const size_t smem = orth_smem_bytes<VT, NC>();
  auto kern = orth_kernel<VT, B, NC>;
  check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "orth smem attr");
  void* args[] = {&a};
  check_cuda(cudaLaunchCooperativeKernel((void*)kern, dim3(p.grid), dim3(kOT), args, smem, s), "orth cooperative launch");
}

template <typename VT, int B>
static void orth_launch_b(const OrthPlan& p, int J, int j, cudaStream_t s) {
  if (J <= 128) orth_launch_t<VT, B, 1>(p, J, j, s);
  else orth_launch_t<VT, B, 2>(p, J, j, s);
}

void launch_orth(const OrthPlan& p, VecType vt, int J, int j, int B, cudaStream_t s) {
  if (J > 256) fail(SFAIRSC_ERR_UNSUPPORTED, "Krylov basis larger than 256 columns");
  if ((J & 3) + B > 4) fail(SFAIRSC_ERR_UNSUPPORTED, "a new block must fit in one 4-column panel");
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
  const size_t smem = orth_smem_bytes<VT, NC>();
  check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "orth smem attr");
  int per_sm = 0, dev = 0, sms = 0;
  check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kOT, smem), "orth occupancy");
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
