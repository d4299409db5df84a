// Fused s-FairSC operator: out = L_n^sigma w = P(L_n(P w)) - sigma P w + sigma w
// (Sec. 3.4 (i)), with P w = w - C (C^T C)^{-1} C^T w (eq. mv-Pw),
// C = D^{-1/2} F and F built from the group labels (Lemma 2.1).
//
// With labels, C^T w needs only h group sums:
//   (C^T w)_s = T_s - z_s sum_t T_t,   T_s = sum_{i in V_s} d_i^{-1/2} w_i,
// and (C a)_i = d_i^{-1/2} (a'_{g_i} - z.a) with a'_s = a_s (s < h-1), a'_{h-1} = 0.
// Writing y = P w, t = L_n y and b = (C^T C)^{-1} C^T t, the operator is
//   out = t - C (b - sigma a),
// an exact rewrite of Sec. 3.4 (i) (P t - sigma y + sigma w = t - C b + sigma C a).
//
// One cooperative launch, every CTA owning a contiguous row range:
//   A  group sums T over own rows                       -> grid barrier 1
//   B  reduce T, solve for a, write ytil = D^{-1/2} y   -> grid barrier 2
//   C  SpMV t_i = y_i - d_i^{-1/2} sum_j w_ij ytil_j,
//      write t, group sums of D^{-1/2} t                -> grid barrier 3
//   D  reduce, solve for b, out = t - C (b - sigma a)
// The unnormalized extension replaces D^{-1/2} by 1 in C and uses L = D - W.
#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"

namespace sfairsc {

template <typename VT, typename MT>
struct OpArgs {
  int n, h, normalized, batch_rows, lanes;
  int mode;  // 0: out = L_n^sigma w;  1: out = P w (projection only)
  const int32_t* __restrict__ row_ptr;
  const int32_t* __restrict__ col;
  const MT* __restrict__ val;
  const uint8_t* __restrict__ lab;
  const VT* __restrict__ dinv;
  const double* __restrict__ deg;
  const double* __restrict__ params;
  const VT* __restrict__ w;
  int64_t wrs, wcs;  // element (r, v) of the input is w[r * wrs + v * wcs]
  VT* out;
  int64_t ors, ocs;  // element (r, v) of the output is out[r * ors + v * ocs]
  VT* ytil;
  double* partial;
  const int32_t* __restrict__ cta_rows;
  GridBarrier bar;
  unsigned* err;
  unsigned* work;  // dynamic row-block counter of the SpMV phase
  unsigned long long wait_ns;  // bound of every grid-barrier wait
  const unsigned* stall;       // fault-injection hook: wait for this (never set) word first
  // shared-memory windows of ytil (WindowTable for this block size); seg_row == nullptr: none
  const int32_t* __restrict__ seg_row;
  const int32_t* __restrict__ seg_ws;
  const int32_t* __restrict__ cta_seg;
  int win_rows;
  int win_off;  // byte offset of the window in dynamic shared memory
  // dense constraints: F (n x fp, row-major, in the vector type) replaces the group labels
  const VT* __restrict__ Fd;
  int fp;
  // C^T t from the projected input: K (n x kpad in 4-column panels, kpad = h rounded up to 4) with
  // C^T t = sum_c y_c K_c; nullptr: the group sums of t in a pass of their own after the SpMV
  const VT* __restrict__ Kp;
  int kpad;
  double* partial2;  // per-CTA sums y^T K (grid x (kpad + 1) x B)
};

template <typename VT, int B>
__device__ __forceinline__ void load_row(const VT* p, VT (&x)[B]);

// B contiguous values through L2 (data written by other CTAs in this launch).
template <typename VT, int B>
__device__ __forceinline__ void load_row_cg(const VT* p, VT (&x)[B]) {
  if constexpr (sizeof(VT) == 4 && B == 4) {
    const float4 v = __ldcg(reinterpret_cast<const float4*>(p));
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
  } else {
#pragma unroll
    for (int v = 0; v < B; ++v) x[v] = __ldcg(p + v);
  }
}

// Element v of row r of a strided n x B block (rs, cs): one vector load when the rows are contiguous.
template <typename VT, int B>
__device__ __forceinline__ void load_strided(const VT* base, int64_t r, int64_t rs, int64_t cs, VT (&x)[B]) {
  if (cs == 1 && rs == B) {
    load_row<VT, B>(base + r * B, x);
  } else {
#pragma unroll
    for (int v = 0; v < B; ++v) x[v] = base[r * rs + v * cs];
  }
}

template <typename VT, int B>
__device__ __forceinline__ void load_row(const VT* p, VT (&x)[B]) {
  if constexpr (sizeof(VT) == 4 && B == 4) {
    float4 v = *reinterpret_cast<const float4*>(p);
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
  } else if constexpr (sizeof(VT) == 4 && B == 2) {
    float2 v = *reinterpret_cast<const float2*>(p);
    x[0] = v.x; x[1] = v.y;
  } else if constexpr (sizeof(VT) == 8 && B == 4) {
    double2 u = reinterpret_cast<const double2*>(p)[0];
    double2 v = reinterpret_cast<const double2*>(p)[1];
    x[0] = u.x; x[1] = u.y; x[2] = v.x; x[3] = v.y;
  } else if constexpr (sizeof(VT) == 8 && B == 2) {
    double2 u = *reinterpret_cast<const double2*>(p);
    x[0] = u.x; x[1] = u.y;
  } else {
#pragma unroll
    for (int v = 0; v < B; ++v) x[v] = p[v];
  }
}

// Sum partial[cta][p] over all CTAs in a fixed order into out[p] (shared).
__device__ __forceinline__ void reduce_partials(const double* partial, int nctas, int P, double* scratch, double* out) {
  const int T = blockDim.x;
  const int nchunk = max(1, min(nctas, T / P));
  const int t = threadIdx.x;
  const int p = t % P, c = t / P;
  if (c < nchunk) {
    const int lo = (int)((long long)c * nctas / nchunk), hi = (int)((long long)(c + 1) * nctas / nchunk);
    double s = 0.0;
    int i = lo;
    for (; i + 4 <= hi; i += 4) {  // four loads in flight, added in order
      const double x0 = __ldcg(partial + (size_t)i * P + p), x1 = __ldcg(partial + (size_t)(i + 1) * P + p);
      const double x2 = __ldcg(partial + (size_t)(i + 2) * P + p), x3 = __ldcg(partial + (size_t)(i + 3) * P + p);
      s += x0;
      s += x1;
      s += x2;
      s += x3;
    }
    for (; i < hi; ++i) s += __ldcg(partial + (size_t)i * P + p);
    scratch[c * P + p] = s;
  }
  __syncthreads();
  if (t < P) {
    double s = 0.0;
    for (int cc = 0; cc < nchunk; ++cc) s += scratch[cc * P + t];
    out[t] = s;
  }
  __syncthreads();
}

// Four consecutive values (16 or 32 bytes, aligned).
template <typename VT>
__device__ __forceinline__ void ld_row4(const VT* p, VT (&x)[4]) {
  if constexpr (sizeof(VT) == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
  } else {
    const double2 u = reinterpret_cast<const double2*>(p)[0], v = reinterpret_cast<const double2*>(p)[1];
    x[0] = u.x; x[1] = u.y; x[2] = v.x; x[3] = v.y;
  }
}

// coef = G tot for every (group, vector) in parallel (G precomputed on the host from the Cholesky
// factor of C^T C: the same small solve for every right-hand side), zero past h groups.
template <int B>
__device__ __forceinline__ void apply_group_map(const double* G, const double* tot, int h, double* coef) {
  for (int i = threadIdx.x; i < kMaxGroups * B; i += blockDim.x) {
    double c = 0.0;
    if (i < h * B) {
      const int s = i / B, v = i % B;
      for (int t = 0; t < h; ++t) c = fma(G[s * h + t], tot[t * B + v], c);
    }
    coef[i] = c;
  }
  __syncthreads();
}

// Group sums of f(r) (B values per row) over rows [r0, r1) of this CTA:
// partial[blockIdx.x][s * B + v] = sum over own rows i in V_s of f(i)_v.
// Thread per row; groups are taken 4 per pass with predicated adds (no
// per-row shuffles).  FP32: per-thread windows of 16 rows carried by TwoSum,
// combined over the warp by a TwoSum tree and over warps by TwoSum, then
// converted to FP64 once; FP64: FP64 throughout.  Warps are added in a fixed
// order, so the result is bitwise reproducible.
template <typename VT, int B, typename F>
__device__ void cta_group_sums(int r0, int r1, int h, const uint8_t* __restrict__ lab, double* red, double* partial,
                               F&& f) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int P = h * B;
  for (int s0 = 0; s0 < h; s0 += 4) {
    if constexpr (sizeof(VT) == 4) {
      constexpr int NA = 4 * B;  // accumulator j * B + v: group s0 + j, vector v
      float win[NA];
      Comp32 acc[NA];
#pragma unroll
      for (int q = 0; q < NA; ++q) {
        win[q] = 0.f;
        acc[q].zero();
      }
      int cnt = 0;
      const int T = blockDim.x;
      constexpr int RF = B == 4 ? 2 : 4;  // rows in flight (fewer at B = 4: registers)
      for (int r = r0 + threadIdx.x; r < r1; r += RF * T) {
        // RF rows' loads in flight before their adds
        int g[RF];
        float x[RF][B];
#pragma unroll
        for (int k = 0; k < RF; ++k) {  // loads are not predicated on the label (one round trip)
          const int rk = r + k * T;
          g[k] = rk < r1 ? (int)lab[rk] - s0 : -1;
          if (rk < r1) f(rk, x[k]);
          else
#pragma unroll
            for (int v = 0; v < B; ++v) x[k][v] = 0.f;
        }
#pragma unroll
        for (int k = 0; k < RF; ++k)
#pragma unroll
          for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int v = 0; v < B; ++v) win[j * B + v] += g[k] == j ? x[k][v] : 0.f;
        if (++cnt == 16 / RF) {  // windows of 16 rows
#pragma unroll
          for (int q = 0; q < NA; ++q) {
            acc[q].add(win[q]);
            win[q] = 0.f;
          }
          cnt = 0;
        }
      }
#pragma unroll
      for (int q = 0; q < NA; ++q) acc[q].add(win[q]);
      // the accumulators over the warp by one reduce-scatter tree; lane L then holds
      // accumulator scatter_index(L)
      comp32_reduce_scatter<NA>(acc, lane);
      {
        const int q = scatter_index<NA>(lane), j = q / B, v = q % B;
        if ((lane & (32 / NA - 1)) == 0 && s0 + j < h) red[warp * P + (s0 + j) * B + v] = acc[0].slot();
      }
    } else {
      constexpr int NA = 4 * B;  // accumulator j * B + v: group s0 + j, vector v
      double acc[NA];
#pragma unroll
      for (int q = 0; q < NA; ++q) acc[q] = 0.0;
      for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        const int g = (int)lab[r] - s0;
        if (g >= 0 && g < 4) {
          double x[B];
          f(r, x);
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (g == j)
#pragma unroll
              for (int v = 0; v < B; ++v) acc[j * B + v] += x[v];
        }
      }
      reduce_scatter<NA>(acc, lane);
      const int q = scatter_index<NA>(lane), j = q / B, v = q % B;
      if ((lane & (32 / NA - 1)) == 0 && s0 + j < h) red[warp * P + (s0 + j) * B + v] = acc[0];
    }
  }
  __syncthreads();
  // warps in a fixed order: FP32 (sum, carry) pairs by TwoSum, one conversion
  // per value (no FP64 arithmetic per warp); FP64 values in FP64
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    double s = 0.0;
    if constexpr (sizeof(VT) == 4) {
      s = comp32_slot_sum(red + p, nwarps, P);
    } else {
      for (int wv = 0; wv < nwarps; ++wv) s += red[wv * P + p];
    }
    partial[(size_t)blockIdx.x * P + p] = s;
  }
  __syncthreads();
}

// Dense-constraint sums C^T x over rows [r0, r1) of this CTA (C = D^{-1/2} F,
// the scaling folded into f): partial[blockIdx.x][s * B + v] = sum_r F[r][s] f(r)_v
// for s < p, zero in the slot s = p.  Thread per row, four columns per pass;
// the same FP32 windows and TwoSum carries as the group sums, fixed order.
template <typename VT, int B, typename FL, typename Fn>
__device__ void cta_dense_sums(int r0, int r1, int p, FL&& fload, double* red, double* partial, Fn&& f) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int h = p + 1, P = h * B;
  for (int s0 = 0; s0 < p; s0 += 4) {
    if constexpr (sizeof(VT) == 4) {
      float win[4][B];
      Comp32 acc[4][B];
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int v = 0; v < B; ++v) {
          win[j][v] = 0.f;
          acc[j][v].zero();
        }
      int cnt = 0;
      for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        float x[B], fr[4];
        f(r, x);
        fload(r, s0, fr);
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
          for (int v = 0; v < B; ++v) win[j][v] = fmaf(fr[j], x[v], win[j][v]);
        if (++cnt == 8) {
#pragma unroll
          for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int v = 0; v < B; ++v) {
              acc[j][v].add(win[j][v]);
              win[j][v] = 0.f;
            }
          cnt = 0;
        }
      }
      Comp32 fl[4 * B];
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int v = 0; v < B; ++v) {
          acc[j][v].add(win[j][v]);
          fl[j * B + v] = acc[j][v];
        }
      comp32_reduce_scatter<4 * B>(fl, lane);
      {
        const int q = scatter_index<4 * B>(lane), j = q / B, v = q % B;
        if ((lane & (32 / (4 * B) - 1)) == 0 && s0 + j < p) red[warp * P + (s0 + j) * B + v] = fl[0].slot();
      }
    } else {
      constexpr int NA = 4 * B;
      double acc[NA];
#pragma unroll
      for (int q = 0; q < NA; ++q) acc[q] = 0.0;
      for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        double x[B], fr[4];
        f(r, x);
        fload(r, s0, fr);
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
          for (int v = 0; v < B; ++v) acc[j * B + v] = fma(fr[j], x[v], acc[j * B + v]);
      }
      reduce_scatter<NA>(acc, lane);
      const int q = scatter_index<NA>(lane), j = q / B, v = q % B;
      if ((lane & (32 / NA - 1)) == 0 && s0 + j < p) red[warp * P + (s0 + j) * B + v] = acc[0];
    }
  }
  if (lane == 0)
#pragma unroll
    for (int v = 0; v < B; ++v) red[warp * P + p * B + v] = 0.0;  // a zero (sum, carry) pair packs to 0.0 too
  __syncthreads();
  for (int q = threadIdx.x; q < P; q += blockDim.x) {
    double sum = 0.0;
    if constexpr (sizeof(VT) == 4) {
      sum = comp32_slot_sum(red + q, nwarps, P);
    } else {
      for (int wv = 0; wv < nwarps; ++wv) sum += red[wv * P + q];
    }
    partial[(size_t)blockIdx.x * P + q] = sum;
  }
  __syncthreads();
}

template <typename VT, typename MT, int B>
__global__ void __launch_bounds__(1024, 1) fused_operator_kernel(OpArgs<VT, MT> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const int h = a.h;
  const int P = h * B;
  const bool grouped = h > 1;
  // shared layout
  const int Pr = ((((h + 3) & ~3)) + 1) * B;            // widest per-warp row: group sums or y^T K
  double* red = reinterpret_cast<double*>(smem_raw);  // nwarps * Pr
  double* scratch = red + nwarps * Pr;                 // blockDim.x (+Pr)
  double* tot = scratch + blockDim.x + Pr;             // (32 + 1) * B
  double* avec = tot + (kMaxGroups + 1) * B;           // 32*B
  double* coefA = avec + kMaxGroups * B;               // 32*B
  double* coefD = coefA + kMaxGroups * B;              // 32*B
  double* Gs = coefD + kMaxGroups * B;                 // h x h: group sums -> correction coefficients
  VT* coefAv = reinterpret_cast<VT*>(Gs + h * h);      // 32*B, in the vector type
  VT* coefDv = coefAv + kMaxGroups * B;                // 32*B, in the vector type
  // (rows of the input contiguous: the extra pass re-reads them, which strided columns make dearer
  // than the pass it saves)
  const bool fusedD = a.Kp != nullptr && grouped && a.mode == 0 && (B == 1 || (a.wcs == 1 && a.wrs == B));
  (void)avec;
  for (int i = threadIdx.x; i < h * h; i += blockDim.x) Gs[i] = a.params[kPG + i];  // synced before use

  const int r0 = a.cta_rows[blockIdx.x], r1 = a.cta_rows[blockIdx.x + 1];
  if (a.stall && !wait_flag(a.stall, a.err, a.wait_ns)) return;

  auto scale = [&](int r) -> VT { return a.normalized ? a.dinv[r] : VT(1); };
  const bool dense = a.Fd != nullptr;
  // (C coef)_r / d_r^{-1/2} for the B vectors: the group's entry, or F's row times coef (dense)
  auto corr = [&](int r, const VT* cv, VT (&c)[B]) {
    if (dense) {
#pragma unroll
      for (int v = 0; v < B; ++v) c[v] = VT(0);
      const VT* fr = a.Fd + (size_t)r * a.fp;
      for (int s2 = 0; s2 < a.fp; ++s2) {
        const VT f = fr[s2];
#pragma unroll
        for (int v = 0; v < B; ++v) c[v] = fma(f, cv[s2 * B + v], c[v]);
      }
    } else {
      const int g = a.lab[r];
#pragma unroll
      for (int v = 0; v < B; ++v) c[v] = cv[g * B + v];
    }
  };
  auto group_sums = [&](auto&& f) {
    if (dense)
      cta_dense_sums<VT, B>(
          r0, r1, a.fp,
          [&](int r, int s0, VT(&fr)[4]) {
#pragma unroll
            for (int j = 0; j < 4; ++j) fr[j] = s0 + j < a.fp ? a.Fd[(size_t)r * a.fp + s0 + j] : VT(0);
          },
          red, a.partial, f);
    else cta_group_sums<VT, B>(r0, r1, h, a.lab, red, a.partial, f);
  };

  // ---------------- phase A: group sums of D^{-1/2} w over own rows
  if (grouped) {
    group_sums([&](int r, VT(&x)[B]) {
      const VT sc = scale(r);
      load_strided<VT, B>(a.w, r, a.wrs, a.wcs, x);
#pragma unroll
      for (int v = 0; v < B; ++v) x[v] *= sc;
    });
    if (!grid_sync(a.bar, a.err, a.wait_ns)) return;
    // ---------------- phase B: a = (C^T C)^{-1} C^T w
    reduce_partials(a.partial, gridDim.x, P, scratch, tot);
    apply_group_map<B>(Gs, tot, h, coefA);
  } else {
    for (int i = threadIdx.x; i < kMaxGroups * B; i += blockDim.x) {
      coefA[i] = 0.0;
      avec[i] = 0.0;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < kMaxGroups * B; i += blockDim.x) coefAv[i] = (VT)coefA[i];
  __syncthreads();
  if (a.mode == 1) {  // P w only
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
      const VT sc = scale(r);
      VT cr[B];
      corr(r, coefAv, cr);
#pragma unroll
      for (int v = 0; v < B; ++v) a.out[r * a.ors + v * a.ocs] = a.w[r * a.wrs + v * a.wcs] - sc * cr[v];
    }
    return;
  }
#pragma unroll 4
  for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    const VT sc = scale(r);
    VT cr[B];
    corr(r, coefAv, cr);
#pragma unroll
    for (int v = 0; v < B; ++v) {
      const VT y = a.w[r * a.wrs + v * a.wcs] - sc * cr[v];
      a.ytil[(size_t)r * B + v] = a.normalized ? sc * y : y;
    }
  }
  if (fusedD) {
    // C^T t = sum_c y_c K_c with K_c = d_c^{-1/2} (F_c - sum_r w_rc F_r / d_r) (normalized) or
    // d_c F_c - sum_r w_rc F_r (not): t = L_n y summed against C by the symmetry of W, so the
    // correction is known before the SpMV and its rows can be written in final form
    const size_t pn = (size_t)a.n * 4;
    cta_dense_sums<VT, B>(
        r0, r1, a.kpad,
        [&](int r, int s0, VT(&fr)[4]) { ld_row4<VT>(a.Kp + (size_t)(s0 >> 2) * pn + (size_t)r * 4, fr); },
        red, a.partial2, [&](int r, VT(&x)[B]) {
          const VT sc = scale(r);
          VT cr[B];
          load_strided<VT, B>(a.w, r, a.wrs, a.wcs, x);
          corr(r, coefAv, cr);
#pragma unroll
          for (int v = 0; v < B; ++v) x[v] -= sc * cr[v];
        });
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.work = 0u;  // no CTA takes a row block before the barrier
  if (!grid_sync(a.bar, a.err, a.wait_ns)) return;
  if (fusedD) {
    const int P2 = (a.kpad + 1) * B;
    reduce_partials(a.partial2, gridDim.x, P2, scratch, tot);
    // C u with u = b - sigma a: coefD = G C^T t - sigma coefA
    const double sigma = a.params[kPSigma];
    for (int i = threadIdx.x; i < kMaxGroups * B; i += blockDim.x) {
      double cd = 0.0;
      if (i < P) {
        const int s2 = i / B, v = i % B;
        for (int t = 0; t < h; ++t) cd = fma(Gs[s2 * h + t], tot[t * B + v], cd);
        cd -= sigma * coefA[i];
      }
      coefDv[i] = (VT)cd;
    }
    __syncthreads();
  }

  // ---------------- phase C (no windows): t = L_n y, written to out
  // Warps take blocks of 4 row groups from a global counter (load balance
  // across CTAs); Lr lanes per row, each holding up to U (column, weight)
  // pairs of its row per pass; within a block the pairs of the next row group
  // and the bounds of the group after it are loaded while this group's ytil
  // rows are gathered.  Sums per row by a fixed shuffle tree (reproducible).
  if (!a.seg_row) {
    constexpr int U = sizeof(VT) == 4 ? 8 : 4;
    constexpr int kGroupsPerBlock = 4;
    const int Lr = a.lanes;
    const int sub = lane & (Lr - 1);
    const int rpw = 32 / Lr;
    const int n = a.n;
    auto bounds = [&](int rb, int rend, int& e, int& e1) {
      const int r = rb + lane / Lr;
      if (r < rend) {
        e = __ldg(a.row_ptr + r) + sub;
        e1 = __ldg(a.row_ptr + r + 1);
      } else {
        e = 0;
        e1 = 0;
      }
    };
    auto fetch = [&](int e, int e1, int (&c)[U], VT (&wv)[U]) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int ee = e + u * Lr;
        const bool in = ee < e1;
        c[u] = in ? __ldg(a.col + ee) : -1;
        wv[u] = in ? val_as<VT>(a.val[ee]) : VT(0);
      }
    };
    const int blk_rows = rpw * kGroupsPerBlock;
    const int nblocks = (n + blk_rows - 1) / blk_rows;
    auto grab = [&]() {
      int b = 0;
      if (lane == 0) b = (int)atomicAdd(a.work, 1u);
      return __shfl_sync(0xffffffffu, b, 0);
    };
    // look-ahead iterator over the row groups of the blocks this warp takes
    // (row base n = exhausted); the block after the current one is taken early
    int la_blk = grab(), la_next = grab();
    int la_rb = la_blk < nblocks ? la_blk * blk_rows : n;
    auto advance = [&]() {
      if (la_rb >= n) return;
      la_rb += rpw;
      if (la_rb >= min(n, la_blk * blk_rows + blk_rows)) {
        la_blk = la_next;
        la_rb = la_blk < nblocks ? la_blk * blk_rows : n;
        if (la_blk < nblocks) la_next = grab();
      }
    };
    auto rend_of = [&](int rb) { return min(n, (rb / blk_rows) * blk_rows + blk_rows); };
    int rb_cur = la_rb;
    advance();
    int rb_nx = la_rb;
    advance();
    int e_cur, e1_cur, e_nx, e1_nx;
    int c_cur[U];
    VT w_cur[U];
    bounds(rb_cur, rb_cur < n ? rend_of(rb_cur) : n, e_cur, e1_cur);
    fetch(e_cur, e1_cur, c_cur, w_cur);
    bounds(rb_nx, rb_nx < n ? rend_of(rb_nx) : n, e_nx, e1_nx);
    while (rb_cur < n) {
      int c_nx[U];
      VT w_nx[U];
      fetch(e_nx, e1_nx, c_nx, w_nx);  // the next group's pairs, in flight during this group's gathers
      const int rb_nn = la_rb;
      advance();
      int e_nn, e1_nn;
      bounds(rb_nn, rb_nn < n ? rend_of(rb_nn) : n, e_nn, e1_nn);
      const int rend = rend_of(rb_cur);
      VT sacc[B];
#pragma unroll
      for (int v = 0; v < B; ++v) sacc[v] = VT(0);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (c_cur[u] >= 0) {
          VT y[B];
          load_row<VT, B>(a.ytil + (size_t)c_cur[u] * B, y);
#pragma unroll
          for (int v = 0; v < B; ++v) sacc[v] = fma(w_cur[u], y[v], sacc[v]);
        }
      }
      for (int e = e_cur + U * Lr; e < e1_cur; e += Lr) {  // rows longer than U * Lr entries
        const int c = __ldg(a.col + e);
        const VT w = val_as<VT>(a.val[e]);
        VT y[B];
        load_row<VT, B>(a.ytil + (size_t)c * B, y);
#pragma unroll
        for (int v = 0; v < B; ++v) sacc[v] = fma(w, y[v], sacc[v]);
      }
      for (int o = Lr >> 1; o > 0; o >>= 1)
#pragma unroll
        for (int v = 0; v < B; ++v) sacc[v] += __shfl_xor_sync(0xffffffffu, sacc[v], o);
      const int r = rb_cur + lane / Lr;
      if (r < rend && sub == 0) {
        const VT sc = scale(r);
        VT dd = VT(1);
        if (!a.normalized) dd = (VT)a.deg[r];
        VT wr[B], cr[B], cd[B];
        load_strided<VT, B>(a.w, r, a.wrs, a.wcs, wr);
        corr(r, coefAv, cr);
        if (fusedD) corr(r, coefDv, cd);
#pragma unroll
        for (int v = 0; v < B; ++v) {
          const VT y = wr[v] - sc * cr[v];
          const VT t = a.normalized ? y - sc * sacc[v] : dd * y - sacc[v];
          a.out[r * a.ors + v * a.ocs] = fusedD ? t - sc * cd[v] : t;
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        c_cur[u] = c_nx[u];
        w_cur[u] = w_nx[u];
      }
      e_cur = e_nx;
      e1_cur = e1_nx;
      e_nx = e_nn;
      e1_nx = e1_nn;
      rb_cur = rb_nx;
      rb_nx = rb_nn;
    }
  }
  // ---------------- phase C (windows): t = L_n y over this CTA's rows, written to out
  // The CTA's rows come as segments; a segment with a window first stages
  // ytil rows [ws, ws + win_rows) in shared memory, and each gather reads
  // from there when its column falls inside, from L2 otherwise (one generic
  // load either way).  A warp takes row groups of 32 / Lr rows in turn; Lr
  // lanes per row each hold up to U (column, weight) pairs of the row per
  // pass, and the next group's pairs are loaded while this group's ytil rows
  // are gathered.  Sums per row by a fixed shuffle tree (reproducible).
  if (a.seg_row) {
    constexpr int U = sizeof(VT) == 4 ? 8 : 4;
    const int Lr = a.lanes;
    const int sub = lane & (Lr - 1);
    const int rpw = 32 / Lr;
    const int n = a.n;
    const int warp = threadIdx.x >> 5;
    VT* win = reinterpret_cast<VT*>(smem_raw + a.win_off);
    const int sg0 = a.cta_seg[blockIdx.x];
    const int sg1 = a.cta_seg[blockIdx.x + 1];
    auto fetch = [&](int e, int e1, int (&c)[U], VT (&wv)[U]) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int ee = e + u * Lr;
        const bool in = ee < e1;
        c[u] = in ? __ldg(a.col + ee) : -1;
        wv[u] = in ? val_as<VT>(a.val[ee]) : VT(0);
      }
    };
    for (int sg = sg0; sg < sg1; ++sg) {
      const int rs = a.seg_row[sg];
      const int re = a.seg_row[sg + 1];
      const int ws = a.seg_ws[sg];
      int wlen = 0;
      if (ws >= 0) {
        wlen = min(a.win_rows, n - ws);
        __syncthreads();  // the previous segment's gathers are done with the window
        // ws is a multiple of 4 rows, so the copy starts 16-byte aligned for every b
        const int total = wlen * B;  // VT elements
        constexpr int PER = 16 / (int)sizeof(VT);
        const int nv = total / PER;
        const int4* src = reinterpret_cast<const int4*>(a.ytil + (size_t)ws * B);
        int4* dst = reinterpret_cast<int4*>(win);
        for (int i = threadIdx.x; i < nv; i += blockDim.x) dst[i] = __ldcg(src + i);
        for (int i = nv * PER + threadIdx.x; i < total; i += blockDim.x) win[i] = __ldcg(a.ytil + (size_t)ws * B + i);
        __syncthreads();
      }
      const unsigned wsu = (unsigned)ws, wlenu = (unsigned)wlen;
      const int ngroups = (re - rs + rpw - 1) / rpw;
      auto bounds = [&](int q, int& e, int& e1) {
        const int r = rs + q * rpw + lane / Lr;
        if (q < ngroups && r < re) {
          e = __ldg(a.row_ptr + r) + sub;
          e1 = __ldg(a.row_ptr + r + 1);
        } else {
          e = 0;
          e1 = 0;
        }
      };
      int q = warp;
      int e_cur, e1_cur, e_nx, e1_nx;
      int c_cur[U];
      VT w_cur[U];
      bounds(q, e_cur, e1_cur);
      fetch(e_cur, e1_cur, c_cur, w_cur);
      bounds(q + nwarps, e_nx, e1_nx);
      for (; q < ngroups; q += nwarps) {
        int c_nx[U];
        VT w_nx[U];
        fetch(e_nx, e1_nx, c_nx, w_nx);  // the next group's pairs, in flight during this group's gathers
        int e_nn, e1_nn;
        bounds(q + 2 * nwarps, e_nn, e1_nn);
        VT sacc[B];
#pragma unroll
        for (int v = 0; v < B; ++v) sacc[v] = VT(0);
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (c_cur[u] >= 0) {
            const unsigned off = (unsigned)c_cur[u] - wsu;
            const VT* src = off < wlenu ? win + (size_t)off * B : a.ytil + (size_t)c_cur[u] * B;
            VT y[B];
            load_row<VT, B>(src, y);
#pragma unroll
            for (int v = 0; v < B; ++v) sacc[v] = fma(w_cur[u], y[v], sacc[v]);
          }
        }
        for (int e = e_cur + U * Lr; e < e1_cur; e += Lr) {  // rows longer than U * Lr entries
          const int c = __ldg(a.col + e);
          const VT w = val_as<VT>(a.val[e]);
          const unsigned off = (unsigned)c - wsu;
          const VT* src = off < wlenu ? win + (size_t)off * B : a.ytil + (size_t)c * B;
          VT y[B];
          load_row<VT, B>(src, y);
#pragma unroll
          for (int v = 0; v < B; ++v) sacc[v] = fma(w, y[v], sacc[v]);
        }
        for (int o = Lr >> 1; o > 0; o >>= 1)
#pragma unroll
          for (int v = 0; v < B; ++v) sacc[v] += __shfl_xor_sync(0xffffffffu, sacc[v], o);
        const int r = rs + q * rpw + lane / Lr;
        if (r < re && sub == 0) {
          const VT sc = scale(r);
          VT dd = VT(1);
          if (!a.normalized) dd = (VT)a.deg[r];
          VT wr[B], cr[B], cd[B];
          load_strided<VT, B>(a.w, r, a.wrs, a.wcs, wr);
          corr(r, coefAv, cr);
          if (fusedD) corr(r, coefDv, cd);
#pragma unroll
          for (int v = 0; v < B; ++v) {
            const VT y = wr[v] - sc * cr[v];
            const VT t = a.normalized ? y - sc * sacc[v] : dd * y - sacc[v];
            a.out[r * a.ors + v * a.ocs] = fusedD ? t - sc * cd[v] : t;
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          c_cur[u] = c_nx[u];
          w_cur[u] = w_nx[u];
        }
        e_cur = e_nx;
        e1_cur = e1_nx;
        e_nx = e_nn;
        e1_nx = e1_nn;
      }
    }
  }
  if (!grouped || fusedD) return;
  // t rows were written by any CTA: make them visible, then group sums over own rows (through L2)
  if (!grid_sync(a.bar, a.err, a.wait_ns)) return;
  group_sums([&](int r, VT(&x)[B]) {
    const VT sc = scale(r);
    if (a.ocs == 1 && a.ors == B) {
      load_row_cg<VT, B>(a.out + (size_t)r * B, x);
#pragma unroll
      for (int v = 0; v < B; ++v) x[v] *= sc;
    } else {
#pragma unroll
      for (int v = 0; v < B; ++v) x[v] = sc * __ldcg(a.out + r * a.ors + v * a.ocs);
    }
  });
  if (!grid_sync(a.bar, a.err, a.wait_ns)) return;

  // ---------------- phase D: b = (C^T C)^{-1} C^T t; out = t - C (b - sigma a)
  reduce_partials(a.partial, gridDim.x, P, scratch, tot);
  {
    // C u with u = b - sigma a is linear in the sums: coefD = G C^T t - sigma coefA
    const double sigma = a.params[kPSigma];
    for (int i = threadIdx.x; i < kMaxGroups * B; i += blockDim.x) {
      double cd = 0.0;
      if (i < P) {
        const int s2 = i / B, v = i % B;
        for (int t = 0; t < h; ++t) cd = fma(Gs[s2 * h + t], tot[t * B + v], cd);
        cd -= sigma * coefA[i];
      }
      coefAv[i] = (VT)cd;
    }
    __syncthreads();
  }
#pragma unroll 4
  for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    const VT sc = scale(r);
    VT cr[B];
    corr(r, coefAv, cr);
#pragma unroll
    for (int v = 0; v < B; ++v) {
      VT* o = a.out + r * a.ors + v * a.ocs;
      *o = __ldcg(o) - sc * cr[v];
    }
  }
}

size_t operator_smem_bytes(int threads, int h, int nvec, VecType vt) {
  const int nwarps = threads / 32;
  const size_t vs = vt == VecType::F64 ? 8 : 4;
  const int Pr = (((h + 3) & ~3) + 1) * nvec;
  return sizeof(double) * ((size_t)nwarps * Pr + threads + Pr + (4 * kMaxGroups + 1) * nvec + (size_t)h * h) +
         2 * vs * kMaxGroups * nvec + 64;
}

template <typename VT, typename MT, int B>
static void launch_t(const OpPlan& p, const void* w, int64_t wrs, int64_t wcs, void* out, int64_t ors, int64_t ocs,
                     cudaStream_t s) {
  OpArgs<VT, MT> a;
  a.n = p.n;
  a.h = p.h;
  a.normalized = p.normalized;
  a.batch_rows = p.batch_rows;
  a.lanes = p.lanes_per_row;
  a.mode = p.mode;
  a.row_ptr = p.row_ptr;
  a.col = p.col;
  a.val = static_cast<const MT*>(p.val);
  a.lab = p.lab;
  a.dinv = static_cast<const VT*>(p.dinv);
  a.deg = p.deg;
  a.params = p.params;
  a.w = static_cast<const VT*>(w);
  a.wrs = wrs;
  a.wcs = wcs;
  a.out = static_cast<VT*>(out);
  a.ors = ors;
  a.ocs = ocs;
  a.ytil = static_cast<VT*>(p.ytil);
  a.partial = p.partial;
  a.cta_rows = p.cta_rows;
  a.bar = GridBarrier{p.barrier};
  a.err = p.err;
  a.work = p.work;
  a.wait_ns = p.wait_ns;
  a.stall = p.stall_flag;
  const size_t base = operator_smem_bytes(p.threads, p.h, B, sizeof(VT) == 8 ? VecType::F64 : VecType::F32);
  const WindowTable& wt = p.win[B == 1 ? 0 : B == 2 ? 1 : 2];
  const bool windows = p.mode == 0 && wt.seg_row != nullptr && wt.win_rows > 0;
  a.seg_row = windows ? wt.seg_row : nullptr;
  a.seg_ws = windows ? wt.seg_ws : nullptr;
  a.cta_seg = windows ? wt.cta_seg : nullptr;
  a.win_rows = windows ? wt.win_rows : 0;
  a.win_off = (int)((base + 15) / 16 * 16);
  a.Fd = static_cast<const VT*>(p.Fd);
  a.fp = p.Fd ? p.h - 1 : 0;
  a.Kp = static_cast<const VT*>(p.Kp);
  a.kpad = (p.h + 3) & ~3;
  a.partial2 = p.partial2;
  const size_t smem = (size_t)a.win_off + (windows ? (size_t)wt.win_rows * B * sizeof(VT) : 0);
  auto kern = fused_operator_kernel<VT, MT, B>;
  check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "operator smem attr");
  void* args[] = {&a};
  check_cuda(cudaLaunchCooperativeKernel((void*)kern, dim3(p.grid), dim3(p.threads), args, smem, s),
             "operator cooperative launch");
}

template <typename VT, typename MT>
static void launch_b(const OpPlan& p, const void* w, int64_t wrs, int64_t wcs, void* out, int64_t ors, int64_t ocs,
                     int nvec, cudaStream_t s) {
  const size_t vs = sizeof(VT);
  int done = 0;
  while (done < nvec) {
    const int left = nvec - done;
    const char* wp = static_cast<const char*>(w) + (size_t)done * wcs * vs;
    char* op = static_cast<char*>(out) + (size_t)done * ocs * vs;
    if (left >= 4) {
      launch_t<VT, MT, 4>(p, wp, wrs, wcs, op, ors, ocs, s);
      done += 4;
    } else if (left >= 2) {
      launch_t<VT, MT, 2>(p, wp, wrs, wcs, op, ors, ocs, s);
      done += 2;
    } else {
      launch_t<VT, MT, 1>(p, wp, wrs, wcs, op, ors, ocs, s);
      done += 1;
    }
  }
}

void launch_operator(const OpPlan& p, VecType vt, const void* w, int64_t wrs, int64_t wcs, void* out, int64_t ors,
                     int64_t ocs, int nvec, cudaStream_t s) {
  if (vt == VecType::F64) {
    switch (p.val_dtype) {
      case SFAIRSC_F64: return launch_b<double, double>(p, w, wrs, wcs, out, ors, ocs, nvec, s);
      case SFAIRSC_F32: return launch_b<double, float>(p, w, wrs, wcs, out, ors, ocs, nvec, s);
      default: return launch_b<double, __nv_bfloat16>(p, w, wrs, wcs, out, ors, ocs, nvec, s);
    }
  } else {
    switch (p.val_dtype) {
      case SFAIRSC_F64: return launch_b<float, double>(p, w, wrs, wcs, out, ors, ocs, nvec, s);
      case SFAIRSC_F32: return launch_b<float, float>(p, w, wrs, wcs, out, ors, ocs, nvec, s);
      default: return launch_b<float, __nv_bfloat16>(p, w, wrs, wcs, out, ors, ocs, nvec, s);
    }
  }
}

template <typename VT, typename MT, int B>
static int max_grid_t(int threads, size_t smem) {
  auto kern = fused_operator_kernel<VT, MT, B>;
  check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "operator smem attr");
  int per_sm = 0;
  check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem), "operator occupancy");
  int dev = 0, sms = 0;
  check_cuda(cudaGetDevice(&dev), "get device");
  check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "sm count");
  return per_sm * sms;
}

int operator_max_grid(VecType vt, int val_dtype, int nvec, int threads, size_t smem) {
  // One CTA per SM (cooperative grid); the smallest co-resident grid over the instantiations.
  int best = 1 << 30;
  auto upd = [&](int g) { best = g < best ? g : best; };
  if (vt == VecType::F64) {
    switch (val_dtype) {
      case SFAIRSC_F64: upd(max_grid_t<double, double, 4>(threads, smem)); upd(max_grid_t<double, double, 1>(threads, smem)); break;
      case SFAIRSC_F32: upd(max_grid_t<double, float, 4>(threads, smem)); upd(max_grid_t<double, float, 1>(threads, smem)); break;
      default: upd(max_grid_t<double, __nv_bfloat16, 4>(threads, smem)); upd(max_grid_t<double, __nv_bfloat16, 1>(threads, smem)); break;
    }
  } else {
    switch (val_dtype) {
      case SFAIRSC_F64: upd(max_grid_t<float, double, 4>(threads, smem)); upd(max_grid_t<float, double, 1>(threads, smem)); break;
      case SFAIRSC_F32: upd(max_grid_t<float, float, 4>(threads, smem)); upd(max_grid_t<float, float, 1>(threads, smem)); break;
      default: upd(max_grid_t<float, __nv_bfloat16, 4>(threads, smem)); upd(max_grid_t<float, __nv_bfloat16, 1>(threads, smem)); break;
    }
  }
  (void)nvec;
  return best;
}

}  // namespace sfairsc

namespace sfairsc {

// ---------------------------------------------------------------- FP64-grade SpMV on the FP32 pipe
// t = L_n x for FP64 vectors x (b columns), with FP64-grade accuracy but FP32 arithmetic: the
// final residual check of the MIXED path applies the operator to Ritz vectors that already lie
// in null(C^T) (the FP64 projection just before), so A x = P (L_n x) and only the SpMV needs the
// precision.  GB300's FP64 rate would bound an FP64 SpMV; here every product and sum is carried
// as an unevaluated pair of floats (hi + lo) with the error-free transforms TwoSum (Knuth) and
// TwoProduct by FMA (Ogita, Rump and Oishi, 2005), about 2^-44 relative, far below the 1e-6
// residual it verifies.  ytil = D^{-1/2} x is formed in FP64 and stored as (hi, lo) float pairs.
namespace {

struct F2 {
  float hi, lo;
};

__device__ __forceinline__ F2 split_f64(double v) {
  const float hi = __double2float_rn(v);
  return F2{hi, __double2float_rn(v - (double)hi)};
}

// Sums and differences as fused multiply-adds with a multiplier of +-1 that the compiler cannot
// see (a kernel argument): a * 1 is exact, so fma(a, 1, b) rounds a + b once, bit for bit like an
// add, but issues on the FMA pipe (plain FP32 adds share a narrower pipe on this GPU).
struct FmaAdd {
  float one;
  __device__ __forceinline__ float add(float a, float b) const { return __fmaf_rn(a, one, b); }
  __device__ __forceinline__ float sub(float a, float b) const { return __fmaf_rn(b, -one, a); }
  // TwoSum (Knuth): s + e == a + b exactly
  __device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) const {
    s = add(a, b);
    const float bb = sub(s, a);
    e = add(sub(a, sub(s, bb)), sub(b, bb));
  }
};

// s += w * y (w = w_hi + w_lo, y = y.hi + y.lo), the pair renormalised
__device__ __forceinline__ void df_mac(const FmaAdd& f, F2& s, float w_hi, float w_lo, F2 y) {
  const float p = __fmul_rn(w_hi, y.hi);
  float pe = __fmaf_rn(w_hi, y.hi, -p);
  pe = __fmaf_rn(w_hi, y.lo, pe);
  pe = __fmaf_rn(w_lo, y.hi, pe);
  float t, e;
  f.two_sum(s.hi, p, t, e);
  e = f.add(e, f.add(s.lo, pe));
  s.hi = f.add(t, e);
  s.lo = f.sub(e, f.sub(s.hi, t));
}

__device__ __forceinline__ F2 df_add(const FmaAdd& f, F2 a, F2 b) {
  float t, e;
  f.two_sum(a.hi, b.hi, t, e);
  e = f.add(e, f.add(a.lo, b.lo));
  F2 r;
  r.hi = f.add(t, e);
  r.lo = f.sub(e, f.sub(r.hi, t));
  return r;
}

template <typename MT>
__device__ __forceinline__ void weight_split(MT v, float& hi, float& lo) {
  if constexpr (sizeof(MT) == 8) {
    hi = __double2float_rn((double)v);
    lo = __double2float_rn((double)v - (double)hi);
  } else {
    hi = val_as<float>(v);  // BF16 and FP32 weights are exact floats
    lo = 0.f;
  }
}

__global__ void df_ytil_kernel(int n, int b, const double* __restrict__ X, const double* __restrict__ dinv,
                               int normalized, F2* ytil) {
  const int64_t total = (int64_t)n * b;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / b, v = e % b;
    const double x = X[r + v * (int64_t)n];
    ytil[e] = split_f64(normalized ? dinv[r] * x : x);
  }
}

// Warp-per-row-group SpMV: Lr lanes per row, U pairs per lane per pass, row groups taken in turn
// by the warps of the grid.  T[:, v] = x_v - d^{-1/2} (W ytil)_v  (normalized), d x_v - W x_v (not).
template <typename MT, int B>
__global__ void __launch_bounds__(256) df_spmv_kernel(int n, const int32_t* __restrict__ row_ptr,
                                                      const int32_t* __restrict__ col, const MT* __restrict__ val,
                                                      const double* __restrict__ dinv,
                                                      const double* __restrict__ deg, int normalized, int Lr,
                                                      const double* __restrict__ X, const F2* __restrict__ ytil,
                                                      double* T, float one) {
  constexpr int U = 4;
  const FmaAdd fa{one};
  const int lane = threadIdx.x & 31;
  const int sub = lane & (Lr - 1);
  const int rpw = 32 / Lr;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  const int ngroups = (n + rpw - 1) / rpw;
  for (int q = gw; q < ngroups; q += nw) {
    const int r = q * rpw + lane / Lr;
    const bool live = r < n;
    const int e0 = live ? __ldg(row_ptr + r) : 0, e1 = live ? __ldg(row_ptr + r + 1) : 0;
    F2 acc[B];
#pragma unroll
    for (int v = 0; v < B; ++v) acc[v] = F2{0.f, 0.f};
    for (int e = e0 + sub; e < e1; e += U * Lr) {
      int c[U];
      float wh[U], wl[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int ee = e + u * Lr;
        const bool in = ee < e1;
        c[u] = in ? __ldg(col + ee) : -1;
        if (in) weight_split<MT>(val[ee], wh[u], wl[u]);
        else wh[u] = wl[u] = 0.f;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (c[u] >= 0) {
          F2 y[B];
          const F2* p = ytil + (size_t)c[u] * B;
          if constexpr (B % 2 == 0) {  // rows of B pairs, 16-byte aligned: two pairs per load
#pragma unroll
            for (int q = 0; q < B / 2; ++q) {
              const float4 a = __ldg(reinterpret_cast<const float4*>(p) + q);
              y[2 * q] = F2{a.x, a.y};
              y[2 * q + 1] = F2{a.z, a.w};
            }
          } else {
#pragma unroll
            for (int v = 0; v < B; ++v) y[v] = p[v];
          }
#pragma unroll
          for (int v = 0; v < B; ++v) df_mac(fa, acc[v], wh[u], wl[u], y[v]);
        }
      }
    }
    // pairs summed over the row's lanes by a fixed tree
    for (int o = Lr >> 1; o > 0; o >>= 1)
#pragma unroll
      for (int v = 0; v < B; ++v) {
        F2 other;
        other.hi = __shfl_xor_sync(0xffffffffu, acc[v].hi, o);
        other.lo = __shfl_xor_sync(0xffffffffu, acc[v].lo, o);
        acc[v] = df_add(fa, acc[v], other);
      }
    // every lane of the row holds its sums: lane sub of the row forms the columns sub, sub + Lr, ...
    // Each column's pair is picked by FP32 selects first, so a lane issues one FP64 epilogue per
    // column it owns: FP64 is a narrow pipe on this part, and FP64 instructions predicated off
    // still take their issue slots (one predicated epilogue per column and lane cost 2 ms a solve).
    if (live)
      for (int c0 = sub; c0 < B; c0 += Lr) {
        float hi = acc[0].hi, lo = acc[0].lo;
#pragma unroll
        for (int v = 1; v < B; ++v)
          if (c0 == v) {
            hi = acc[v].hi;
            lo = acc[v].lo;
          }
        const double s = (double)hi + (double)lo;
        const double x = X[(size_t)r + (size_t)c0 * n];
        T[(size_t)r + (size_t)c0 * n] = normalized ? x - dinv[r] * s : deg[r] * x - s;
      }
  }
}

template <typename MT>
void df_spmv_launch(int n, const int32_t* row_ptr, const int32_t* col, const void* val, const double* dinv,
                    const double* deg, int normalized, int Lr, const double* X, int b, F2* ytil, double* T, int sms,
                    cudaStream_t s) {
  df_ytil_kernel<<<4 * sms, 256, 0, s>>>(n, b, X, dinv, normalized, ytil);
  const MT* v = static_cast<const MT*>(val);
  const int grid = 8 * sms;
  switch (b) {
    case 8: df_spmv_kernel<MT, 8><<<grid, 256, 0, s>>>(n, row_ptr, col, v, dinv, deg, normalized, Lr, X, ytil, T, 1.f); break;
    case 4: df_spmv_kernel<MT, 4><<<grid, 256, 0, s>>>(n, row_ptr, col, v, dinv, deg, normalized, Lr, X, ytil, T, 1.f); break;
    case 3: df_spmv_kernel<MT, 3><<<grid, 256, 0, s>>>(n, row_ptr, col, v, dinv, deg, normalized, Lr, X, ytil, T, 1.f); break;
    case 2: df_spmv_kernel<MT, 2><<<grid, 256, 0, s>>>(n, row_ptr, col, v, dinv, deg, normalized, Lr, X, ytil, T, 1.f); break;
    default: df_spmv_kernel<MT, 1><<<grid, 256, 0, s>>>(n, row_ptr, col, v, dinv, deg, normalized, Lr, X, ytil, T, 1.f);
  }
}

}  // namespace

void launch_df_spmv(int n, const int32_t* row_ptr, const int32_t* col, const void* val, int val_dtype,
                    const double* dinv64, const double* deg, int normalized, int lanes, const double* X, int b,
                    void* ytil_pairs, double* T, int sms, cudaStream_t s) {
  if (b < 1 || (b > 4 && b != 8)) fail(SFAIRSC_ERR_INVALID_ARG, "df spmv block");
  F2* yt = static_cast<F2*>(ytil_pairs);
  switch (val_dtype) {
    case SFAIRSC_F64:
      df_spmv_launch<double>(n, row_ptr, col, val, dinv64, deg, normalized, lanes, X, b, yt, T, sms, s);
      break;
    case SFAIRSC_F32:
      df_spmv_launch<float>(n, row_ptr, col, val, dinv64, deg, normalized, lanes, X, b, yt, T, sms, s);
      break;
    default:
      df_spmv_launch<__nv_bfloat16>(n, row_ptr, col, val, dinv64, deg, normalized, lanes, X, b, yt, T, sms, s);
  }
  check_cuda(cudaGetLastError(), "df spmv launch");
}

}  // namespace sfairsc
