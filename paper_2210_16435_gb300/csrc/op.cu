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
};

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

// Adds x (one value per vector, per lane) into lane s's accumulators for the
// lanes whose label is s.  All 32 lanes must call it.  The warp sums run in
// the vector precision (FP64 arithmetic is 1/58 of FP32 on this part); the
// per-lane running sums are carried into FP64 by the caller.
template <int B, typename VT>
__device__ __forceinline__ void warp_group_add(const VT (&x)[B], int label, bool valid, int h, VT (&acc)[B]) {
  const int lane = threadIdx.x & 31;
  for (int s = 0; s < h; ++s) {
    const bool mine = valid && label == s;
    if (__ballot_sync(0xffffffffu, mine) == 0u) continue;
#pragma unroll
    for (int v = 0; v < B; ++v) {
      const VT t = warp_allsum(mine ? x[v] : VT(0));
      if (lane == s) acc[v] += t;
    }
  }
}

// Block reduction of the per-warp group accumulators (lane s holds group s)
// into partial[blockIdx.x][s * B + v], in a fixed warp order.
template <int B>
__device__ __forceinline__ void block_group_store(const double (&acc)[B], int h, double* red, double* partial) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int P = h * B;
  if (lane < h) {
#pragma unroll
    for (int v = 0; v < B; ++v) red[warp * P + lane * B + v] = acc[v];
  }
  __syncthreads();
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    double s = 0.0;
    for (int wv = 0; wv < nwarps; ++wv) s += red[wv * P + p];
    partial[(size_t)blockIdx.x * P + p] = s;
  }
  __syncthreads();
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
    for (int i = lo; i < hi; ++i) s += __ldcg(partial + (size_t)i * P + p);
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

// From the group sums tot[s*B+v] (s < h) of D^{-1/2} x, solve
// (C^T C) a = C^T x for every vector and return the per-group correction
// coef[s*B+v] = a'_s - z.a so that (C a)_i = d_i^{-1/2} coef[g_i].
// Also returns a itself (for the shift term).  Threads v < B work.
template <int B>
__device__ __forceinline__ void solve_groups(const double* tot, const double* params, int h, double* a_out,
                                             double* coef) {
  const int v = threadIdx.x;
  if (v < B) {
    const int p = h - 1;
    double sum = 0.0;
    for (int s = 0; s < h; ++s) sum += tot[s * B + v];
    double y[kMaxGroups];
    // forward: L y = rhs, rhs_s = tot_s - z_s * sum
    for (int s = 0; s < p; ++s) {
      double r = tot[s * B + v] - params[kPZ + s] * sum;
      for (int q = 0; q < s; ++q) r -= params[kPL + s * kLStride + q] * y[q];
      y[s] = r / params[kPL + s * kLStride + s];
    }
    // backward: L^T a = y
    for (int s = p - 1; s >= 0; --s) {
      double r = y[s];
      for (int q = s + 1; q < p; ++q) r -= params[kPL + q * kLStride + s] * y[q];
      y[s] = r / params[kPL + s * kLStride + s];
    }
    double za = 0.0;
    for (int s = 0; s < p; ++s) za += params[kPZ + s] * y[s];
    for (int s = 0; s < p; ++s) {
      a_out[s * B + v] = y[s];
      coef[s * B + v] = y[s] - za;
    }
    coef[p * B + v] = -za;
  }
  __syncthreads();
}

template <typename VT, typename MT, int B>
__global__ void __launch_bounds__(1024, 1) fused_operator_kernel(OpArgs<VT, MT> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int h = a.h;
  const int P = h * B;
  const bool grouped = h > 1;
  // shared layout
  VT* rows_s = reinterpret_cast<VT*>(smem_raw);                                     // nwarps * 32 * B
  double* red = reinterpret_cast<double*>(smem_raw + sizeof(VT) * nwarps * 32 * B);  // nwarps * P
  double* scratch = red + nwarps * P;                                                // blockDim.x (+P)
  double* tot = scratch + blockDim.x + P;                                            // P
  double* avec = tot + kMaxGroups * B;                                               // 32*B
  double* coefA = avec + kMaxGroups * B;                                             // 32*B
  double* coefD = coefA + kMaxGroups * B;                                            // 32*B
  int* rp_s = reinterpret_cast<int*>(coefD + kMaxGroups * B);                         // nwarps * 33

  const int r0 = a.cta_rows[blockIdx.x], r1 = a.cta_rows[blockIdx.x + 1];

  auto scale = [&](int r) -> VT { return a.normalized ? a.dinv[r] : VT(1); };

  // ---------------- phase A: group sums of D^{-1/2} w over own rows
  if (grouped) {
    double acc[B];
    VT accw[B];
#pragma unroll
    for (int v = 0; v < B; ++v) {
      acc[v] = 0.0;
      accw[v] = VT(0);
    }
    int nb = 0;
    for (int base = r0 + warp * 32; base < r1; base += nwarps * 32) {
      const int r = base + lane;
      const bool valid = r < r1;
      VT x[B];
      int g = 0;
      if (valid) {
        g = a.lab[r];
        const VT sc = scale(r);
#pragma unroll
        for (int v = 0; v < B; ++v) x[v] = a.w[r * a.wrs + v * a.wcs] * sc;
      } else {
#pragma unroll
        for (int v = 0; v < B; ++v) x[v] = VT(0);
      }
      warp_group_add<B>(x, g, valid, h, accw);
      if (++nb == 8) {
#pragma unroll
        for (int v = 0; v < B; ++v) {
          acc[v] += (double)accw[v];
          accw[v] = VT(0);
        }
        nb = 0;
      }
    }
#pragma unroll
    for (int v = 0; v < B; ++v) acc[v] += (double)accw[v];
    block_group_store<B>(acc, h, red, a.partial);
    if (!grid_sync(a.bar, a.err)) return;
    // ---------------- phase B: a = (C^T C)^{-1} C^T w
    reduce_partials(a.partial, gridDim.x, P, scratch, tot);
    solve_groups<B>(tot, a.params, h, avec, coefA);
  } else {
    for (int i = threadIdx.x; i < kMaxGroups * B; i += blockDim.x) {
      coefA[i] = 0.0;
      avec[i] = 0.0;
    }
    __syncthreads();
  }
  if (a.mode == 1) {  // P w only
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
      const int g = a.lab[r];
      const VT sc = scale(r);
#pragma unroll
      for (int v = 0; v < B; ++v) a.out[r * a.ors + v * a.ocs] = a.w[r * a.wrs + v * a.wcs] - sc * (VT)coefA[g * B + v];
    }
    return;
  }
#pragma unroll 4
  for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    const int g = a.lab[r];
    const VT sc = scale(r);
#pragma unroll
    for (int v = 0; v < B; ++v) {
      const VT y = a.w[r * a.wrs + v * a.wcs] - sc * (VT)coefA[g * B + v];
      a.ytil[(size_t)r * B + v] = a.normalized ? sc * y : y;
    }
  }
  if (!grid_sync(a.bar, a.err)) return;

  // ---------------- phase C: t = L_n y, written to out; group sums of D^{-1/2} t
  // Each warp sweeps the stored entries of a 32-row batch as one flat,
  // coalesced stream (entry e0 + 32u + lane), gathers ytil, and sums the
  // products per row with a segmented warp scan; the tail lane of every row
  // segment adds it to that row's shared-memory sum.  The summation tree is
  // fixed, so results are bitwise reproducible.
  double acc[B];
  VT accw[B];
#pragma unroll
  for (int v = 0; v < B; ++v) {
    acc[v] = 0.0;
    accw[v] = VT(0);
  }
  int nbc = 0;
  VT* myrows = rows_s + warp * 32 * B;
  int* rps = rp_s + warp * 33;
  constexpr int UCH = B >= 4 ? 2 : 4;  // 32-entry chunks per stage
  const int RB = a.batch_rows;          // rows per warp batch (1..32)
  for (int base = r0 + warp * RB; base < r1; base += nwarps * RB) {
    const int nr = min(RB, r1 - base);
    if (lane < nr) rps[lane] = __ldg(a.row_ptr + base + lane);
    if (lane == 0) rps[nr] = __ldg(a.row_ptr + base + nr);
#pragma unroll
    for (int v = 0; v < B; ++v) myrows[lane * B + v] = VT(0);
    __syncwarp();
    if constexpr (sizeof(VT) == 8) {
      // FP64 vectors: L lanes per row, one FMA per entry and log2(L) shuffle
      // levels per row (a flat scan would cost several FP64 adds per entry).
      const int L = a.lanes, sub = lane & (L - 1), per = 32 / L;
      for (int pass = 0; pass * per < nr; ++pass) {
        const int rib = pass * per + lane / L;
        VT sacc[B];
#pragma unroll
        for (int v = 0; v < B; ++v) sacc[v] = VT(0);
        if (rib < nr) {
          int e = rps[rib] + sub;
          const int e1 = rps[rib + 1];
          for (; e + L < e1; e += 2 * L) {
            const int c0 = __ldg(a.col + e), c1 = __ldg(a.col + e + L);
            const VT w0 = val_as<VT>(a.val[e]), w1 = val_as<VT>(a.val[e + L]);
            VT y0[B], y1[B];
            load_row<VT, B>(a.ytil + (size_t)c0 * B, y0);
            load_row<VT, B>(a.ytil + (size_t)c1 * B, y1);
#pragma unroll
            for (int v = 0; v < B; ++v) sacc[v] = fma(w1, y1[v], fma(w0, y0[v], sacc[v]));
          }
          if (e < e1) {
            const int c0 = __ldg(a.col + e);
            const VT w0 = val_as<VT>(a.val[e]);
            VT y0[B];
            load_row<VT, B>(a.ytil + (size_t)c0 * B, y0);
#pragma unroll
            for (int v = 0; v < B; ++v) sacc[v] = fma(w0, y0[v], sacc[v]);
          }
        }
        for (int o = L >> 1; o > 0; o >>= 1) {
#pragma unroll
          for (int v = 0; v < B; ++v) sacc[v] += __shfl_xor_sync(0xffffffffu, sacc[v], o);
        }
        if (sub == 0 && rib < nr) {
#pragma unroll
          for (int v = 0; v < B; ++v) myrows[rib * B + v] = sacc[v];
        }
      }
    } else {
      const int E0 = rps[0], E1 = rps[nr];
      int cur = 0;
      int cc[UCH];
      VT wv[UCH];
      auto fetch = [&](int e0, int (&c)[UCH], VT (&w)[UCH]) {
  #pragma unroll
        for (int u = 0; u < UCH; ++u) {
          const int e = e0 + 32 * u + lane;
          const bool ok = e < E1;
          c[u] = ok ? __ldg(a.col + e) : 0;
          w[u] = ok ? val_as<VT>(a.val[e]) : VT(0);
        }
      };
      fetch(E0, cc, wv);
      for (int e0 = E0; e0 < E1; e0 += 32 * UCH) {
        VT y[UCH][B];
  #pragma unroll
        for (int u = 0; u < UCH; ++u) load_row<VT, B>(a.ytil + (size_t)cc[u] * B, y[u]);
        int ncc[UCH];
        VT nwv[UCH];
        fetch(e0 + 32 * UCH, ncc, nwv);  // next stage's indices and weights, in flight during this one
  #pragma unroll
        for (int u = 0; u < UCH; ++u) {
          const int e = e0 + 32 * u + lane;
          const bool ok = e < E1;
          if (ok)
            while (e >= rps[cur + 1]) ++cur;
          const int rid = ok ? cur : 32;
          VT p[B];
  #pragma unroll
          for (int v = 0; v < B; ++v) p[v] = wv[u] * y[u][v];
  #pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int ro = __shfl_up_sync(0xffffffffu, rid, o);
  #pragma unroll
            for (int v = 0; v < B; ++v) {
              const VT t = __shfl_up_sync(0xffffffffu, p[v], o);
              if (lane >= o && ro == rid) p[v] += t;
            }
          }
          const int rn = __shfl_down_sync(0xffffffffu, rid, 1);
          if (ok && (lane == 31 || rn != rid)) {
  #pragma unroll
            for (int v = 0; v < B; ++v) myrows[rid * B + v] += p[v];
          }
          __syncwarp();
        }
  #pragma unroll
        for (int u = 0; u < UCH; ++u) {
          cc[u] = ncc[u];
          wv[u] = nwv[u];
        }
      }
    }
    __syncwarp();
    const int r = base + lane;
    const bool valid = lane < nr;
    VT x[B];
    int g = 0;
    if (valid) {
      g = a.lab[r];
      const VT sc = scale(r);
      const VT dd = a.normalized ? VT(1) : (VT)a.deg[r];
#pragma unroll
      for (int v = 0; v < B; ++v) {
        const VT y = a.w[r * a.wrs + v * a.wcs] - sc * (VT)coefA[g * B + v];
        const VT t = a.normalized ? y - sc * myrows[lane * B + v] : dd * y - myrows[lane * B + v];
        a.out[r * a.ors + v * a.ocs] = t;
        x[v] = sc * t;
      }
    } else {
#pragma unroll
      for (int v = 0; v < B; ++v) x[v] = VT(0);
    }
    __syncwarp();
    if (grouped) {
      warp_group_add<B>(x, g, valid, h, accw);
      if (++nbc == 8) {
#pragma unroll
        for (int v = 0; v < B; ++v) {
          acc[v] += (double)accw[v];
          accw[v] = VT(0);
        }
        nbc = 0;
      }
    }
  }
  if (!grouped) return;
#pragma unroll
  for (int v = 0; v < B; ++v) acc[v] += (double)accw[v];
  block_group_store<B>(acc, h, red, a.partial);
  if (!grid_sync(a.bar, a.err)) return;

  // ---------------- phase D: b = (C^T C)^{-1} C^T t; out = t - C (b - sigma a)
  reduce_partials(a.partial, gridDim.x, P, scratch, tot);
  {
    // reuse solve_groups on tot, then fold in -sigma a
    double* bvec = scratch;  // scratch is free now (reduce_partials synced)
    solve_groups<B>(tot, a.params, h, bvec, coefD);
    const double sigma = a.params[kPSigma];
    if (threadIdx.x < B) {
      const int v = threadIdx.x;
      const int p = h - 1;
      double zu = 0.0;
      for (int s = 0; s < p; ++s) {
        const double u = bvec[s * B + v] - sigma * avec[s * B + v];
        zu += a.params[kPZ + s] * u;
        coefD[s * B + v] = u;
      }
      for (int s = 0; s < p; ++s) coefD[s * B + v] -= zu;
      coefD[p * B + v] = -zu;
    }
    __syncthreads();
  }
#pragma unroll 4
  for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    const int g = a.lab[r];
    const VT sc = scale(r);
#pragma unroll
    for (int v = 0; v < B; ++v) a.out[r * a.ors + v * a.ocs] -= sc * (VT)coefD[g * B + v];
  }
}

size_t operator_smem_bytes(int threads, int h, int nvec, VecType vt) {
  const int nwarps = threads / 32;
  const size_t vs = vt == VecType::F64 ? 8 : 4;
  const int P = h * nvec;
  return vs * nwarps * 32 * nvec + sizeof(double) * ((size_t)nwarps * P + threads + P + 4 * kMaxGroups * nvec) +
         sizeof(int) * nwarps * 33 + 64;
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
  a.bar = GridBarrier{p.barrier, p.barrier + 1};
  a.err = p.err;
  const size_t smem = operator_smem_bytes(p.threads, p.h, B, sizeof(VT) == 8 ? VecType::F64 : VecType::F32);
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
  // Occupancy is limited by the 1024-thread CTA; every instantiation fits one CTA per SM.
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
