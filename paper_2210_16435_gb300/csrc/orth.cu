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
// row-major array), so consecutive rows of a panel are one contiguous run.
// A sweep streams the CTA's rows as slices of SR rows of every panel and of
// U: each warp copies its next slice into its own shared-memory buffer with
// cp.async while it works on the current one (no CTA barrier inside a sweep),
// and treats each slice in two phases:
//   phase A, LPA lanes per row: subtract V c from the row of U (coefficients
//     broadcast from shared memory), store it, add its Gram entries;
//   phase B, LPR lanes per row, lane p holding panel p: add the rows'
//     products to the new coefficients V^T u.
// Both phases read the panels from the slice, so V leaves HBM once per sweep.
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
  // the (sum, carry) pair packed into 8 bytes, to be combined by slot_sum
  // without FP64 arithmetic in every lane (after reduce)
  __device__ __forceinline__ double slot() const { return k.slot(); }
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
  __device__ __forceinline__ double slot() const { return w; }
};

// Sum of n slots p[0], p[stride], ... written by Acc::slot(): FP32 (sum,
// carry) pairs are added by TwoSum and converted to FP64 once; FP64 slots
// are added in FP64.  Fixed order.
template <typename VT>
__device__ __forceinline__ double slot_sum(const double* p, int n, int stride) {
  if constexpr (sizeof(VT) == 4) {
    return comp32_slot_sum(p, n, stride);
  } else {
    double t = 0.0;
    for (int i = 0; i < n; ++i) t += p[(size_t)i * stride];
    return t;
  }
}

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

// 4 * B consecutive coefficients (a panel's columns times the block's vectors) from shared
// memory in 16-byte pieces (the array starts 16-byte aligned and 4 * B * sizeof(VT) is a
// multiple of 16).
template <typename VT, int B>
__device__ __forceinline__ void ld_coefs(const VT* p, VT (&c)[4 * B]) {
  if constexpr (sizeof(VT) == 4) {
#pragma unroll
    for (int q = 0; q < B; ++q) {
      const float4 v = reinterpret_cast<const float4*>(p)[q];
      c[4 * q] = v.x;
      c[4 * q + 1] = v.y;
      c[4 * q + 2] = v.z;
      c[4 * q + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < 2 * B; ++q) {
      const double2 v = reinterpret_cast<const double2*>(p)[q];
      c[2 * q] = v.x;
      c[2 * q + 1] = v.y;
    }
  }
}

__device__ __forceinline__ int lanes_for(int np) {
  return np <= 1 ? 1 : np <= 2 ? 2 : np <= 4 ? 4 : np <= 8 ? 8 : np <= 16 ? 16 : 32;
}

// Fixed-order sums over the rows of the partials (row i, one per CTA, starts
// at partial + i * stride).
// The rows are cut into nch contiguous chunks, each summed by its own thread
// with several loads in flight, and the chunk sums are added in a fixed
// pairwise tree in shared memory.  The shape depends only on the row count
// and the number of values, so every CTA that forms a value forms the same bits.
__device__ __forceinline__ int chunk_count(int per_row) {
  int nch = 1;
  while (nch < 256 && 2 * nch * per_row <= kOT) nch *= 2;
  return nch;
}

// Pairwise tree over the nch chunk sums held at scratch[(c * cnt + q) * w + e]
// (c < nch, q < cnt, e < w); leaves the totals in chunk 0.  Every thread of
// the CTA calls it.
__device__ __forceinline__ void chunk_tree(double* scratch, int nch, int cnt, int w) {
  const int t = threadIdx.x, q = t % cnt, c = t / cnt;
  __syncthreads();
  for (int h = nch >> 1; h >= 1; h >>= 1) {
    if (c < h)
      for (int e = 0; e < w; ++e) scratch[(c * cnt + q) * w + e] += scratch[((c + h) * cnt + q) * w + e];
    __syncthreads();
  }
}

// CTA b owns coefficients p = b, b + grid, ...; writes out[p] = sum over rows
// i < nrows of partial[i][p].  Ends with __syncthreads.
__device__ __forceinline__ void reduce_owned(const double* partial, int stride, int nrows, int P, double* out,
                                             double* scratch) {
  const int nct = gridDim.x;
  const int Q = P > (int)blockIdx.x ? (P - (int)blockIdx.x + nct - 1) / nct : 0;
  if (Q == 0) {
    __syncthreads();
    return;
  }
  const int nch = chunk_count(Q);
  const int t = threadIdx.x, q = t % Q, c = t / Q;
  if (c < nch) {
    const int lo = (int)((long long)c * nrows / nch), hi = (int)((long long)(c + 1) * nrows / nch);
    const double* src = partial + blockIdx.x + (size_t)q * nct;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    int i = lo;
    for (; i + 4 <= hi; i += 4) {
      double x[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) x[e] = __ldcg(src + (size_t)(i + e) * stride);
#pragma unroll
      for (int e = 0; e < 4; ++e) s[e] += x[e];
    }
    for (; i < hi; ++i) s[0] += __ldcg(src + (size_t)i * stride);
    scratch[c * Q + q] = (s[0] + s[1]) + (s[2] + s[3]);
  }
  chunk_tree(scratch, nch, Q, 1);
  if (t < Q) out[blockIdx.x + t * nct] = scratch[t];
  __syncthreads();
}

// All CTAs: out[t] = sum over rows i < nrows of partial[i][off + t], t < cnt
// (cnt <= 16; off even).  Ends with __syncthreads.
__device__ __forceinline__ void reduce_all(const double* partial, int stride, int nrows, int off, int cnt, double* out,
                                           double* scratch) {
  const int w = (cnt & 1) ? 1 : 2;  // values per load
  const int nl = cnt / w;           // loads per row
  const int nch = chunk_count(nl);
  const int t = threadIdx.x, q = t % nl, c = t / nl;
  if (c < nch) {
    const int lo = (int)((long long)c * nrows / nch), hi = (int)((long long)(c + 1) * nrows / nch);
    double s[4][2] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
    if (w == 2) {
      const double2* src = reinterpret_cast<const double2*>(partial + off) + q;
      const int st2 = stride / 2;
      int i = lo;
      for (; i + 4 <= hi; i += 4) {
        double2 x[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) x[e] = __ldcg(src + (size_t)(i + e) * st2);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          s[e][0] += x[e].x;
          s[e][1] += x[e].y;
        }
      }
      for (; i < hi; ++i) {
        const double2 x = __ldcg(src + (size_t)i * st2);
        s[0][0] += x.x;
        s[0][1] += x.y;
      }
    } else {
      const double* src = partial + off + q;
      int i = lo;
      for (; i + 4 <= hi; i += 4) {
        double x[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) x[e] = __ldcg(src + (size_t)(i + e) * stride);
#pragma unroll
        for (int e = 0; e < 4; ++e) s[e][0] += x[e];
      }
      for (; i < hi; ++i) s[0][0] += __ldcg(src + (size_t)i * stride);
    }
    for (int e = 0; e < w; ++e) scratch[(c * nl + q) * w + e] = (s[0][e] + s[1][e]) + (s[2][e] + s[3][e]);
  }
  chunk_tree(scratch, nch, nl, w);
  if (t < nl)
    for (int e = 0; e < w; ++e) out[t * w + e] = scratch[t * w + e];
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
  unsigned long long wait_ns;  // bound of every grid-barrier wait
  // deferred second projection: pend_in (j x B, nullable) is the pending correction of the
  // input block V[:, j:j+B] against V[:, 0:j]; with defer the new block is stored without its
  // second projection, whose correction (J x B) goes to pend_out
  const double* pend_in;
  double* pend_out;
  int defer;
};

// Sweep slices: SR consecutive rows of every panel V[:, 4p:4p+4] (p < np)
// and of U, copied by the warp that will use them into its own shared-memory
// buffer with cp.async (16 bytes per lane, zero fill past the CTA's rows),
// two buffers per warp so the next slice is in flight while one is used.  A
// slice is row-major: row i holds the row's np panel entries and then its row
// of U, rsc 16-byte chunks apart, rsc padded so that the lanes of a quarter
// warp reading different rows fall in different banks.
constexpr int kWarpBuf = 13312;  // bytes of slice buffer per warp (two slices)
// the fixed slice geometry: 16 rows, 26 chunks per row (row stride = 2 mod 8 chunks, so the two
// lanes of each of four consecutive rows in phase A hit distinct bank groups), up to 25 panels + U
constexpr int kFSR = 16, kFRSC = 26, kFNP = kFRSC - 1, kFSB = kFSR * kFRSC * 16;
static_assert(2 * kFSB <= kWarpBuf, "two fixed-shape slices fit in a warp's buffer");
// phase B reads at most chunk kFNP of row 15 of the second slice (lanes past the last panel read chunk 0)
static_assert(kFSB + (15 * kFRSC + kFNP + 1) * 16 <= kWarpBuf, "phase B reads stay inside the warp's buffer");

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned n = valid ? 16u : 0u;  // src-size 0 fills the 16 bytes with zeros
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(smem)), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Slice geometry for np panels: rows per slice, lanes per row in phase A, and
// the row stride in 16-byte chunks.
struct SliceShape {
  int sr, lpa, rsc;
};
template <typename VT>
__host__ __device__ inline SliceShape slice_shape(int np) {
  constexpr int ch = (int)sizeof(VT) / 4;  // 16-byte chunks per panel row
  for (int sr = 16; sr >= 2; sr >>= 1) {
    const int lpa = 32 / sr;
    int rsc = (np + 1) * ch;
    if (ch == 1)
      while ((rsc & 7) != (lpa & 7)) ++rsc;
    else
      rsc |= 1;
    if (2 * sr * rsc * 16 <= kWarpBuf) return SliceShape{sr, lpa, rsc};
  }
  return SliceShape{0, 0, 0};
}

// Shared memory: the slice buffers (kOW x kWarpBuf; between sweeps the
// per-warp partials, kOW x red_stride doubles, reuse them), the coefficients
// (kCoefMax VT) and the reduction scratch (1024 doubles).
template <typename VT, int NC>
constexpr size_t orth_smem_bytes() {
  return (size_t)kOW * kWarpBuf + sizeof(VT) * kCoefMax + sizeof(double) * 1024 + 128;
}
static_assert(sizeof(double) * kOW * (1024 + 16) <= (size_t)kOW * kWarpBuf, "per-warp partials fit in the slice buffers");

template <typename VT, int B, int NC>
__global__ void __launch_bounds__(kOT, 1) orth_kernel(OrthArgs<VT> a) {
  extern __shared__ __align__(128) unsigned char smraw[];
  constexpr int kRed = red_stride<NC>();
  constexpr int kXo = kRed - 16;                                                      // extras offset
  double* red = reinterpret_cast<double*>(smraw);                                     // kOW x kRed, between sweeps
  VT* cfs = reinterpret_cast<VT*>(smraw + (size_t)kOW * kWarpBuf);                    // coefficients c*B + v
  double* scratch = reinterpret_cast<double*>(smraw + (size_t)kOW * kWarpBuf + sizeof(VT) * kCoefMax);
  __shared__ double gram_s[16], R1[16], R2[16], Rd1[16], Rd2[16], unorm[4], Rdi1[4], Rdi2[4];
  __shared__ int brk, again;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r0 = a.cta_rows[blockIdx.x], r1 = a.cta_rows[blockIdx.x + 1];
  const int J = a.J, P = J * B;
  const int np = (J + 3) / 4;  // panels holding columns 0..J-1
  const size_t pn = (size_t)a.n * 4;
  constexpr int NG = B * (B + 1) / 2;  // unique Gram entries
  constexpr int NA = NG > B ? NG : B;
  VT* U = a.U;
  unsigned char* wbuf = smraw + (size_t)warp * kWarpBuf;  // this warp's two slices
  if (threadIdx.x == 0) brk = 0;
  __syncthreads();

  // Slice loop with a fixed geometry, for FP32 blocks of 4 against at most kFNP panels (the
  // common case: a basis of up to 100 columns).  Slices of kFSR = 16 rows, a row stride of
  // kFRSC = 26 chunks, two lanes per row in phase A and one panel per lane in phase B, all
  // compile-time, so every shared-memory offset inside a slice is an immediate.  The same
  // arithmetic in the same order as the general loop.  Lanes whose panel is past np in phase B
  // accumulate whatever their chunk holds; their sums are never written out.
  auto fixed_shape = [&](int npp) { return sizeof(VT) == 4 && B == 4 && NC == 1 && npp <= kFNP; };
  auto fixed_slices = [&](int kind, bool fix, int Jd, int npp, Acc<VT> (&ac)[4][B], Acc<VT> (&gacc)[NA]) {
   if constexpr (sizeof(VT) == 4 && B == 4 && NC == 1) {
    const bool upd = kind >= 1, want_c = kind <= 1;
    const int nsl = (r1 - r0 + kFSR - 1) / kFSR;
    const int npd = Jd >> 2;                     // panels of the row update (Jd % 4 == 0: blocks of 4)
    const int pt = fix ? (a.j >> 2) : 0;         // the input block's panel
    auto fetch_f = [&](int k) {
      const int sl = warp + kOW * k;
      if (sl < nsl) {
        const int rb = r0 + sl * kFSR;
        const int i = lane & (kFSR - 1);
        const bool valid = rb + i < r1;
        const size_t roff = (size_t)(valid ? rb + i : r0) * 4;
        int c = lane >> 4;
        unsigned char* d = wbuf + (k & 1) * kFSB + (i * kFRSC + c) * 16;
        const VT* src = a.V + (size_t)c * pn + roff;
        for (; c < npp; c += 2, d += 32, src += 2 * pn) cp_async16(d, src, valid);
        if (c == npp) cp_async16(d, U + roff, valid);
      }
      cp_async_commit();
    };
    const int ia = lane >> 1, g = lane & 1;  // phase A: row, panel parity
    fetch_f(0);
    for (int k = 0; warp + kOW * k < nsl; ++k) {
      fetch_f(k + 1);
      cp_async_wait<1>();
      __syncwarp();
      const int rb = r0 + (warp + kOW * k) * kFSR;
      const int rows = min(kFSR, r1 - rb);
      unsigned char* sb = wbuf + (k & 1) * kFSB;
      // ---- phase A: d = V[row, 0:Jd] c over this lane's panels g, g + 2, ...; the pair of lanes adds
      float d[4] = {0.f, 0.f, 0.f, 0.f};
      if (npd > 0) {
        float d1[4] = {0.f, 0.f, 0.f, 0.f};
        const unsigned char* xa = sb + (ia * kFRSC + g) * 16;
        const float* ca = reinterpret_cast<const float*>(cfs) + g * 16;
        int pp = g;
        for (; pp + 2 < npd; pp += 4, xa += 64, ca += 64) {
          float x0[4], x1[4], c0[16], c1[16];
          ld4(reinterpret_cast<const float*>(xa), x0);
          ld4(reinterpret_cast<const float*>(xa + 32), x1);
          ld_coefs<float, 4>(ca, c0);
          ld_coefs<float, 4>(ca + 32, c1);
#pragma unroll
          for (int jj = 0; jj < 4; ++jj)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
              d[v] = fmaf(x0[jj], c0[jj * 4 + v], d[v]);
              d1[v] = fmaf(x1[jj], c1[jj * 4 + v], d1[v]);
            }
        }
        if (pp < npd) {
          float x0[4], c0[16];
          ld4(reinterpret_cast<const float*>(xa), x0);
          ld_coefs<float, 4>(ca, c0);
#pragma unroll
          for (int jj = 0; jj < 4; ++jj)
#pragma unroll
            for (int v = 0; v < 4; ++v) d[v] = fmaf(x0[jj], c0[jj * 4 + v], d[v]);
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          d[v] += d1[v];
          d[v] += __shfl_xor_sync(0xffffffffu, d[v], 1);
        }
      }
      if (g == 0 && ia < rows) {
        if (fix) {  // the input block's row (panel pt, J % 4 == 0), corrected in the slice and in V
          float* xp = reinterpret_cast<float*>(sb + (ia * kFRSC + pt) * 16);
          float x[4];
          ld4(xp, x);
#pragma unroll
          for (int v = 0; v < 4; ++v) x[v] -= d[v];
          st4(xp, x);
          st4(a.V + (size_t)pt * pn + (size_t)(rb + ia) * 4, x);
        }
        float* up = reinterpret_cast<float*>(sb + (ia * kFRSC + npp) * 16);
        float u[4];
        ld4(up, u);
        if (upd) {
#pragma unroll
          for (int v = 0; v < 4; ++v) u[v] -= d[v];
          st4(up, u);
          st4(U + (size_t)(rb + ia) * 4, u);
        }
        if (kind == 0) {
#pragma unroll
          for (int v = 0; v < 4; ++v) gacc[v].fma_(u[v], u[v]);
        } else {
          int e = 0;
#pragma unroll
          for (int v = 0; v < 4; ++v)
#pragma unroll
            for (int w2 = v; w2 < 4; ++w2) gacc[e++].fma_(u[v], u[w2]);
        }
      }
      __syncwarp();
      // ---- phase B: lane p (16 or 32 lanes per row) adds V[row, 4p:4p+4]^T u[row] over the slice
      if (want_c) {
        auto rowb = [&](const unsigned char* xb, const unsigned char* ub) {
          float x[4], u[4];
          ld4(reinterpret_cast<const float*>(xb), x);
          ld4(reinterpret_cast<const float*>(ub), u);
#pragma unroll
          for (int jj = 0; jj < 4; ++jj)
#pragma unroll
            for (int v = 0; v < 4; ++v) ac[jj][v].fma_(x[jj], u[v]);
        };
        if (npp > 16) {
          const unsigned char* xb = sb + (lane < npp ? lane : 0) * 16;
          const unsigned char* ub = sb + npp * 16;
#pragma unroll
          for (int i = 0; i < kFSR; ++i) rowb(xb + i * kFRSC * 16, ub + i * kFRSC * 16);
        } else {
          const int r2 = lane >> 4;
          const unsigned char* xb = sb + (r2 * kFRSC + ((lane & 15) < npp ? (lane & 15) : 0)) * 16;
          const unsigned char* ub = sb + (r2 * kFRSC + npp) * 16;
#pragma unroll
          for (int i = 0; i < kFSR; i += 2) rowb(xb + i * kFRSC * 16, ub + i * kFRSC * 16);
        }
      }
      if ((k & 3) == 3) {
#pragma unroll
        for (int jj = 0; jj < 4; ++jj)
#pragma unroll
          for (int v = 0; v < 4; ++v) ac[jj][v].flush();
#pragma unroll
        for (int e = 0; e < NA; ++e) gacc[e].flush();
      }
      __syncwarp();  // the buffer is free for slice k + 2
    }
   }
  };

  // sweep kinds: 0 = coefficients + input norms; 1 = update with a.coef, then the
  // next coefficients and the Gram matrix; 2 = update with a.coef, then the Gram matrix.
  // A warp takes the slices r0 + (warp + kOW k) SR, each in two phases:
  //   phase A, LPA lanes per row, lane g summing panels g, g + LPA, ...:
  //     u <- u - V c, written back to the slice and to U, Gram entries;
  //   phase B, LPR lanes per row, lane p0 (+32 q) holding panel p0 (+32 q):
  //     the new coefficients V^T u.
  auto sweep = [&](int kind) -> bool {
    const bool upd = kind >= 1, want_c = kind <= 1;
    // kind 0 with a pending correction first finishes the input block: V[:, j:j+B] -= V[:, 0:j] e
    const bool fix = kind == 0 && a.pend_in != nullptr;
    const int Jd = upd ? J : (fix ? a.j : 0);  // columns of the row update V[:, 0:Jd] c
    if (upd)
      for (int i = threadIdx.x; i < P; i += blockDim.x) cfs[i] = (VT)__ldcg(a.coef + i);
    else if (fix)
      for (int i = threadIdx.x; i < a.j * B; i += blockDim.x) cfs[i] = (VT)__ldcg(a.pend_in + i);
    __syncthreads();  // coefficients in place; the slice buffers are free
    constexpr int CH = (int)sizeof(VT) / 4;
    const SliceShape sh = slice_shape<VT>(np);
    const int SR = sh.sr, LPA = sh.lpa, rsc = sh.rsc;
    const int lsr = 31 - __clz(SR);  // SR is a power of two
    const int sbytes = SR * rsc * 16;  // one slice
    // phase B lanes per row: one per panel (the fixed shape: 16 or 32)
    const int LPR = fixed_shape(np) ? (np > 16 ? 32 : 16) : NC == 1 ? lanes_for(np) : 32;
    const int RPW = 32 / LPR;
    const int p0 = lane & (LPR - 1), ri = lane / LPR;
    const int nsl = (r1 - r0 + SR - 1) / SR;  // slices of this CTA
    const int ncols = (np + 1) * CH;          // chunks per row to copy
    // copy slice k of this warp into buffer k & 1 (one commit group, possibly empty)
    auto fetch = [&](int k) {
      const int sl = warp + kOW * k;
      if (sl < nsl) {
        const int rb = r0 + sl * SR;
        unsigned char* dst = wbuf + (k & 1) * sbytes;
        // lane: row i, chunks c0, c0 + 32 / SR, ... (lanes run down a column: coalesced rows)
        const int i = lane & (SR - 1);
        const bool valid = rb + i < r1;
        const size_t roff = (size_t)(valid ? rb + i : r0) * 4;
        unsigned char* d = dst + (size_t)i * rsc * 16;
        for (int c = lane >> lsr; c < ncols; c += 32 >> lsr) {
          const int col = CH == 1 ? c : c >> 1;
          const VT* base = col < np ? a.V + (size_t)col * pn : U;
          cp_async16(d + c * 16, base + roff + (CH == 1 ? 0 : (c & 1) * 2), valid);
        }
      }
      cp_async_commit();
    };
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
    if (fixed_shape(np)) {
      if constexpr (sizeof(VT) == 4 && B == 4 && NC == 1)
        fixed_slices(kind, fix, Jd, np, acc[0], ga);
    } else {
    fetch(0);
    for (int k = 0; warp + kOW * k < nsl; ++k) {
      fetch(k + 1);
      cp_async_wait<1>();
      __syncwarp();
      const int rb = r0 + (warp + kOW * k) * SR;
      const int rows = min(SR, r1 - rb);
      const unsigned char* sl = wbuf + (k & 1) * sbytes;
      auto at = [&](int i, int col) { return reinterpret_cast<const VT*>(sl + ((size_t)i * rsc + col * CH) * 16); };
      // ---- phase A
      {
        const int i = lane / LPA, g = lane & (LPA - 1);
        VT d[B];
#pragma unroll
        for (int v = 0; v < B; ++v) d[v] = VT(0);
        if (Jd > 0) {
          const int nfull = Jd >> 2;  // panels whose 4 columns are all < Jd
          VT d1[B];  // a second set of chains: two panels' loads in flight per step
#pragma unroll
          for (int v = 0; v < B; ++v) d1[v] = VT(0);
          int pp = g;
          for (; pp + LPA < nfull; pp += 2 * LPA) {
            VT x0[4], x1[4], c0[4 * B], c1[4 * B];
            ld4(at(i, pp), x0);
            ld4(at(i, pp + LPA), x1);
            ld_coefs<VT, B>(cfs + 4 * pp * B, c0);  // a panel's 4 x B coefficients: 16-byte loads
            ld_coefs<VT, B>(cfs + 4 * (pp + LPA) * B, c1);
#pragma unroll
            for (int jj = 0; jj < 4; ++jj)
#pragma unroll
              for (int v = 0; v < B; ++v) {
                d[v] = fma(x0[jj], c0[jj * B + v], d[v]);
                d1[v] = fma(x1[jj], c1[jj * B + v], d1[v]);
              }
          }
          if (pp < nfull) {
            VT x[4], c0[4 * B];
            ld4(at(i, pp), x);
            ld_coefs<VT, B>(cfs + 4 * pp * B, c0);
#pragma unroll
            for (int jj = 0; jj < 4; ++jj)
#pragma unroll
              for (int v = 0; v < B; ++v) d[v] = fma(x[jj], c0[jj * B + v], d[v]);
          }
          if (nfull < np && (nfull & (LPA - 1)) == g) {
            VT x[4];
            ld4(at(i, nfull), x);
            for (int jj = 0; jj < (Jd & 3); ++jj)
#pragma unroll
              for (int v = 0; v < B; ++v) d1[v] = fma(x[jj], cfs[(4 * nfull + jj) * B + v], d1[v]);
          }
#pragma unroll
          for (int v = 0; v < B; ++v) d[v] += d1[v];
          for (int o = 1; o < LPA; o <<= 1)
#pragma unroll
            for (int v = 0; v < B; ++v) d[v] += __shfl_xor_sync(0xffffffffu, d[v], o);
        }
        if (g == 0 && i < rows) {
          if (fix) {  // the input block's row, corrected in the slice (for phase B) and in V
            const int pt = a.j >> 2, c0 = a.j & 3;
            VT x[4];
            ld4(at(i, pt), x);
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
              for (int v = 0; v < B; ++v)
                if (q == c0 + v) x[q] -= d[v];
            st4(const_cast<VT*>(at(i, pt)), x);
            st4(a.V + (size_t)pt * pn + (size_t)(rb + i) * 4, x);
          }
          VT u[4];
          ld4(at(i, np), u);
          if (upd) {
#pragma unroll
            for (int v = 0; v < B; ++v) u[v] -= d[v];
            st4(const_cast<VT*>(at(i, np)), u);
            st4(U + (size_t)(rb + i) * 4, u);
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
        }
      }
      __syncwarp();
      // ---- phase B (rows past the CTA's end are zero in the slice)
      if (want_c) {
        for (int s0 = 0; s0 < SR; s0 += 2 * RPW) {
          VT xs[2][NC][4], us[2][4];
#pragma unroll
          for (int tt = 0; tt < 2; ++tt) {
            const int i = s0 + ri + RPW * tt;
            const bool in = i < SR;
            if (in) ld4(at(i, np), us[tt]);
            else us[tt][0] = us[tt][1] = us[tt][2] = us[tt][3] = VT(0);
#pragma unroll
            for (int q = 0; q < NC; ++q) {
              const int pp = p0 + 32 * q;
              if (in && pp < np) {
                ld4(at(i, pp), xs[tt][q]);
                if (4 * pp + 4 > J)
#pragma unroll
                  for (int jj = 0; jj < 4; ++jj)
                    if (4 * pp + jj >= J) xs[tt][q][jj] = VT(0);
              } else {
                xs[tt][q][0] = xs[tt][q][1] = xs[tt][q][2] = xs[tt][q][3] = VT(0);
              }
            }
          }
#pragma unroll
          for (int tt = 0; tt < 2; ++tt)
#pragma unroll
            for (int q = 0; q < NC; ++q)
#pragma unroll
              for (int jj = 0; jj < 4; ++jj)
#pragma unroll
                for (int v = 0; v < B; ++v) acc[q][jj][v].fma_(xs[tt][q][jj], us[tt][v]);
        }
      }
      if ((k & 3) == 3) {
#pragma unroll
        for (int q = 0; q < NC; ++q)
#pragma unroll
          for (int jj = 0; jj < 4; ++jj)
#pragma unroll
            for (int v = 0; v < B; ++v) acc[q][jj][v].flush();
#pragma unroll
        for (int e = 0; e < NA; ++e) ga[e].flush();
      }
      __syncwarp();  // the buffer is free for slice k + 2
    }
    }
    cp_async_wait<0>();
    __syncthreads();  // every warp is done with its slices: the buffers take the partials
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
              for (int v = 0; v < B; ++v) rw[(4 * pp + jj) * B + v] = acc[q][jj][v].slot();
      }
    if (lane == 0) {
      if (kind == 0) {
#pragma unroll
        for (int v = 0; v < B; ++v) rw[kXo + v] = ga[v].slot();
      } else {
        int e = 0;
#pragma unroll
        for (int v = 0; v < B; ++v)
#pragma unroll
          for (int w2 = v; w2 < B; ++w2) {
            const double g = ga[e++].slot();
            rw[kXo + v * B + w2] = g;
            rw[kXo + w2 * B + v] = g;
          }
      }
    }
    __syncthreads();
    if (want_c)
      for (int i = threadIdx.x; i < P; i += blockDim.x)
        a.partial[(size_t)blockIdx.x * kStride + i] = slot_sum<VT>(red + i, kOW, kRed);
    const int ne = kind == 0 ? B : B * B;
    if ((int)threadIdx.x < ne)
      a.partial[(size_t)blockIdx.x * kStride + (kind == 0 ? kNormOff : kGramOff) + threadIdx.x] =
          slot_sum<VT>(red + kXo + threadIdx.x, kOW, kRed);
    return true;
  };

  // Thread-per-row Gram of U (B x B) over this CTA's rows to partial[off..],
  // optionally after U <- U R1^{-1}; four rows per thread in flight.
  auto gram_rows = [&](int off, bool apply_r1) {
    Acc<VT> g[NG];
#pragma unroll
    for (int e = 0; e < NG; ++e) g[e].zero();
    VT rd[B][B];  // R1 in the row type, converted once
#pragma unroll
    for (int q = 0; q < B; ++q)
#pragma unroll
      for (int v = 0; v < B; ++v) rd[q][v] = (VT)Rd1[q * B + v];
    VT rdi[B];  // reciprocals of the diagonal: one division per thread, multiplications per row
#pragma unroll
    for (int v = 0; v < B; ++v) rdi[v] = VT(1) / rd[v][v];
    auto rows = [&](int lo, int hi) {
      int nb = 0;
      for (int rb = lo + threadIdx.x; rb < hi; rb += 4 * kOT) {
        VT u[4][4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          if (rb + t * kOT < hi) ld4(U + (size_t)(rb + t * kOT) * 4, u[t]);
          else u[t][0] = u[t][1] = u[t][2] = u[t][3] = VT(0);
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          if (apply_r1) {
#pragma unroll
            for (int v = 0; v < B; ++v) {
              VT s = u[t][v];
#pragma unroll
              for (int q = 0; q < v; ++q) s -= u[t][q] * rd[q][v];
              u[t][v] = s * rdi[v];
            }
            if (rb + t * kOT < hi) st4(U + (size_t)(rb + t * kOT) * 4, u[t]);
          }
          int e = 0;
#pragma unroll
          for (int v = 0; v < B; ++v)
#pragma unroll
            for (int w2 = v; w2 < B; ++w2) g[e++].fma_(u[t][v], u[t][w2]);
        }
        if (++nb == 4) {
#pragma unroll
          for (int ee = 0; ee < NG; ++ee) g[ee].flush();
          nb = 0;
        }
      }
    };
    rows(r0, r1);
#pragma unroll
    for (int e = 0; e < NG; ++e) g[e].reduce(1);
    __syncthreads();
    if (lane == 0) {
      int e = 0;
#pragma unroll
      for (int v = 0; v < B; ++v)
#pragma unroll
        for (int w2 = v; w2 < B; ++w2) {
          const double x = g[e++].slot();
          scratch[warp * 16 + v * B + w2] = x;
          scratch[warp * 16 + w2 * B + v] = x;
        }
    }
    __syncthreads();
    if ((int)threadIdx.x < B * B)
      a.partial[(size_t)blockIdx.x * kStride + off + threadIdx.x] = slot_sum<VT>(scratch + threadIdx.x, kOW, 16);
  };

  // Cholesky of gram_s = R^T R (R upper).  A column whose remaining norm
  // vanishes relative to its input norm marks a breakdown: its row of R is
  // zero (as recorded in H) and Rd keeps a unit divisor.
  auto cholesky = [&](double* R, double* Rd, double* Rdi) {
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
    if (threadIdx.x == 0)
      for (int v = 0; v < B; ++v) Rdi[v] = 1.0 / Rd[v * B + v];
    __syncthreads();
  };

  // Entry (r, c), c < j, of the projected matrix V[:, 0:J]^T A V[:, 0:j]: the upper triangle holds
  // the square part (symmetric), rows of the input block hold its R block and restart couplings.
  auto hfull = [&](int r, int c) -> double {
    return r <= c ? a.H[(size_t)r + (size_t)a.ldh * c]
                  : (r < a.j ? a.H[(size_t)c + (size_t)a.ldh * r] : a.H[(size_t)r + (size_t)a.ldh * c]);
  };
  const bool defer = a.defer != 0 && J > 0;
  int sweeps = 0;
  if (J > 0) {
    // sweep 1: (finish the input block;) c1 = V^T U and the input norms
    if (!sweep(0)) return;
    ++sweeps;
    if (!grid_sync(a.bar, a.err, a.wait_ns)) return;
    reduce_owned(a.partial, kStride, gridDim.x, P, a.coef, scratch);
    // The operator saw the input block before its correction: A q = A q_stored - A V[:, 0:j] e, and
    // V^T A V[:, 0:j] e = H[0:J, 0:j] e, so the recorded coefficients drop that term.  (The
    // projected vector itself is unchanged: U - V c1 removes everything in span(V) either way.)
    // one thread per owned coefficient (the correction below is a j-term FP64 dot product, and
    // FP64 is a narrow pipe: done by every thread of the CTA it cost more than a sweep); its
    // operands are first staged in shared memory by the whole CTA, one round trip instead of j
    const int Qown = P > (int)blockIdx.x ? (P - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
    const bool staged = a.j > 0 && a.pend_in != nullptr && a.j * B + Qown * a.j <= kOW * kRed;
    if (staged) {
      double* pe = red;              // pend_in, j x B
      double* hr = red + a.j * B;    // the owned rows of H[:, 0:j]
      for (int i = threadIdx.x; i < a.j * B; i += blockDim.x) pe[i] = __ldcg(a.pend_in + i);
      for (int i = threadIdx.x; i < Qown * a.j; i += blockDim.x) {
        const int q = i / a.j, c = i % a.j;
        hr[i] = hfull((int)(blockIdx.x + gridDim.x * q) / B, c);
      }
      __syncthreads();
      for (int q = threadIdx.x; q < Qown; q += blockDim.x) {
        const int p = blockIdx.x + gridDim.x * q, v = p % B;
        double t = 0.0;
        for (int c = 0; c < a.j; ++c) t = fma(hr[q * a.j + c], pe[c * B + v], t);
        a.H[(size_t)(p / B) + (size_t)a.ldh * (a.j + v)] = a.coef[p] - t;
      }
      __syncthreads();
    }
    if (a.j >= 0 && !staged)
      for (int p = blockIdx.x + gridDim.x * threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        double hv = a.coef[p];
        if (a.pend_in) {
          const int r = p / B, v = p % B;
          double t = 0.0;
          for (int c = 0; c < a.j; ++c) t = fma(hfull(r, c), a.pend_in[c * B + v], t);
          hv -= t;
        }
        a.H[(size_t)(p / B) + (size_t)a.ldh * (a.j + p % B)] = hv;
      }
    reduce_all(a.partial, kStride, gridDim.x, kNormOff, B, unorm, scratch);
    if (!grid_sync(a.bar, a.err, a.wait_ns)) return;
    // sweep 2: U -= V c1; c2 = V^T U; Gram
    if (!sweep(1)) return;
    ++sweeps;
    if (!grid_sync(a.bar, a.err, a.wait_ns)) return;
    reduce_all(a.partial, kStride, gridDim.x, kGramOff, B * B, gram_s, scratch);
    if (threadIdx.x == 0) {
      again = 0;
      for (int v = 0; v < B; ++v)
        if (gram_s[v * B + v] < 0.5 * unorm[v]) again = 1;  // DGKS: kept less than 1/sqrt(2) of the norm
    }
    __syncthreads();
    if (defer) {
      // the second projection U -= V c2 is left to the next launch: its coefficients join H, and
      // the Gram matrix of the projected block is G - c2^T c2 (V^T V = I, V^T U = c2)
      reduce_owned(a.partial, kStride, gridDim.x, P, a.coef, scratch);
      if (a.j >= 0)
        for (int p = blockIdx.x + gridDim.x * threadIdx.x; p < P; p += gridDim.x * blockDim.x)
          a.H[(size_t)(p / B) + (size_t)a.ldh * (a.j + p % B)] += a.coef[p];
      if (!grid_sync(a.bar, a.err, a.wait_ns)) return;
      // c2 staged in shared memory by all threads (one round trip), then the B x B products
      for (int i = threadIdx.x; i < P; i += blockDim.x) red[i] = __ldcg(a.coef + i);
      __syncthreads();
      if ((int)threadIdx.x < B * B) {
        const int v = threadIdx.x / B, w2 = threadIdx.x % B;
        double t = 0.0;
        for (int c = 0; c < J; ++c) t = fma(red[c * B + v], red[c * B + w2], t);
        scratch[threadIdx.x] = t;
      }
      __syncthreads();
      if ((int)threadIdx.x < B * B) gram_s[threadIdx.x] -= scratch[threadIdx.x];
      __syncthreads();
    } else if (again) {
      reduce_owned(a.partial, kStride, gridDim.x, P, a.coef, scratch);
      if (a.j >= 0)
        for (int p = blockIdx.x + gridDim.x * threadIdx.x; p < P; p += gridDim.x * blockDim.x)
          a.H[(size_t)(p / B) + (size_t)a.ldh * (a.j + p % B)] += a.coef[p];
      if (!grid_sync(a.bar, a.err, a.wait_ns)) return;
      // sweep 3: U -= V c2; Gram
      if (!sweep(2)) return;
      ++sweeps;
      if (!grid_sync(a.bar, a.err, a.wait_ns)) return;
      reduce_all(a.partial, kStride, gridDim.x, kGramOff, B * B, gram_s, scratch);
    }
  } else {
    if (threadIdx.x < B) unorm[threadIdx.x] = 0.0;
    gram_rows(kGramOff, false);
    if (!grid_sync(a.bar, a.err, a.wait_ns)) return;
    reduce_all(a.partial, kStride, gridDim.x, kGramOff, B * B, gram_s, scratch);
  }
  cholesky(R1, Rd1, Rdi1);

  // deferred mode: e1 = c2 R1^{-1} (J x B) in scratch, the pending correction after the first QR
  auto pending_times_rinv = [&](const double* Rd, const double* Rdi, bool from_coef) {
    if ((int)threadIdx.x < J) {
      const int c = threadIdx.x;
      double x[4];
#pragma unroll
      for (int v = 0; v < B; ++v) x[v] = from_coef ? __ldcg(a.coef + c * B + v) : scratch[c * B + v];
      // row c of x R^{-1}: forward substitution with the upper factor
#pragma unroll
      for (int v = 0; v < B; ++v) {
        double t = x[v];
#pragma unroll
        for (int q = 0; q < v; ++q) t -= x[q] * Rd[q * B + v];
        x[v] = t * Rdi[v];
      }
#pragma unroll
      for (int v = 0; v < B; ++v) scratch[c * B + v] = x[v];
    }
    __syncthreads();
  };
  if (defer) pending_times_rinv(Rd1, Rdi1, true);
  if (B > 1) {
    // Cholesky QR a second time: U <- U R1^{-1}, Gram again
    double e1tv = 0.0;  // thread v * B + w: (e1^T e1)_vw
    if (defer) {
      if ((int)threadIdx.x < B * B) {
        const int v = threadIdx.x / B, w2 = threadIdx.x % B;
        for (int c = 0; c < J; ++c) e1tv = fma(scratch[c * B + v], scratch[c * B + w2], e1tv);
      }
      // keep e1 while gram_rows and reduce_all reuse scratch: in this CTA's own partial row, whose
      // coefficient slots are free once every CTA has reduced c2 (a grid barrier ago)
      for (int i = threadIdx.x; i < J * B; i += blockDim.x) a.partial[(size_t)blockIdx.x * kStride + i] = scratch[i];
      __syncthreads();
    }
    gram_rows(kGram2Off, true);
    if (!grid_sync(a.bar, a.err, a.wait_ns)) return;
    reduce_all(a.partial, kStride, gridDim.x, kGram2Off, B * B, gram_s, scratch);
    if (defer) {
      if ((int)threadIdx.x < B * B) gram_s[threadIdx.x] -= e1tv;
      for (int i = threadIdx.x; i < J * B; i += blockDim.x) scratch[i] = a.partial[(size_t)blockIdx.x * kStride + i];
    }
    if (threadIdx.x < B) unorm[threadIdx.x] = 0.0;
    __syncthreads();
    cholesky(R2, Rd2, Rdi2);
    if (defer) pending_times_rinv(Rd2, Rdi2, false);
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
  VT rf[B][B];  // the divisor factor (R2, or R1 when B = 1) in the row type
#pragma unroll
  for (int q = 0; q < B; ++q)
#pragma unroll
    for (int v = 0; v < B; ++v) rf[q][v] = (VT)(B > 1 ? Rd2[q * B + v] : Rd1[q * B + v]);
  VT rfi[B];
#pragma unroll
  for (int v = 0; v < B; ++v) rfi[v] = VT(1) / rf[v][v];
  auto final_rows = [&](int lo, int hi) {
    for (int rb = lo + threadIdx.x; rb < hi; rb += 4 * kOT) {
      VT u[4][4];
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (rb + t * kOT < hi) ld4(U + (size_t)(rb + t * kOT) * 4, u[t]);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int r = rb + t * kOT;
        if (r >= hi) continue;
#pragma unroll
        for (int v = 0; v < B; ++v) {
          VT s = u[t][v];
#pragma unroll
          for (int q = 0; q < v; ++q) s -= u[t][q] * rf[q][v];
          u[t][v] = s * rfi[v];
        }
        if (B == 4) {  // then J % 4 == 0: the block fills panel J / 4
          st4(Vp + (size_t)r * 4, u[t]);
          st4(a.Q + (size_t)r * 4, u[t]);
        } else {
#pragma unroll
          for (int v = 0; v < B; ++v) {
            Vp[(size_t)r * 4 + c0 + v] = u[t][v];
            a.Q[(size_t)r * 4 + v] = u[t][v];
          }
        }
      }
    }
  };
  final_rows(r0, r1);
  if (defer && blockIdx.x == 0)
    for (int i = threadIdx.x; i < J * B; i += blockDim.x) a.pend_out[i] = scratch[i];
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
static void orth_launch_t(const OrthPlan& p, int J, int j, bool pend_in, bool defer, cudaStream_t s) {
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
  a.bar = GridBarrier{p.barrier};
  a.err = p.err;
  a.brk_step = p.brk_step;
  a.sweeps = p.sweeps;
  a.J = J;
  a.j = j;
  a.wait_ns = p.wait_ns;
  a.pend_in = pend_in ? p.pend : nullptr;
  a.pend_out = defer ? p.pend : nullptr;
  a.defer = defer ? 1 : 0;
  const size_t smem = orth_smem_bytes<VT, NC>();
  auto kern = orth_kernel<VT, B, NC>;
  check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "orth smem attr");
  void* args[] = {&a};
  check_cuda(cudaLaunchCooperativeKernel((void*)kern, dim3(p.grid), dim3(kOT), args, smem, s), "orth cooperative launch");
}

template <typename VT, int B>
static void orth_launch_b(const OrthPlan& p, int J, int j, bool pend_in, bool defer, cudaStream_t s) {
  if (J <= 128) orth_launch_t<VT, B, 1>(p, J, j, pend_in, defer, s);
  else orth_launch_t<VT, B, 2>(p, J, j, pend_in, defer, s);
}

void launch_orth(const OrthPlan& p, VecType vt, int J, int j, int B, bool pend_in, bool defer, cudaStream_t s) {
  if (J > 256) fail(SFAIRSC_ERR_UNSUPPORTED, "Krylov basis larger than 256 columns");
  if ((J & 3) + B > 4) fail(SFAIRSC_ERR_UNSUPPORTED, "a new block must fit in one 4-column panel");
  if ((pend_in || defer) && (j < 0 || !p.pend)) fail(SFAIRSC_ERR_INVALID_ARG, "deferred projection needs a step and a buffer");
  if (vt == VecType::F64) {
    if (B == 1) orth_launch_b<double, 1>(p, J, j, pend_in, defer, s);
    else if (B == 2) orth_launch_b<double, 2>(p, J, j, pend_in, defer, s);
    else orth_launch_b<double, 4>(p, J, j, pend_in, defer, s);
  } else {
    if (B == 1) orth_launch_b<float, 1>(p, J, j, pend_in, defer, s);
    else if (B == 2) orth_launch_b<float, 2>(p, J, j, pend_in, defer, s);
    else orth_launch_b<float, 4>(p, J, j, pend_in, defer, s);
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
