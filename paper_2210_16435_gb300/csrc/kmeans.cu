// Seeded k-means on the rows of H (Algorithm 3 step 4).
//
// The paper only says "apply k-means to the rows of H".  This implementation
// fixes every unstated detail so that results are exactly reproducible,
// independent of thread scheduling:
//  * data X = float32(H); a squared distance is accumulated in float32 in
//    dimension order, one rounding per subtract / multiply / add (no FMA);
//  * draws: splitmix64 (Steele, Lea and Flood 2014) as a counter generator,
//    draw q of seed s = mix(s + (q + 1) * 0x9E3779B97F4A7C15); replicate r
//    uses draws r*k + t;
//  * k-means++ (Arthur and Vassilvitskii 2007): center 0 = row
//    floor(r64 * n / 2^64); center t > 0 = first row whose prefix sum of
//    integer weights q_i = trunc(D2_i * 2^S) exceeds floor(r64 * total / 2^64),
//    S = 62 - bitlen(n) - e for max D2 = f 2^e, 1/2 <= f < 1;
//  * Lloyd: nearest float32(centroid), lowest index on ties; stop when no
//    label changes or after max_iter assignments; centroids are exact
//    fixed-point sums (scale from max |X|) divided once in FP64; an empty
//    cluster takes the row farthest from its own centroid (lowest row on
//    ties), clusters in increasing order;
//  * the replicate with the smallest quantised inertia wins (lowest index on ties).
// Integer sums are associative, so atomics give the same bits in any order.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace sfairsc {

static uint64_t host_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static uint64_t host_draw(uint64_t seed, uint64_t q) { return host_mix64(seed + (q + 1) * 0x9E3779B97F4A7C15ull); }
static uint64_t host_mulhi(uint64_t a, uint64_t b) { return (uint64_t)(((unsigned __int128)a * b) >> 64); }
static int bitlen(uint64_t n) { return n ? 64 - __builtin_clzll(n) : 0; }

// trunc(x * 2^s) for a float32 x, exactly, with integer operations only.
__device__ __forceinline__ long long quantise_f32(float x, int s) {
  const unsigned b = __float_as_uint(x);
  const unsigned ex = (b >> 23) & 0xFF;
  unsigned long long m = b & 0x7FFFFF;
  int e2;
  if (ex == 0) {
    e2 = -149;  // subnormal: m * 2^-149
  } else {
    m |= 0x800000;
    e2 = (int)ex - 150;
  }
  const int sh = e2 + s;
  unsigned long long mag;
  if (m == 0) mag = 0;
  else if (sh >= 0) mag = m << sh;
  else if (sh <= -64) mag = 0;
  else mag = m >> (-sh);
  return (b >> 31) ? -(long long)mag : (long long)mag;
}

// Scale exponent S for nonnegative values up to maxbits (float bits), n summands.
__device__ __forceinline__ int scale_shift(float maxv, long long n) {
  int e;
  frexpf(maxv, &e);
  return 62 - (64 - __clzll((unsigned long long)n)) - e;
}

// sum over j in order of (x_j - m_j)^2, each operation rounded once; the subtract and the add run
// as fma(., +-one, .) with one = 1 from the launch (exact like a plain add, on the FMA pipe)
__device__ __forceinline__ float dist_rn(const float* x, const float* m, int d, float one) {
  float acc = 0.f;
  if ((d & 1) == 0) {  // rows of even length start 8-byte aligned: the point's coordinates two at a time
    const float2* x2 = reinterpret_cast<const float2*>(x);
    for (int j2 = 0; j2 < (d >> 1); ++j2) {
      const float2 xv = x2[j2];
      const float t0 = __fmaf_rn(m[2 * j2], -one, xv.x);
      acc = __fmaf_rn(acc, one, __fmul_rn(t0, t0));
      const float t1 = __fmaf_rn(m[2 * j2 + 1], -one, xv.y);
      acc = __fmaf_rn(acc, one, __fmul_rn(t1, t1));
    }
    return acc;
  }
  for (int j = 0; j < d; ++j) {
    const float t = __fmaf_rn(m[j], -one, x[j]);
    acc = __fmaf_rn(acc, one, __fmul_rn(t, t));
  }
  return acc;
}

__global__ void to_f32_kernel(long long nd, const double* __restrict__ X, float* X32, unsigned* maxbits) {
  unsigned best = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nd; i += (long long)gridDim.x * blockDim.x) {
    const float v = __double2float_rn(X[i]);
    X32[i] = v;
    const unsigned b = __float_as_uint(fabsf(v));
    best = b > best ? b : best;
  }
  best = warp_max(best);
  if ((threadIdx.x & 31) == 0) atomicMax(maxbits, best);
}

// ---------------------------------------------------------------- k-means++ seeding
// D2 <- (t == 1 ? dist(x, c) : min(D2, dist(x, c))) for the newest center c; block maxima.
__global__ void seed_dist_kernel(int n, int d, const float* __restrict__ X32, int k, const int* __restrict__ centers,
                                 int t, float* D2, unsigned* blockmax, float one) {
  extern __shared__ float csh[];
  const int r = blockIdx.y;
  const int c = centers[r * k + t - 1];
  for (int j = threadIdx.x; j < d; j += blockDim.x) csh[j] = X32[(size_t)c * d + j];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned mb = 0;
  if (i < n) {
    float v = dist_rn(X32 + (size_t)i * d, csh, d, one);
    float* p = D2 + (size_t)r * n + i;
    if (t > 1) v = fminf(*p, v);
    *p = v;
    mb = __float_as_uint(v);
  }
  mb = warp_max(mb);
  __shared__ unsigned red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mb;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = red[w] > b ? red[w] : b;
    blockmax[(size_t)r * gridDim.x + blockIdx.x] = b;
  }
}

__global__ void seed_gmax_kernel(int nb, const unsigned* __restrict__ blockmax, unsigned* gmax) {
  const int r = blockIdx.x;
  unsigned b = 0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) b = max(b, blockmax[(size_t)r * nb + i]);
  b = warp_max(b);
  __shared__ unsigned red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = b;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = max(m, red[w]);
    gmax[r] = m;
  }
}

__global__ void seed_qsum_kernel(int n, const float* __restrict__ D2, const unsigned* __restrict__ gmax,
                                 long long* blocksum) {
  const int r = blockIdx.y;
  const float mx = __uint_as_float(gmax[r]);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  long long q = 0;
  if (mx > 0.f && i < n) q = quantise_f32(D2[(size_t)r * n + i], scale_shift(mx, n));
  // exact integer block sum
  for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
  __shared__ long long red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = q;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    blocksum[(size_t)r * gridDim.x + blockIdx.x] = s;
  }
}

// One CTA (1024 threads) per replicate: locate the row where the prefix sum crosses the target.
__global__ void seed_select_kernel(int n, int nb, int bs, const float* __restrict__ D2, const unsigned* __restrict__ gmax,
                                   const long long* __restrict__ blocksum, const unsigned long long* __restrict__ r64,
                                   int k, int t, int* centers) {
  const int r = blockIdx.x;
  const unsigned long long draw = r64[r * k + t];
  const float mx = __uint_as_float(gmax[r]);
  __shared__ long long tsum[1024];
  __shared__ int found_block;
  __shared__ long long before;
  if (!(mx > 0.f)) {
    if (threadIdx.x == 0) centers[r * k + t] = (int)__umul64hi(draw, (unsigned long long)n);
    return;
  }
  const int s = scale_shift(mx, n);
  const long long* bsum = blocksum + (size_t)r * nb;
  const int T = blockDim.x;
  const int per = (nb + T - 1) / T;
  const int lo = threadIdx.x * per, hi = min(nb, lo + per);
  long long mine = 0;
  for (int i = lo; i < hi; ++i) mine += bsum[i];
  tsum[threadIdx.x] = mine;
  __syncthreads();
  // inclusive scan of tsum (Hillis-Steele on 1024 entries)
  for (int o = 1; o < T; o <<= 1) {
    const long long v = threadIdx.x >= o ? tsum[threadIdx.x - o] : 0;
    __syncthreads();
    tsum[threadIdx.x] += v;
    __syncthreads();
  }
  const long long total = tsum[T - 1];
  const unsigned long long target = __umul64hi(draw, (unsigned long long)total);
  if (threadIdx.x == 0) found_block = -1;
  __syncthreads();
  {
    long long cum = threadIdx.x > 0 ? tsum[threadIdx.x - 1] : 0;
    if ((unsigned long long)tsum[threadIdx.x] > target && (unsigned long long)cum <= target) {
      for (int i = lo; i < hi; ++i) {
        if ((unsigned long long)(cum + bsum[i]) > target) {
          found_block = i;
          before = cum;
          break;
        }
        cum += bsum[i];
      }
    }
  }
  __syncthreads();
  const int b = found_block;
  if (b < 0) {  // unreachable when total > 0; keep every index in range regardless
    if (threadIdx.x == 0) centers[r * k + t] = 0;
    return;
  }
  // scan the rows of block b (bs <= 1024 rows)
  const int row = b * bs + threadIdx.x;
  long long q = 0;
  if (threadIdx.x < bs && row < n) q = quantise_f32(D2[(size_t)r * n + row], s);
  tsum[threadIdx.x] = q;
  __syncthreads();
  for (int o = 1; o < T; o <<= 1) {
    const long long v = threadIdx.x >= o ? tsum[threadIdx.x - o] : 0;
    __syncthreads();
    tsum[threadIdx.x] += v;
    __syncthreads();
  }
  const long long cum_incl = before + tsum[threadIdx.x];
  const long long cum_excl = before + (threadIdx.x > 0 ? tsum[threadIdx.x - 1] : 0);
  if (threadIdx.x < bs && row < n && (unsigned long long)cum_incl > target && (unsigned long long)cum_excl <= target)
    centers[r * k + t] = row;
}

__global__ void init_centroids_kernel(int d, int k, const float* __restrict__ X32, const int* __restrict__ centers,
                                      double* mu, int* lab, int n, int R) {
  const int r = blockIdx.y;
  for (int i = threadIdx.x + blockIdx.x * blockDim.x; i < k * d; i += blockDim.x * gridDim.x) {
    const int c = i / d, j = i % d;
    mu[(size_t)r * k * d + i] = (double)X32[(size_t)centers[r * k + c] * d + j];
  }
  for (int i = threadIdx.x + blockIdx.x * blockDim.x; i < n; i += blockDim.x * gridDim.x) lab[(size_t)r * n + i] = -1;
}

// ---------------------------------------------------------------- Lloyd
// Packed pairs of float32 for the Blackwell f32x2 add / sub / mul: each half
// is rounded on its own, exactly as the scalar operation would round it.
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void unpack2(unsigned long long v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long sub2_rn(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long mul2_rn(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// Nearest centroid of each row.  The squared distance is the float32 sum
// over dimensions in order of (x_j - m_j)^2, each subtract, square and add
// rounded once; the subtracts and squares of dimensions j and j + 1 run as
// one packed pair, and two centroids are scanned together (two independent
// sums).  An odd dimension count is padded with x = m = 0, whose +0 term
// leaves the sum unchanged.
// The adds of the distance sums run as fma(a, one, b) with one = 1 passed at launch (opaque to the
// compiler): a * 1 is exact, so each rounds a + b once exactly as an add does, but issues on the
// FMA pipe (plain FP32 adds share a narrower pipe on this GPU).
template <int DMAX>
__global__ void __launch_bounds__(256, 3) assign_kernel(int n, int d, int k, const float* __restrict__ X32, const double* __restrict__ mu,
                              int* lab, float* dist, unsigned* changed, const int* __restrict__ done, float one) {
  static_assert(DMAX % 2 == 0, "dimension pairs");
  // centroids in groups of four, interleaved by dimension pair: element (c, j) at
  // ((c / 4) * dp / 2 + j / 2) * 8 + (c % 4) * 2 + j % 2, so one 16-byte load brings a dimension pair of
  // two centroids (dp = d rounded up to even, zero padded; k rounded up to 4 with zero centroids)
  extern __shared__ float msh[];
  const int r = blockIdx.y;
  if (done[r]) return;
  const int dp = (d + 1) & ~1;
  const int k4 = (k + 3) & ~3;
  for (int t = threadIdx.x; t < k4 * dp; t += blockDim.x) {
    const int c = t / dp, j = t - c * dp;
    msh[((c >> 2) * (dp >> 1) + (j >> 1)) * 8 + (c & 3) * 2 + (j & 1)] =
        (c < k && j < d) ? __double2float_rn(mu[(size_t)r * k * d + (size_t)c * d + j]) : 0.f;
  }
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  bool ch = false;
  if (i < n) {
    float x[DMAX];
    if ((d & 1) == 0) {
      const float2* xr = reinterpret_cast<const float2*>(X32 + (size_t)i * d);
#pragma unroll
      for (int j2 = 0; j2 < DMAX / 2; ++j2) {
        const float2 v = 2 * j2 < d ? xr[j2] : make_float2(0.f, 0.f);
        x[2 * j2] = v.x;
        x[2 * j2 + 1] = v.y;
      }
    } else {
#pragma unroll
      for (int j = 0; j < DMAX; ++j) x[j] = j < d ? X32[(size_t)i * d + j] : 0.f;
    }
    float best = 0.f;
    int bi = 0;
    // four centroids at a time: four independent chains of adds (each in dimension order) keep the
    // FMA pipe busy between the dependent adds of one chain
    for (int c = 0; c < k; c += 4) {
      const float4* mg = reinterpret_cast<const float4*>(msh + (size_t)(c >> 2) * (dp >> 1) * 8);
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int j2 = 0; j2 < DMAX / 2; ++j2) {
        if (2 * j2 < d) {
          const unsigned long long xp = pack2(x[2 * j2], x[2 * j2 + 1]);
          const float4 m01 = mg[2 * j2], m23 = mg[2 * j2 + 1];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float2 p = q == 0 ? make_float2(m01.x, m01.y) : q == 1 ? make_float2(m01.z, m01.w)
                           : q == 2 ? make_float2(m23.x, m23.y) : make_float2(m23.z, m23.w);
            const unsigned long long t = sub2_rn(xp, pack2(p.x, p.y));
            float s0, s1;
            unpack2(mul2_rn(t, t), s0, s1);
            acc[q] = __fmaf_rn(__fmaf_rn(acc[q], one, s0), one, s1);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (c + q < k && ((c + q) == 0 || acc[q] < best)) {  // first minimum in centroid order
          best = acc[q];
          bi = c + q;
        }
    }
    int* lp = lab + (size_t)r * n + i;
    ch = *lp != bi;
    *lp = bi;
    dist[(size_t)r * n + i] = best;
  }
  const unsigned b = __ballot_sync(0xffffffffu, ch);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(changed + r, (unsigned)__popc(b));
}

// Exact fixed-point centroid sums.  Each warp walks a contiguous run of rows,
// lanes over dimensions, keeping a running sum while the label repeats.
__global__ void update_sums_kernel(int n, int d, int k, const float* __restrict__ X32, const int* __restrict__ lab,
                                   int xshift, long long* sums, long long* counts, const int* __restrict__ done,
                                   int rows_per_warp) {
  extern __shared__ long long ssum[];  // k * d + k
  const int r = blockIdx.y;
  if (done[r]) return;
  for (int i = threadIdx.x; i < k * d + k; i += blockDim.x) ssum[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // CTAs take the row blocks from the last one down: the assignment just before read the points in
  // ascending order, so the first CTAs to run find their rows still in L2 (and the next assignment,
  // ascending again, starts on the rows read here last)
  const long long w0 = ((long long)(gridDim.x - 1 - blockIdx.x) * nw + warp) * rows_per_warp;
  const int* lb = lab + (size_t)r * n;
  // trunc(x 2^xshift): scaling by a power of two is exact (the scaled value
  // stays below 2^63, and one below 2^-126 truncates to 0 either way), and the
  // float-to-integer conversion truncates exactly
  const bool fast = xshift >= -126 && xshift <= 127;
  const float scale = fast ? __int_as_float((xshift + 127) << 23) : 0.f;
  auto quant = [&](float x) -> long long {
    return fast ? __float2ll_rz(__fmul_rn(x, scale)) : quantise_f32(x, xshift);
  };
  int cur = -1;
  long long a0 = 0, a1 = 0, cnt = 0;
  const long long wend = min((long long)n, w0 + rows_per_warp);
  // eight rows' labels and coordinates in flight before they are added (integer sums: the order
  // of the adds does not change the result)
  constexpr int RF = 8;
  for (long long i0 = w0; i0 < wend; i0 += RF) {
    int l[RF];
    float x0[RF], x1[RF];
#pragma unroll
    for (int q = 0; q < RF; ++q) {
      const long long i = i0 + q;
      const bool in = i < wend;
      l[q] = in ? lb[i] : -1;
      x0[q] = in && lane < d ? X32[(size_t)i * d + lane] : 0.f;
      x1[q] = in && lane + 32 < d ? X32[(size_t)i * d + lane + 32] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < RF; ++q) {
      if (l[q] < 0) break;
      if (l[q] != cur) {
        if (cur >= 0) {
          if (lane < d) atomicAdd((unsigned long long*)&ssum[cur * d + lane], (unsigned long long)a0);
          if (lane + 32 < d) atomicAdd((unsigned long long*)&ssum[cur * d + lane + 32], (unsigned long long)a1);
          if (lane == 0) atomicAdd((unsigned long long*)&ssum[k * d + cur], (unsigned long long)cnt);
        }
        cur = l[q];
        a0 = a1 = cnt = 0;
      }
      if (lane < d) a0 += quant(x0[q]);
      if (lane + 32 < d) a1 += quant(x1[q]);
      cnt += 1;
    }
  }
  if (cur >= 0) {
    if (lane < d) atomicAdd((unsigned long long*)&ssum[cur * d + lane], (unsigned long long)a0);
    if (lane + 32 < d) atomicAdd((unsigned long long*)&ssum[cur * d + lane + 32], (unsigned long long)a1);
    if (lane == 0) atomicAdd((unsigned long long*)&ssum[k * d + cur], (unsigned long long)cnt);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < k * d; i += blockDim.x)
    if (ssum[i]) atomicAdd((unsigned long long*)&sums[(size_t)r * k * d + i], (unsigned long long)ssum[i]);
  for (int i = threadIdx.x; i < k; i += blockDim.x)
    if (ssum[k * d + i]) atomicAdd((unsigned long long*)&counts[(size_t)r * k + i], (unsigned long long)ssum[k * d + i]);
}

// One CTA per replicate: convergence test, new centroids, empty-cluster relocation, reset.
__global__ void finalize_kernel(int n, int d, int k, const float* __restrict__ X32, float* dist, int xshift,
                                long long* sums, long long* counts, unsigned* changed, double* mu, int* done,
                                int* iters, int it, int max_iter) {
  const int r = blockIdx.x;
  if (done[r]) return;
  __shared__ int stop;
  if (threadIdx.x == 0) {
    stop = 0;
    if (it > 0 && changed[r] == 0u) {
      done[r] = 1;
      iters[r] = it + 1;
      stop = 1;
    }
  }
  __syncthreads();
  long long* S = sums + (size_t)r * k * d;
  long long* C = counts + (size_t)r * k;
  if (!stop) {
    for (int i = threadIdx.x; i < k * d; i += blockDim.x) {
      const int c = i / d;
      if (C[c] > 0) mu[(size_t)r * k * d + i] = ldexp(__ll2double_rn(S[i]), -xshift) / (double)C[c];
    }
    __syncthreads();
    // empty clusters, in order: farthest row from its own centroid, lowest row on ties
    __shared__ unsigned long long bestkey[32];
    for (int c = 0; c < k; ++c) {
      if (C[c] > 0) continue;
      unsigned long long key = 0;  // (dist bits + 1) << 32 | ~row ; 0 = none
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float v = dist[(size_t)r * n + i];
        if (v >= 0.f) {
          const unsigned long long kk = ((unsigned long long)(__float_as_uint(v) + 1u) << 32) | (0xFFFFFFFFull - i);
          key = kk > key ? kk : key;
        }
      }
      key = warp_max(key);
      if ((threadIdx.x & 31) == 0) bestkey[threadIdx.x >> 5] = key;
      __syncthreads();
      if (threadIdx.x == 0) {
        unsigned long long b = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = bestkey[w] > b ? bestkey[w] : b;
        bestkey[0] = b;
      }
      __syncthreads();
      const unsigned long long b = bestkey[0];
      if (b != 0) {
        const int row = (int)(0xFFFFFFFFull - (b & 0xFFFFFFFFull));
        for (int j = threadIdx.x; j < d; j += blockDim.x) mu[((size_t)r * k + c) * d + j] = (double)X32[(size_t)row * d + j];
        if (threadIdx.x == 0) dist[(size_t)r * n + row] = -1.f;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0 && it == max_iter - 1) {
      done[r] = 1;
      iters[r] = max_iter;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < k * d; i += blockDim.x) S[i] = 0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) C[i] = 0;
  if (threadIdx.x == 0) changed[r] = 0u;
}

// Inertia: distance of each row to its own centroid; max, then exact quantised sum.
__global__ void own_dist_kernel(int n, int d, int k, const float* __restrict__ X32, const double* __restrict__ mu,
                                const int* __restrict__ lab, float* dist, unsigned* maxbits, float one) {
  extern __shared__ float msh[];
  const int r = blockIdx.y;
  for (int i = threadIdx.x; i < k * d; i += blockDim.x) msh[i] = __double2float_rn(mu[(size_t)r * k * d + i]);
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned mb = 0;
  if (i < n) {
    const int c = lab[(size_t)r * n + i];
    const float v = dist_rn(X32 + (size_t)i * d, msh + c * d, d, one);
    dist[(size_t)r * n + i] = v;
    mb = __float_as_uint(v);
  }
  mb = warp_max(mb);
  if ((threadIdx.x & 31) == 0) atomicMax(maxbits + r, mb);
}

__global__ void qsum_all_kernel(int n, const float* __restrict__ dist, const unsigned* __restrict__ maxbits,
                                long long* total) {
  const int r = blockIdx.y;
  const float mx = __uint_as_float(maxbits[r]);
  long long q = 0;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (mx > 0.f && i < n) q = quantise_f32(dist[(size_t)r * n + i], scale_shift(mx, n));
  for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
  if ((threadIdx.x & 31) == 0 && q) atomicAdd((unsigned long long*)(total + r), (unsigned long long)q);
}

__global__ void pick_labels_kernel(int n, const int* __restrict__ lab, int* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = lab[i];
}

template <typename T>
static T* dalloc(size_t count, cudaStream_t s, std::vector<void*>& bag) {
  void* p = nullptr;
  if (count == 0) count = 1;
  const cudaError_t e = cudaMallocAsync(&p, count * sizeof(T), s);
  if (e != cudaSuccess) fail(SFAIRSC_ERR_OOM, "k-means workspace allocation failed");
  bag.push_back(p);
  return static_cast<T*>(p);
}

KmeansResult run_kmeans(int64_t n64, int d, const double* X, int kc, uint64_t seed, int n_init, int max_iter,
                        int32_t* labels, double* centroids, cudaStream_t s) {
  if (n64 <= 0 || n64 > (1ll << 30) || d < 1 || d > 64 || kc < 1 || kc > n64 || n_init < 1 || max_iter < 1)
    fail(SFAIRSC_ERR_INVALID_ARG, "k-means arguments out of range (1 <= d <= 64, 1 <= k <= n)");
  if ((size_t)kc * d * sizeof(long long) + kc * sizeof(long long) > 200 * 1024)
    fail(SFAIRSC_ERR_UNSUPPORTED, "k-means: k * d too large for one CTA's shared memory");
  const int n = (int)n64, R = n_init, k = kc;
  std::vector<void*> bag;
  const int bs = 256;
  const int nb = (n + bs - 1) / bs;
  KmeansResult res;
  try {
    float* X32 = dalloc<float>((size_t)n * d, s, bag);
    float* D2 = dalloc<float>((size_t)R * n, s, bag);
    float* dist = dalloc<float>((size_t)R * n, s, bag);
    int* lab = dalloc<int>((size_t)R * n, s, bag);
    double* mu = dalloc<double>((size_t)R * k * d, s, bag);
    long long* sums = dalloc<long long>((size_t)R * k * d, s, bag);
    long long* counts = dalloc<long long>((size_t)R * k, s, bag);
    int* centers = dalloc<int>((size_t)R * k, s, bag);
    unsigned long long* r64 = dalloc<unsigned long long>((size_t)R * k, s, bag);
    unsigned* blockmax = dalloc<unsigned>((size_t)R * nb, s, bag);
    long long* blocksum = dalloc<long long>((size_t)R * nb, s, bag);
    // small words: [0] xmax bits, [1..R] gmax, [..] changed, done, iters, maxbits, totals
    unsigned* xmax = dalloc<unsigned>(1, s, bag);
    unsigned* gmax = dalloc<unsigned>(R, s, bag);
    unsigned* changed = dalloc<unsigned>(R, s, bag);
    int* done = dalloc<int>(R, s, bag);
    int* iters = dalloc<int>(R, s, bag);
    unsigned* maxd = dalloc<unsigned>(R, s, bag);
    long long* tot = dalloc<long long>(R, s, bag);
    check_cuda(cudaMemsetAsync(xmax, 0, sizeof(unsigned), s), "memset");
    check_cuda(cudaMemsetAsync(sums, 0, sizeof(long long) * R * k * d, s), "memset");
    check_cuda(cudaMemsetAsync(counts, 0, sizeof(long long) * R * k, s), "memset");
    check_cuda(cudaMemsetAsync(changed, 0, sizeof(unsigned) * R, s), "memset");
    check_cuda(cudaMemsetAsync(done, 0, sizeof(int) * R, s), "memset");
    check_cuda(cudaMemsetAsync(iters, 0, sizeof(int) * R, s), "memset");
    check_cuda(cudaMemsetAsync(maxd, 0, sizeof(unsigned) * R, s), "memset");
    check_cuda(cudaMemsetAsync(tot, 0, sizeof(long long) * R, s), "memset");

    to_f32_kernel<<<std::min(1024, (int)(((long long)n * d + 255) / 256)), 256, 0, s>>>((long long)n * d, X, X32, xmax);
    // splitmix64 draws and the first centers on the host
    std::vector<unsigned long long> draws((size_t)R * k);
    std::vector<int> first((size_t)R * k, 0);
    for (int r = 0; r < R; ++r)
      for (int t = 0; t < k; ++t) draws[(size_t)r * k + t] = host_draw(seed, (uint64_t)r * k + t);
    for (int r = 0; r < R; ++r) first[(size_t)r * k] = (int)host_mulhi(draws[(size_t)r * k], (uint64_t)n);
    check_cuda(cudaMemcpyAsync(r64, draws.data(), sizeof(unsigned long long) * R * k, cudaMemcpyHostToDevice, s), "h2d");
    check_cuda(cudaMemcpyAsync(centers, first.data(), sizeof(int) * R * k, cudaMemcpyHostToDevice, s), "h2d");
    check_cuda(cudaStreamSynchronize(s), "k-means upload");  // host vectors go out of scope below
    res.launches = 1 + 4 * (k - 1) + 1;
    for (int t = 1; t < k; ++t) {
      seed_dist_kernel<<<dim3(nb, R), bs, sizeof(float) * d, s>>>(n, d, X32, k, centers, t, D2, blockmax, 1.f);
      seed_gmax_kernel<<<R, 1024, 0, s>>>(nb, blockmax, gmax);
      seed_qsum_kernel<<<dim3(nb, R), bs, 0, s>>>(n, D2, gmax, blocksum);
      seed_select_kernel<<<R, 1024, 0, s>>>(n, nb, bs, D2, gmax, blocksum, r64, k, t, centers);
    }
    init_centroids_kernel<<<dim3(std::max(1, std::min(256, nb)), R), 256, 0, s>>>(d, k, X32, centers, mu, lab, n, R);
    check_cuda(cudaGetLastError(), "k-means seeding");
    unsigned xbits = 0;
    check_cuda(cudaMemcpyAsync(&xbits, xmax, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "d2h");
    check_cuda(cudaStreamSynchronize(s), "k-means sync");
    float xm;
    std::memcpy(&xm, &xbits, sizeof(float));
    int xshift = 0;
    if (xm > 0.f) {
      int e;
      std::frexp((double)xm, &e);
      xshift = 62 - bitlen((uint64_t)n) - e;
    }
    const size_t msmem = sizeof(float) * (size_t)k * d;
    const size_t amsmem = sizeof(float) * (size_t)((k + 3) & ~3) * ((d + 1) & ~1);  // padded for assign_kernel
    const size_t ssmem = sizeof(long long) * ((size_t)k * d + k);
    const int rows_per_warp = 64;
    const int ub = 256;
    const int unb = (int)((n + (long long)(ub / 32) * rows_per_warp - 1) / ((ub / 32) * rows_per_warp));
    check_cuda(cudaFuncSetAttribute(update_sums_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssmem), "attr");
    auto assign = [&](void) {
      if (d <= 16) {
        check_cuda(cudaFuncSetAttribute(assign_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)amsmem), "attr");
        assign_kernel<16><<<dim3(nb, R), bs, amsmem, s>>>(n, d, k, X32, mu, lab, dist, changed, done, 1.f);
      } else if (d <= 32) {
        check_cuda(cudaFuncSetAttribute(assign_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)amsmem), "attr");
        assign_kernel<32><<<dim3(nb, R), bs, amsmem, s>>>(n, d, k, X32, mu, lab, dist, changed, done, 1.f);
      } else if (d <= 56) {
        check_cuda(cudaFuncSetAttribute(assign_kernel<56>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)amsmem), "attr");
        assign_kernel<56><<<dim3(nb, R), bs, amsmem, s>>>(n, d, k, X32, mu, lab, dist, changed, done, 1.f);
      } else {
        check_cuda(cudaFuncSetAttribute(assign_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)amsmem), "attr");
        assign_kernel<64><<<dim3(nb, R), bs, amsmem, s>>>(n, d, k, X32, mu, lab, dist, changed, done, 1.f);
      }
    };
    std::vector<int> hdone(R);
    for (int it = 0; it < max_iter; ++it) {
      res.launches += 3;
      assign();
      update_sums_kernel<<<dim3(unb, R), ub, ssmem, s>>>(n, d, k, X32, lab, xshift, sums, counts, done, rows_per_warp);
      finalize_kernel<<<R, 1024, 0, s>>>(n, d, k, X32, dist, xshift, sums, counts, changed, mu, done, iters, it, max_iter);
      check_cuda(cudaGetLastError(), "lloyd launch");
      if ((it & 3) == 3 || it == max_iter - 1) {
        check_cuda(cudaMemcpyAsync(hdone.data(), done, sizeof(int) * R, cudaMemcpyDeviceToHost, s), "d2h");
        check_cuda(cudaStreamSynchronize(s), "lloyd sync");
        if (std::all_of(hdone.begin(), hdone.end(), [](int v) { return v != 0; })) break;
      }
    }
    res.launches += 3;
    own_dist_kernel<<<dim3(nb, R), bs, msmem, s>>>(n, d, k, X32, mu, lab, dist, maxd, 1.f);
    qsum_all_kernel<<<dim3(nb, R), bs, 0, s>>>(n, dist, maxd, tot);
    check_cuda(cudaGetLastError(), "inertia launch");
    std::vector<unsigned> hmax(R);
    std::vector<long long> htot(R);
    std::vector<int> hit(R);
    check_cuda(cudaMemcpyAsync(hmax.data(), maxd, sizeof(unsigned) * R, cudaMemcpyDeviceToHost, s), "d2h");
    check_cuda(cudaMemcpyAsync(htot.data(), tot, sizeof(long long) * R, cudaMemcpyDeviceToHost, s), "d2h");
    check_cuda(cudaMemcpyAsync(hit.data(), iters, sizeof(int) * R, cudaMemcpyDeviceToHost, s), "d2h");
    check_cuda(cudaStreamSynchronize(s), "inertia sync");
    int win = 0;
    double best = 0.0;
    for (int r = 0; r < R; ++r) {
      float mx;
      std::memcpy(&mx, &hmax[r], sizeof(float));
      double val = 0.0;
      if (mx > 0.f) {
        int e;
        std::frexp((double)mx, &e);
        const int sh = 62 - bitlen((uint64_t)n) - e;
        val = std::ldexp((double)htot[r], -sh);
      }
      if (r == 0 || val < best) {
        best = val;
        win = r;
      }
    }
    pick_labels_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, lab + (size_t)win * n, labels);
    if (centroids)
      check_cuda(cudaMemcpyAsync(centroids, mu + (size_t)win * k * d, sizeof(double) * k * d, cudaMemcpyDeviceToDevice, s),
                 "centroids copy");
    check_cuda(cudaGetLastError(), "labels launch");
    res.inertia = best;
    res.iterations = hit[win];
    for (void* p : bag) cudaFreeAsync(p, s);
    bag.clear();
    check_cuda(cudaStreamSynchronize(s), "k-means end");
  } catch (...) {
    for (void* p : bag) cudaFreeAsync(p, s);
    throw;
  }
  return res;
}

}  // namespace sfairsc
