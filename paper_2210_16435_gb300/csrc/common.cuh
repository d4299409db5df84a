// Device helpers shared by the s-FairSC kernels: value/vector type traits,
// a bounded grid barrier, warp reductions, and error-free FP32 transforms.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace sfairsc {

constexpr int kWarp = 32;
constexpr int kMaxGroups = 32;

// Error bits written by kernels into the context's device error word.
enum : unsigned {
  kErrBarrierTimeout = 1u << 0,
  kErrBreakdown = 1u << 1,
  kErrNonFinite = 1u << 2,
};

// ---------------------------------------------------------------- load helpers
// A BF16 value is the upper half of the FP32 with the same sign, exponent and
// leading mantissa bits, so widening is an exact 16-bit shift (integer pipe).
__device__ __forceinline__ float bf16_bits_to_f32(__nv_bfloat16 v) {
  return __uint_as_float(((unsigned)__bfloat16_as_ushort(v)) << 16);
}
__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(float v) { return (double)v; }
__device__ __forceinline__ double to_f64(__nv_bfloat16 v) { return (double)bf16_bits_to_f32(v); }
__device__ __forceinline__ float to_f32(double v) { return (float)v; }
__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return bf16_bits_to_f32(v); }

template <typename VT>
__device__ __forceinline__ VT cvt(double v);
template <>
__device__ __forceinline__ double cvt<double>(double v) { return v; }
template <>
__device__ __forceinline__ float cvt<float>(double v) { return (float)v; }

template <typename VT, typename MT>
__device__ __forceinline__ VT val_as(MT v);
template <>
__device__ __forceinline__ double val_as<double, double>(double v) { return v; }
template <>
__device__ __forceinline__ double val_as<double, float>(float v) { return (double)v; }
template <>
__device__ __forceinline__ double val_as<double, __nv_bfloat16>(__nv_bfloat16 v) { return (double)bf16_bits_to_f32(v); }
template <>
__device__ __forceinline__ float val_as<float, double>(double v) { return (float)v; }
template <>
__device__ __forceinline__ float val_as<float, float>(float v) { return v; }
template <>
__device__ __forceinline__ float val_as<float, __nv_bfloat16>(__nv_bfloat16 v) { return bf16_bits_to_f32(v); }

// ---------------------------------------------------------------- warp sums
template <typename T>
__device__ __forceinline__ T warp_allsum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u > v ? u : v;
  }
  return v;
}

// ---------------------------------------------------------------- error-free transforms
// TwoSum (Knuth) and TwoProd (FMA): s + e == a + b and p + e == a * b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Compensated dot-product accumulator (Ogita, Rump and Oishi, "Accurate sum
// and dot product", 2005, Algorithm Dot2): the result is as accurate as if
// computed in twice the working precision and then rounded.
struct Dot2 {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    float pe = __fmaf_rn(a, b, -p);
    float t, e;
    two_sum(s, p, t, e);
    s = t;
    c = __fadd_rn(c, __fadd_rn(pe, e));
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// FP32 running sum with a TwoSum carry: s + c carries about twice FP32 precision.
struct Comp32 {
  float s, c;
  __device__ __forceinline__ void zero() {
    s = 0.f;
    c = 0.f;
  }
  __device__ __forceinline__ void add(float x) {
    float t, e;
    two_sum(s, x, t, e);
    s = t;
    c = __fadd_rn(c, e);
  }
  // sum over lanes whose ids differ in bits >= from
  __device__ __forceinline__ void reduce(int from) {
    for (int o = from; o < 32; o <<= 1) {
      const float os = __shfl_xor_sync(0xffffffffu, s, o), oc = __shfl_xor_sync(0xffffffffu, c, o);
      float t, e;
      two_sum(s, os, t, e);
      s = t;
      c = __fadd_rn(__fadd_rn(c, oc), e);
    }
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
  // (s, c) packed into 8 bytes, for comp32_slot_sum: lets many pairs be
  // combined in FP32 with one conversion to FP64 at the end
  __device__ __forceinline__ double slot() const {
    return __longlong_as_double((long long)(((unsigned long long)__float_as_uint(c) << 32) | __float_as_uint(s)));
  }
};

// Warp reduce-scatter of N compensated accumulators (N a power of two, 1..32):
// recursive halving over lane bits 16, 8, ... -- at each level a lane keeps the
// half of its accumulators selected by that bit of its lane id and receives its
// partner's copy of the same half, adding by TwoSum -- then plain halving of the
// one remaining accumulator over the lower lane bits.  Afterwards lane L holds
// in acc[0] the full warp sum of accumulator scatter_index<N>(L) (lanes that
// differ only in bits below log2(N) hold the same sum).  N + ... + 1 exchanges
// instead of 5 N for a butterfly on every accumulator; the order of the adds
// is fixed, so the result is bitwise reproducible.
template <int N>
__device__ __forceinline__ int scatter_index(int lane) {
  int idx = 0;
#pragma unroll
  for (int half = N / 2, o = 16; half >= 1; half >>= 1, o >>= 1)
    if (lane & o) idx += half;
  return idx;
}

__device__ __forceinline__ Comp32 comp32_combine(Comp32 a, float os, float oc) {
  float t, e;
  two_sum(a.s, os, t, e);
  Comp32 r;
  r.s = t;
  r.c = __fadd_rn(__fadd_rn(a.c, oc), e);
  return r;
}

template <int N>
__device__ __forceinline__ void comp32_reduce_scatter(Comp32 (&acc)[N], int lane) {
  static_assert(N >= 1 && N <= 32 && (N & (N - 1)) == 0, "a power of two up to the warp width");
  int o = 16;
#pragma unroll
  for (int half = N / 2; half >= 1; half >>= 1, o >>= 1) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const Comp32 lo = acc[i], hi = acc[i + half];
      const Comp32 send = upper ? lo : hi, keep = upper ? hi : lo;
      const float rs = __shfl_xor_sync(0xffffffffu, send.s, o), rc = __shfl_xor_sync(0xffffffffu, send.c, o);
      acc[i] = comp32_combine(keep, rs, rc);
    }
  }
  for (; o >= 1; o >>= 1) {
    const float rs = __shfl_xor_sync(0xffffffffu, acc[0].s, o), rc = __shfl_xor_sync(0xffffffffu, acc[0].c, o);
    acc[0] = comp32_combine(acc[0], rs, rc);
  }
}

// The same tree for plain values (FP64): N + ... + 1 adds per lane instead of 5 N, which matters
// where FP64 is a narrow pipe.
template <int N, typename T>
__device__ __forceinline__ void reduce_scatter(T (&acc)[N], int lane) {
  static_assert(N >= 1 && N <= 32 && (N & (N - 1)) == 0, "a power of two up to the warp width");
  int o = 16;
#pragma unroll
  for (int half = N / 2; half >= 1; half >>= 1, o >>= 1) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const T lo = acc[i], hi = acc[i + half];
      const T send = upper ? lo : hi, keep = upper ? hi : lo;
      acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  for (; o >= 1; o >>= 1) acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], o);
}

// Sum of n packed pairs p[0], p[stride], ... (Comp32::slot) by TwoSum in
// FP32, in order, converted to FP64 once.
__device__ __forceinline__ double comp32_slot_sum(const double* p, int n, int stride) {
  Comp32 t;
  t.zero();
  for (int i = 0; i < n; ++i) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(p[(size_t)i * stride]);
    t.add(__uint_as_float((unsigned)b));
    t.add(__uint_as_float((unsigned)(b >> 32)));
  }
  return t.value();
}

// Nanosecond global timer (PTX %globaltimer).
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------- grid barrier
// Barrier over all CTAs of a cooperative launch on one 64-bit arrival counter
// that only grows: a CTA adds 1 and waits until the counter reaches the next
// multiple of the grid size.  All CTAs of one barrier arrive before any CTA
// can arrive at the next, so the arrivals of barrier i return values in
// [i G, (i + 1) G) for grid size G.  A counter therefore serves every launch
// of kernels with one grid size (each passes all of its barriers); it starts
// at zero and is zeroed again after an error.  The spin is bounded: after
// `limit_ns` nanoseconds the waiting CTA sets kErrBarrierTimeout in *err and
// the barrier returns false, so no launch can hang.  Co-residency of all CTAs
// is guaranteed by the cooperative launch.
struct GridBarrier {
  unsigned long long* count;  // arrivals so far
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned atom_add_acqrel_gpu(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ unsigned long long ld_acquire_gpu_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long atom_add_acqrel_gpu_u64(unsigned long long* p, unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.add.acq_rel.gpu.global.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
  return old;
}

__device__ __forceinline__ bool grid_sync(GridBarrier bar, unsigned* err, unsigned long long limit_ns = 2000000000ull) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned long long g = (unsigned long long)gridDim.x * gridDim.y * gridDim.z;
    const unsigned long long old = atom_add_acqrel_gpu_u64(bar.count, 1ull);
    const unsigned long long target = (old / g + 1ull) * g;
    if (ld_acquire_gpu_u64(bar.count) < target) {
      const unsigned long long t0 = globaltimer_ns();
      while (ld_acquire_gpu_u64(bar.count) < target) {
        if (globaltimer_ns() - t0 > limit_ns) {
          atomicOr(err, kErrBarrierTimeout);
          ok = 0;
          break;
        }
      }
    }
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// Bounded wait of the whole CTA for *flag to become nonzero (a fault-injection
// hook: the caller passes a word that nothing sets).  Thread 0 polls; after
// limit_ns it sets kErrBarrierTimeout in *err.  Returns true if the flag was seen.
__device__ __forceinline__ bool wait_flag(const unsigned* flag, unsigned* err, unsigned long long limit_ns) {
  __shared__ int seen_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int seen = 1;
    const unsigned long long t0 = globaltimer_ns();
    while (ld_acquire_gpu(flag) == 0u) {
      if (globaltimer_ns() - t0 > limit_ns) {
        atomicOr(err, kErrBarrierTimeout);
        seen = 0;
        break;
      }
    }
    seen_s = seen;
  }
  __syncthreads();
  return seen_s != 0;
}

}  // namespace sfairsc

namespace sfairsc {

// ---------------------------------------------------------------- bulk async copies (TMA engine)
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for an mbarrier phase: gives up after limit_ns, sets kErrBarrierTimeout, returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned* err,
                                          unsigned long long limit_ns = 2000000000ull) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer_ns() - t0 > limit_ns) {
      atomicOr(err, kErrBarrierTimeout);
      return false;
    }
  }
  return true;
}
// 1-D bulk copy global -> shared completing on an mbarrier (16-byte aligned, size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

}  // namespace sfairsc
