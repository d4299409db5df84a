// Thick restart of the restarted block Lanczos (Algorithm 3 step 3) on the tensor cores: the
// kept Ritz vectors V[:, 0:K] <- V[:, 0:m] Y and the carried block V[:, K:K+B] <- V[:, m:m+B]
// - V[:, 0:m] E are one product V[:, 0:m] [Y | -E] of an n x m basis with an m x (K + B) matrix,
// a dense contraction (about 22 flops per byte at m = 100), here with tcgen05.mma kind::tf32.
//
// Accuracy: FP32 operands are split into TF32 parts a = a_hi + a_lo (a_hi = a rounded to TF32,
// a_lo = a - a_hi exactly, then rounded to TF32 as well), and the product is taken as
// a_hi y_hi + a_hi y_lo + a_lo y_hi (the three-pass TF32 scheme; the dropped a_lo y_lo and the
// rounding of the low parts are below 2^-21 of each term).  The tensor cores' FP32 accumulation is
// not round-to-nearest over long chains (with one accumulator over all 13 K steps of m = 100 the
// kept vectors lost orthogonality at the 3e-6 level), so the hi * hi products go to several
// accumulators, each over a short run of K steps, whose partial sums the epilogue adds in FP32
// with round-to-nearest; the corrections, 2^-11 of the size, share one accumulator.
//
// Layout: the basis is stored as panels of 4 columns (panel p = an n x 4 row-major array), so a
// 128-row tile of one panel is 2 KB of 8-row x 16-byte core matrices, the canonical K-major
// layout without swizzle; one 3-D TMA copy (4 columns x 128 rows x all panels) brings a row
// tile of the whole basis.  [Y | -E] is prepared once per restart, split and transposed into the
// same K-major panel form (Y^T in 16-byte pieces), and held in shared memory by every CTA.
//
// One CTA of 256 threads per SM walks row tiles; with two tile buffers the TMA copy of the next
// tile runs under the split, the MMAs and the epilogue of the current one.  Thread 0 issues the
// copies and the MMAs; the eight warps split the tile in place, then read the accumulator back
// (warp w: TMEM lanes 32 (w % 4) .., column half w / 4) and write rows of panels (16 bytes per
// row, coalesced over a warp's 32 rows).  Every wait on an mbarrier is bounded.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "internal.h"

namespace sfairsc {

namespace {

constexpr int kRT = 128;        // rows per tile = MMA M
constexpr int kRThreads = 256;  // 8 warps

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Shared-memory matrix descriptor: start, leading (K-direction) and stride (M/N-direction) byte
// offsets between 8-row x 16-byte core matrices, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::tf32: D in FP32, A and B TF32, both K-major, M = 128, N.
__host__ __device__ constexpr uint32_t tf32_idesc(int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kRT >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(dtm),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_cta() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive 32-bit accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tma_rows(void* dst, const CUtensorMap* tm, int row0, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(0), "r"(row0), "r"(0), "r"(smem_u32(bar))
      : "memory");
}

struct RestartTcArgs {
  float* V;
  size_t pn;        // floats per panel (n x 4)
  int n, m, K, B;   // basis columns m, kept K, carried block B (= 4)
  int Kd, Np;       // contraction length (m rounded up to 8), output columns (K + B rounded up to 16)
  int stages;       // tile buffers (1 or 2)
  uint32_t tcols;   // TMEM columns allocated (a power of two >= (nreg + 1) rstride)
  int nreg;         // accumulators of the hi * hi products (each a run of consecutive K steps)
  int rstride;      // TMEM columns between accumulators (Np rounded up to 32, the allocation granule)
  const float* Yt;  // [2][Kd / 4][Np][4]: hi and lo parts of [Y | -E]^T in K-major panels
  float* Q;         // n x 4 copy of the carried block
  unsigned* err;
  unsigned long long wait_ns;
};

__global__ void __launch_bounds__(kRThreads, 1) restart_tc_kernel(const __grid_constant__ CUtensorMap tm,
                                                                  RestartTcArgs a) {
  extern __shared__ unsigned char rsm_raw[];
  __shared__ __align__(8) uint64_t tma_bar[2];
  __shared__ __align__(8) uint64_t mma_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int stop;
  // 1 KB-aligned base (the copies and the descriptors want 128-byte alignment at least)
  unsigned char* sm = rsm_raw + ((1024u - (smem_u32(rsm_raw) & 1023u)) & 1023u);
  const uint32_t abytes = (uint32_t)a.Kd * kRT * 4;  // one tile of the basis (Kd / 4 panels x 2 KB)
  const uint32_t ybytes = (uint32_t)a.Kd * a.Np * 4;
  unsigned char* Abuf[2] = {sm, sm + (a.stages == 2 ? abytes : 0)};
  unsigned char* Alo = sm + (size_t)a.stages * abytes;
  unsigned char* Yhi = Alo + abytes;
  unsigned char* Ylo = Yhi + ybytes;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = (a.n + kRT - 1) / kRT;

  if (tid == 0) {
    mbar_init(&tma_bar[0], 1);
    mbar_init(&tma_bar[1], 1);
    mbar_init(&mma_bar, 1);
    mbar_fence_init();
    stop = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(a.tcols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // [Y | -E]^T, both parts, into shared memory
  {
    const float4* src = reinterpret_cast<const float4*>(a.Yt);
    float4* dst = reinterpret_cast<float4*>(Yhi);
    for (uint32_t i = tid; i < 2 * ybytes / 16; i += kRThreads) dst[i] = __ldg(src + i);
  }
  fence_proxy_async_cta();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = tf32_idesc(a.Np);

  int tile = blockIdx.x;
  if (tid == 0 && tile < ntiles) {
    mbar_arrive_expect_tx(&tma_bar[0], abytes);
    tma_rows(Abuf[0], &tm, tile * kRT, &tma_bar[0]);
  }
  unsigned tcount[2] = {0u, 0u};  // completed phases of each copy barrier (thread 0)
  bool tma_out[2] = {tid == 0 && tile < ntiles, false};  // copies issued and not yet waited for (thread 0)
  bool mma_out = false;                                    // MMAs committed and not yet waited for
  unsigned mma_par = 0u;
  for (int it = 0; tile < ntiles; tile += gridDim.x, ++it) {
    const int buf = a.stages == 2 ? (it & 1) : 0;
    const int next = tile + gridDim.x;
    if (a.stages == 2 && tid == 0 && next < ntiles) {  // the other buffer's MMAs finished last iteration
      mbar_arrive_expect_tx(&tma_bar[buf ^ 1], abytes);
      tma_rows(Abuf[buf ^ 1], &tm, next * kRT, &tma_bar[buf ^ 1]);
      tma_out[buf ^ 1] = true;
    }
    if (tid == 0) {
      if (mbar_wait(&tma_bar[buf], tcount[buf] & 1u, a.err, a.wait_ns)) {
        ++tcount[buf];
        tma_out[buf] = false;
      } else {
        stop = 1;
      }
    }
    __syncthreads();
    if (stop) break;
    // split the tile in place: hi part over the raw values, lo part beside it
    {
      float4* hi = reinterpret_cast<float4*>(Abuf[buf]);
      float4* lo = reinterpret_cast<float4*>(Alo);
      for (uint32_t i = tid; i < abytes / 16; i += kRThreads) {
        const float4 x = hi[i];
        float4 h, l;
        h.x = tf32_round(x.x);
        h.y = tf32_round(x.y);
        h.z = tf32_round(x.z);
        h.w = tf32_round(x.w);
        l.x = tf32_round(x.x - h.x);
        l.y = tf32_round(x.y - h.y);
        l.z = tf32_round(x.z - h.z);
        l.w = tf32_round(x.w - h.w);
        hi[i] = h;
        lo[i] = l;
      }
    }
    fence_proxy_async_cta();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t ah = smem_u32(Abuf[buf]), al = smem_u32(Alo), bh = smem_u32(Yhi), bl = smem_u32(Ylo);
      const uint32_t alb = kRT * 16, blb = (uint32_t)a.Np * 16;  // K-direction core-matrix strides
      // hi * hi products into nreg accumulators of consecutive K steps (short accumulation chains;
      // the partial sums are added with round-to-nearest FP32 adds in the epilogue), the two
      // correction products (2^-11 of the size) into one more accumulator after them
      const int nkk = a.Kd / 8;
      const uint32_t dcor = tmem + (uint32_t)(a.nreg * a.rstride);
      for (int kk = 0; kk < nkk; ++kk) {
        const int rg = kk * a.nreg / nkk;
        const bool first = kk == 0 || (kk - 1) * a.nreg / nkk != rg;
        const uint64_t dah = smem_desc(ah + kk * 2 * alb, alb, 128), dal = smem_desc(al + kk * 2 * alb, alb, 128);
        const uint64_t dbh = smem_desc(bh + kk * 2 * blb, blb, 128), dbl = smem_desc(bl + kk * 2 * blb, blb, 128);
        mma_tf32(tmem + (uint32_t)(rg * a.rstride), dah, dbh, idesc, first ? 0u : 1u);
        mma_tf32(dcor, dah, dbl, idesc, kk > 0 ? 1u : 0u);
        mma_tf32(dcor, dal, dbh, idesc, 1u);
      }
      mma_commit(&mma_bar);
      mma_out = true;
      mma_par = (unsigned)it & 1u;
      if (mbar_wait(&mma_bar, mma_par, a.err, a.wait_ns)) mma_out = false;
      else stop = 1;
      if (!stop && a.stages == 1 && next < ntiles) {  // the single buffer is free once the MMAs are done
        mbar_arrive_expect_tx(&tma_bar[0], abytes);
        tma_rows(Abuf[0], &tm, next * kRT, &tma_bar[0]);
        tma_out[0] = true;
      }
    }
    __syncthreads();
    if (stop) break;
    tc_fence_after();
    // epilogue: rows 32 (w % 4) + lane of the tile, column half w / 4
    {
      const int row = tile * kRT + (warp & 3) * 32 + lane;
      const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16);
      const int ngroups = a.Np / 16;
      const bool live = row < a.n;
      for (int g = warp >> 2; g < ngroups; g += 2) {
        float v[16], t[16];
        tmem_ld16(tl + (uint32_t)(g * 16), v);
        for (int rg = 1; rg <= a.nreg; ++rg) {  // the other runs, then the corrections, in a fixed order
          tmem_ld16(tl + (uint32_t)(rg * a.rstride + g * 16), t);
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] += t[i];
        }
        if (!live) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int o = g * 16 + 4 * q;  // first output column of this panel (K % 4 == 0)
          if (o < a.K) {
            *reinterpret_cast<float4*>(a.V + (size_t)(o >> 2) * a.pn + (size_t)row * 4) =
                make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
          } else if (o == a.K) {  // the carried block: its old value plus the product with -E
            const float4 x = *reinterpret_cast<const float4*>(a.V + (size_t)(a.m >> 2) * a.pn + (size_t)row * 4);
            const float4 y = make_float4(x.x + v[4 * q], x.y + v[4 * q + 1], x.z + v[4 * q + 2], x.w + v[4 * q + 3]);
            *reinterpret_cast<float4*>(a.V + (size_t)(o >> 2) * a.pn + (size_t)row * 4) = y;
            *reinterpret_cast<float4*>(a.Q + (size_t)row * 4) = y;
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();  // the accumulator and the lo buffer are free for the next tile
  }
  // leave with nothing in flight: after a timeout, give the outstanding copy and MMAs a bounded
  // chance to land before the tensor memory is released
  if (tid == 0) {
    if (mma_out) mbar_wait(&mma_bar, mma_par, a.err, a.wait_ns);
    for (int b = 0; b < 2; ++b)
      if (tma_out[b]) mbar_wait(&tma_bar[b], tcount[b] & 1u, a.err, a.wait_ns);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tcols) : "memory");
  }
}

// [Y | -E]^T split into TF32 hi and lo parts, in K-major panels: element (o, c) (output column o,
// basis column c) at [part][c / 4][o][c % 4]; zero past m rows and K + B columns.
__global__ void restart_tc_prep_kernel(int m, int K, int B, int Kd, int Np, const float* __restrict__ Y,
                                       const double* __restrict__ E, float* Yt) {
  const int total = Kd * Np;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int c = e / Np, o = e % Np;
    float val = 0.f;
    if (c < m) {
      if (o < K) val = Y[(size_t)c * K + o];
      else if (o < K + B && E) val = -(float)E[(size_t)c * B + (o - K)];
    }
    const float hi = tf32_round(val);
    const float lo = tf32_round(val - hi);
    const size_t at = ((size_t)(c >> 2) * Np + o) * 4 + (c & 3);
    Yt[at] = hi;
    Yt[(size_t)Kd * Np + at] = lo;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    check_cuda(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q),
               "tensor map entry point");
    if (q != cudaDriverEntryPointSuccess || !p) fail(SFAIRSC_ERR_CUDA, "cuTensorMapEncodeTiled not available");
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

}  // namespace

size_t restart_tc_smem(int m, int K, int B, int stages) {
  const int Kd = (m + 7) / 8 * 8, Np = (K + B + 15) / 16 * 16;
  return (size_t)(stages + 1) * Kd * kRT * 4 + 2 * (size_t)Kd * Np * 4 + 1024;
}

bool restart_tc_fits(int n, int64_t ldv, int m, int K, int B) {
  if (B != 4 || (m & 3) || (K & 3) || K + B > m || n < 1) return false;
  const int Kd = (m + 7) / 8 * 8, Np = (K + B + 15) / 16 * 16;
  if (Np > 256 || Kd / 4 > 256 || Kd > ldv) return false;
  return restart_tc_smem(m, K, B, 1) <= 227 * 1024;
}

void launch_restart_tc(int n, float* V, int64_t ldv, int m, int K, int B, const float* Y, float* Q, const double* E,
                       float* Yt, int sms, unsigned* err, unsigned long long wait_ns, cudaStream_t s) {
  if (!restart_tc_fits(n, ldv, m, K, B)) fail(SFAIRSC_ERR_UNSUPPORTED, "restart shape outside the tensor-core path");
  const int Kd = (m + 7) / 8 * 8, Np = (K + B + 15) / 16 * 16;
  restart_tc_prep_kernel<<<(Kd * Np + 255) / 256, 256, 0, s>>>(m, K, B, Kd, Np, Y, E, Yt);
  check_cuda(cudaGetLastError(), "restart prep launch");
  // the basis as a 3-D tensor: 4 columns (16 bytes) x n rows x ldv / 4 panels
  CUtensorMap tm;
  const cuuint64_t gdim[3] = {4, (cuuint64_t)n, (cuuint64_t)(ldv / 4)};
  const cuuint64_t gstride[2] = {16, (cuuint64_t)n * 16};
  const cuuint32_t box[3] = {4, (cuuint32_t)kRT, (cuuint32_t)(Kd / 4)};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = tensor_map_encoder()(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, V, gdim, gstride, box, estr,
                                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) fail(SFAIRSC_ERR_CUDA, "tensor map for the restart");
  RestartTcArgs a;
  a.V = V;
  a.pn = (size_t)n * 4;
  a.n = n;
  a.m = m;
  a.K = K;
  a.B = B;
  a.Kd = Kd;
  a.Np = Np;
  a.stages = restart_tc_smem(m, K, B, 2) <= 227 * 1024 ? 2 : 1;
  // as many hi * hi runs as tensor memory holds beside the corrections (512 columns: 4 at Np = 80)
  a.rstride = (Np + 31) / 32 * 32;
  a.nreg = std::max(1, std::min(Kd / 8, 512 / a.rstride - 1));
  uint32_t tc = 32;
  while ((int)tc < (a.nreg + 1) * a.rstride) tc <<= 1;
  a.tcols = tc;
  a.Yt = Yt;
  a.Q = Q;
  a.err = err;
  a.wait_ns = wait_ns;
  const size_t smem = restart_tc_smem(m, K, B, a.stages);
  check_cuda(cudaFuncSetAttribute(restart_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
             "restart smem attr");
  const int ntiles = (n + kRT - 1) / kRT;
  const int grid = std::min(ntiles, sms);
  restart_tc_kernel<<<grid, kRThreads, smem, s>>>(tm, a);
  check_cuda(cudaGetLastError(), "restart launch");
}

}  // namespace sfairsc
