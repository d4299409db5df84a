// sfairsc_apply_operator_static: one application of L_n^sigma that allocates
// no memory, for callers that cannot call cudaMalloc (see include/sfairsc.h).
//
// All scratch lives in one file-scope __device__ array (g_static_scratch,
// about 20 MB, sized for n <= kStaticMaxN); every GPU that loads the library
// holds it until the process exits.  Host code never touches the symbol
// itself: the first call on each device resolves its device address with
// cudaGetSymbolAddress (with that device current) and caches it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "common.cuh"
#include "internal.h"

namespace sfairsc {

constexpr int64_t kStaticMaxN = 524288;                     // vertices
constexpr int kStaticMaxBlocks = (int)((kStaticMaxN + 255) / 256);  // 256-row setup blocks
constexpr int kStaticMaxGrid = 256;                         // cooperative CTAs of the operator
constexpr int kStaticMaxDevices = 64;

struct StaticScratch {
  double deg[kStaticMaxN];
  double dinv64[kStaticMaxN];
  float dinv32[kStaticMaxN];
  float ytil[4 * kStaticMaxN];
  double blocksums[kStaticMaxBlocks * 2 * kMaxGroups];
  double blockmax[kStaticMaxBlocks];
  double partial[kStaticMaxGrid * kMaxGroups * 4];
  double params[kParams];
  int32_t cta_rows[kStaticMaxGrid + 1];
  uint8_t lab[kStaticMaxN];
  unsigned long long gbar;  // grid barrier arrival counter
  unsigned words[8];        // [0] validation flags, [1] degree flags, [4] kernel error word, [5] SpMV work
};

static __device__ __align__(256) StaticScratch g_static_scratch;

namespace {

std::mutex g_static_mu;
StaticScratch* g_static_addr[kStaticMaxDevices] = {};
// host staging for the setup reductions (used under g_static_mu)
double g_host_blocksums[kStaticMaxBlocks * 2 * kMaxGroups];
double g_host_blockmax[kStaticMaxBlocks];
double g_host_params[kParams];

StaticScratch* scratch_on(int dev) {
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    check_cuda(cudaGetSymbolAddress(&p, g_static_scratch), "cudaGetSymbolAddress(static scratch)");
    g_static_addr[dev] = static_cast<StaticScratch*>(p);
  }
  return g_static_addr[dev];
}

bool on_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

static int apply_static(int64_t n64, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx, const float* values,
                        const int32_t* labels, int h, const float* w, float* out, int nvec, cudaStream_t s,
                        std::string& msg) {
  if (n64 < 2 || nnz < 1 || nnz > 0x7fffffffll || !row_ptr || !col_idx || !values || !labels || !w || !out || h < 1 ||
      nvec < 1 || nvec > SFAIRSC_MAX_BLOCK) {
    msg = "invalid argument";
    return SFAIRSC_ERR_INVALID_ARG;
  }
  if (n64 > kStaticMaxN || h > kMaxGroups) {
    msg = "n exceeds " + std::to_string(kStaticMaxN) + " vertices or h exceeds 32 groups (static scratch limit)";
    return SFAIRSC_ERR_UNSUPPORTED;
  }
  for (const void* p : {(const void*)row_ptr, (const void*)col_idx, (const void*)values, (const void*)labels,
                        (const void*)w, (const void*)out})
    if (!on_device(p)) {
      msg = "every pointer must be device memory (host data would need a staging allocation)";
      return SFAIRSC_ERR_INVALID_ARG;
    }
  const int n = (int)n64;
  int dev = 0;
  check_cuda(cudaGetDevice(&dev), "get device");
  if (dev < 0 || dev >= kStaticMaxDevices) fail(SFAIRSC_ERR_UNSUPPORTED, "device index out of range");
  StaticScratch* S = scratch_on(dev);

  // words that must start at zero: flags, barrier, error
  check_cuda(cudaMemsetAsync(&S->gbar, 0, sizeof(S->gbar) + sizeof(S->words), s), "clear scratch words");
  unsigned* vflags = &S->words[0];
  unsigned* dflags = &S->words[1];
  unsigned long long* barrier = &S->gbar;
  unsigned* err = &S->words[4];
  launch_validate(n, nnz, row_ptr, col_idx, values, SFAIRSC_F32, labels, h, 0, vflags, s);
  unsigned hf[2] = {0, 0};
  check_cuda(cudaMemcpyAsync(hf, S->words, 2 * sizeof(unsigned), cudaMemcpyDeviceToHost, s), "d2h");
  check_cuda(cudaStreamSynchronize(s), "validate");
  if (hf[0] & ((1u << 0) | (1u << 1) | (1u << 2))) fail(SFAIRSC_ERR_BAD_CSR, "CSR structure invalid");
  if (hf[0] & (1u << 4)) fail(SFAIRSC_ERR_NONFINITE, "non-finite edge weight");
  if (hf[0] & (1u << 3)) fail(SFAIRSC_ERR_BAD_CSR, "negative edge weight");
  if (hf[0] & (1u << 5)) fail(SFAIRSC_ERR_INVALID_ARG, "group label outside [0, h)");

  // degrees, D^{-1/2}, group sums; sigma = ||L_n||_1
  const int nb = degrees_blocks(n);
  launch_degrees(n, row_ptr, values, SFAIRSC_F32, labels, S->lab, S->deg, S->dinv64, S->dinv32, S->blocksums, nb, h, 1,
                 dflags, s);
  launch_sigma_rows(n, row_ptr, col_idx, values, SFAIRSC_F32, S->dinv64, S->deg, 1, S->blockmax, (n + 255) / 256, s);
  check_cuda(cudaMemcpyAsync(g_host_blocksums, S->blocksums, sizeof(double) * nb * 2 * h, cudaMemcpyDeviceToHost, s),
             "d2h");
  check_cuda(cudaMemcpyAsync(g_host_blockmax, S->blockmax, sizeof(double) * ((n + 255) / 256), cudaMemcpyDeviceToHost, s),
             "d2h");
  check_cuda(cudaMemcpyAsync(&hf[1], dflags, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "d2h");
  check_cuda(cudaStreamSynchronize(s), "degrees");
  if (hf[1] & (1u << 8)) fail(SFAIRSC_ERR_ISOLATED_VERTEX, "a vertex has zero degree");
  double cnt[kMaxGroups] = {}, Ssum[kMaxGroups] = {}, z[kMaxGroups] = {};
  for (int b = 0; b < nb; ++b)
    for (int g = 0; g < h; ++g) {
      cnt[g] += g_host_blocksums[((size_t)b * h + g) * 2 + 0];
      Ssum[g] += g_host_blocksums[((size_t)b * h + g) * 2 + 1];
    }
  double Stot = 0.0;
  for (int g = 0; g < h; ++g) {
    if (cnt[g] < 0.5) fail(SFAIRSC_ERR_EMPTY_GROUP, "group " + std::to_string(g) + " is empty");
    z[g] = cnt[g] / n;
    Stot += Ssum[g];
  }
  double* P = g_host_params;
  std::fill(P, P + kParams, 0.0);
  for (int g = 0; g < h; ++g) P[kPZ + g] = z[g];
  const int p = h - 1;
  for (int a = 0; a < p; ++a)
    for (int b = 0; b <= a; ++b) {
      // (C^T C)_ab = delta_ab S_a - z_b S_a - z_a S_b + z_a z_b sum S, then Cholesky
      double sum = (a == b ? Ssum[a] : 0.0) - z[b] * Ssum[a] - z[a] * Ssum[b] + z[a] * z[b] * Stot;
      for (int q = 0; q < b; ++q) sum -= P[kPL + a * kLStride + q] * P[kPL + b * kLStride + q];
      if (a == b) {
        if (!(sum > 0.0)) fail(SFAIRSC_ERR_EMPTY_GROUP, "C^T C is not positive definite");
        P[kPL + a * kLStride + a] = std::sqrt(sum);
      } else {
        P[kPL + a * kLStride + b] = sum / P[kPL + b * kLStride + b];
      }
    }
  double sigma = 0.0;
  for (int b = 0; b < (n + 255) / 256; ++b) sigma = std::max(sigma, g_host_blockmax[b]);
  P[kPSigma] = sigma;
  for (int a = 0; a + 1 < h; ++a) P[kPLinv + a] = 1.0 / P[kPL + a * kLStride + a];
  fill_group_map(P, h, false);
  check_cuda(cudaMemcpyAsync(S->params, P, sizeof(double) * kParams, cudaMemcpyHostToDevice, s), "h2d");

  // the fused operator, on the static scratch
  const int threads = 1024;
  const size_t smem = operator_smem_bytes(threads, h, 4, VecType::F32);
  const int gmax = std::min(kStaticMaxGrid, operator_max_grid(VecType::F32, SFAIRSC_F32, 4, threads, smem));
  if (gmax < 1) fail(SFAIRSC_ERR_UNSUPPORTED, "operator kernel does not fit on this device");
  const long long work = nnz + 16ll * n;
  const int grid = (int)std::max(1ll, std::min<long long>(gmax, (work + 16383) / 16384));
  launch_row_partition(n, row_ptr, grid, 16, S->cta_rows, s);
  OpPlan o;
  o.n = n;
  o.h = h;
  o.normalized = 1;
  o.grid = grid;
  o.threads = threads;
  o.batch_rows = (int)std::max(1ll, std::min(32ll, (long long)n / grid / 64));
  {
    const double avg = (double)nnz / (double)n;
    int lanes = 2;
    while (lanes < 32 && lanes * 8 < avg) lanes *= 2;
    o.lanes_per_row = lanes;  // lanes per row of the SpMV, 8 entries per lane per pass
  }
  o.row_ptr = row_ptr;
  o.col = col_idx;
  o.val = values;
  o.val_dtype = SFAIRSC_F32;
  o.lab = S->lab;
  o.dinv = S->dinv32;
  o.deg = S->deg;
  o.params = S->params;
  o.ytil = S->ytil;
  o.partial = S->partial;
  o.cta_rows = S->cta_rows;
  o.barrier = barrier;
  o.err = err;
  o.work = &S->words[5];
  launch_operator(o, VecType::F32, w, 1, n, out, 1, n, nvec, s);
  unsigned e = 0;
  check_cuda(cudaMemcpyAsync(&e, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "d2h");
  check_cuda(cudaStreamSynchronize(s), "operator");
  if (e & kErrBarrierTimeout) fail(SFAIRSC_ERR_DEVICE_TIMEOUT, "a grid barrier timed out");
  return SFAIRSC_OK;
}

}  // namespace sfairsc

extern "C" SFAIRSC_API int sfairsc_apply_operator_static(int64_t n, int64_t nnz, const int32_t* row_ptr,
                                                         const int32_t* col_idx, const float* values,
                                                         const int32_t* group_labels, int32_t h, const float* w,
                                                         float* out, int32_t nvec, void* cuda_stream) {
  std::lock_guard<std::mutex> lock(sfairsc::g_static_mu);
  std::string msg;
  try {
    const int rc = sfairsc::apply_static(n, nnz, row_ptr, col_idx, values, group_labels, h, w, out, nvec,
                                         static_cast<cudaStream_t>(cuda_stream), msg);
    sfairsc::set_last_error(msg);
    return rc;
  } catch (const sfairsc::SfError& e) {
    sfairsc::set_last_error(e.msg);
    return e.code;
  } catch (...) {
    sfairsc::set_last_error("unexpected internal error");
    return SFAIRSC_ERR_CUDA;
  }
}
