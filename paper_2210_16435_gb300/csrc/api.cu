// C entry points of libsfairsc.so (declared in include/sfairsc.h).
//
// sfairsc_create: validation and the setup pass of Algorithm 3 steps 1-2.
// sfairsc_solve:  Algorithm 3 steps 3-4 -- a thick-restart block Lanczos on
//   L_n^sigma (eq. asigma), touching the operator only through the fused
//   kernel of Sec. 3.4 (i)-(ii); FP64 Rayleigh quotients and residuals of the
//   final vectors; H = D^{-1/2} X; seeded k-means on the rows of H.
// The thick restart keeps the K best Ritz vectors plus the next block, which
// is mathematically the implicit restart of ARPACK with exact shifts that the
// paper's eigs performs (Sec. 3.4 (i)).
#include <cuda_bf16.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace sfairsc {

static thread_local std::string g_last_error;

void set_last_error(const std::string& msg) { g_last_error = msg; }

void check_cuda(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    if (e == cudaErrorMemoryAllocation) throw SfError{SFAIRSC_ERR_OOM, std::string(what) + ": out of memory"};
    throw SfError{SFAIRSC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e)};
  }
}

void fail(int code, const std::string& msg) { throw SfError{code, msg}; }

static bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  const cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static size_t dtype_size(int dt) { return dt == SFAIRSC_F64 ? 8 : dt == SFAIRSC_F32 ? 4 : 2; }

// Device memory of the contexts comes from one stream-ordered pool per device that keeps the blocks
// it gets back (release threshold: never), so creating and destroying contexts again and again (a
// solve per request) re-uses memory instead of mapping and unmapping it every time.  The pool
// holds, until the process ends, as much as the largest set of contexts alive at once needed.
static cudaMemPool_t context_pool() {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  check_cuda(cudaGetDevice(&dev), "get device");
  if (dev < 0 || dev >= 64) fail(SFAIRSC_ERR_UNSUPPORTED, "device index above 63");
  std::lock_guard<std::mutex> lk(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    check_cuda(cudaMemPoolCreate(&pool, &props), "memory pool");
    uint64_t keep = ~0ull;
    check_cuda(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep), "memory pool threshold");
    pools[dev] = pool;
  }
  return pools[dev];
}

// Pinned host staging buffers of the contexts (a few small ones each), kept by size for the next
// context: pinning host memory costs far more than the buffers' use.
static std::mutex g_pinned_mu;
static std::multimap<size_t, void*> g_pinned_free;
static void* pinned_get(size_t bytes) {
  {
    std::lock_guard<std::mutex> lk(g_pinned_mu);
    auto it = g_pinned_free.find(bytes);
    if (it != g_pinned_free.end()) {
      void* p = it->second;
      g_pinned_free.erase(it);
      return p;
    }
  }
  void* p = nullptr;
  check_cuda(cudaMallocHost(&p, bytes), "pinned allocation");
  return p;
}
static void pinned_put(void* p, size_t bytes) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pinned_mu);
  if (g_pinned_free.size() < 64) g_pinned_free.emplace(bytes, p);
  else cudaFreeHost(p);
}

}  // namespace sfairsc

using namespace sfairsc;

struct sfairsc_ctx {
  int64_t n = 0, nnz = 0;
  int h = 1, k = 1, normalized = 1;
  int vdt = SFAIRSC_F64;  // dtype of the stored values the operator reads
  int vdt_orig = SFAIRSC_F64;
  sfairsc_opts opts{};
  cudaStream_t stream = nullptr;
  VecType vt = VecType::F32;
  int B = 1, m = 20;
  int64_t ldv = 0;
  int ldh = 0;
  int sms = 0;
  double sigma = 0.0;
  std::vector<double> z;

  const int32_t* row_ptr = nullptr;
  const int32_t* col = nullptr;
  const void* val = nullptr;       // values read by the main operator
  const void* val_orig = nullptr;  // values as given (FP64 final check)
  std::vector<void*> owned;

  uint8_t* lab = nullptr;
  double* deg = nullptr;
  double* dinv64 = nullptr;
  float* dinv32 = nullptr;
  double* params = nullptr;
  double* params_host = nullptr;

  // operator workspace
  OpPlan op;      // main precision
  OpPlan op64;    // FP64 vectors, original values (final residual check)
  OpPlan proj64;  // FP64 projection P w only
  void* ytil = nullptr;
  double* ytil64 = nullptr;
  double* dfT = nullptr;  // n x 8 FP64: L_n X of the final check (MIXED)
  double* op_partial = nullptr;
  int32_t* cta_rows = nullptr;
  int32_t* cta_rows_orth = nullptr;
  unsigned* barrier = nullptr;
  unsigned* err = nullptr;
  int* brk_step = nullptr;
  int* sweeps = nullptr;

  // Krylov workspace
  void* V = nullptr;
  void* U = nullptr;
  void* Q = nullptr;
  double* Hd = nullptr;
  double* Yd = nullptr;
  float* Ytc = nullptr;  // [Y | -E]^T split for the tensor-core restart (FP32 basis)
  double* orth_partial = nullptr;
  double* orth_coef = nullptr;
  OrthPlan orth;
  double* Hh = nullptr;  // pinned host copy of the projected matrix
  double* Yh = nullptr;  // pinned host
  void* Ystage = nullptr;  // pinned host: Y row-major in the basis precision, as uploaded

  // results for backward / outputs
  double* X64 = nullptr;  // n x k column-major
  double* AX64 = nullptr;
  double* Hres = nullptr;  // n x k row-major
  double* lam_d = nullptr;
  double* stat_partial = nullptr;
  int stat_blocks = 0;
  unsigned long long* colkey = nullptr;
  double* diag_partial = nullptr;
  int diag_blocks = 0;
  double* bw_partial = nullptr;
  double* bw_A = nullptr;
  double* bw_Hp = nullptr;  // H with rows padded for the backward gathers
  int bw_blocks = 0;
  int32_t* labels_d = nullptr;
  std::vector<double> lam_h;
  bool solved = false;
  bool fault_pending = false;
  const double* Fd64 = nullptr;  // dense constraints (n x (h - 1) row-major FP64), or null: group labels
  float* Fd32 = nullptr;         // its FP32 copy (MIXED)
  double* fth_partial = nullptr; // per-block F^T H (dense constraints)
  bool shift_found = false;    // the last final check met a Ritz vector in range(C)  // opts.fault_inject: the next operator launch waits on a flag nothing sets
  // live kernel timing (opts.profile) and launch counting
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_op, ev_orth, ev_restart;
  int n_launches = 0;
  cudaEvent_t take_event() {
    if (ev_pool.empty()) {
      cudaEvent_t e;
      check_cuda(cudaEventCreate(&e), "event create");
      return e;
    }
    cudaEvent_t e = ev_pool.back();
    ev_pool.pop_back();
    return e;
  }

  template <typename T>
  T* dalloc(size_t count) {
    void* p = nullptr;
    check_cuda(cudaMallocFromPoolAsync(&p, std::max<size_t>(count, 1) * sizeof(T), context_pool(), stream),
               "device allocation");
    owned.push_back(p);
    return static_cast<T*>(p);
  }
  size_t hh_bytes = 0, yh_bytes = 0, ys_bytes = 0;
  cudaStream_t side = nullptr;  // host copies that overlap device work
  ~sfairsc_ctx() {
    for (auto& pr : ev_op) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
    for (auto& pr : ev_orth) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
    for (auto& pr : ev_restart) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    if (side) {
      cudaStreamSynchronize(side);
      cudaStreamDestroy(side);
    }
    for (void* p : owned) cudaFreeAsync(p, stream);  // back to the pool in stream order
    cudaStreamSynchronize(stream);
    pinned_put(Hh, hh_bytes);
    pinned_put(Yh, yh_bytes);
    pinned_put(Ystage, ys_bytes);
    pinned_put(params_host, sizeof(double) * kParams);
  }
};

namespace {

template <typename F>
int guarded(F&& f) {
  try {
    f();
    g_last_error.clear();
    return SFAIRSC_OK;
  } catch (const SfError& e) {
    g_last_error = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return SFAIRSC_ERR_OOM;
  } catch (...) {
    g_last_error = "unexpected internal error";
    return SFAIRSC_ERR_CUDA;
  }
}

// Copy a host array to a new owned device buffer, or borrow a device pointer.
template <typename T>
const T* to_device(sfairsc_ctx* c, const T* p, size_t count, size_t elem = sizeof(T)) {
  if (is_device_ptr(p)) return p;
  void* d = c->dalloc<unsigned char>(std::max<size_t>(count * elem, 1));
  check_cuda(cudaMemcpyAsync(d, p, count * elem, cudaMemcpyHostToDevice, c->stream), "host to device copy");
  return static_cast<const T*>(d);
}

__global__ void f64_to_f32_kernel(int64_t n, const double* in, float* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

void build_context(sfairsc_ctx* c, const int32_t* row_ptr, const int32_t* col_idx, const void* values,
                   const int32_t* labels, const double* F = nullptr) {
  // dense constraints (F given): no groups; the label passes run with one group of all vertices
  const bool dense = F != nullptr;
  const int hl = dense ? 1 : c->h;
  cudaStream_t s = c->stream;
  const int n = (int)c->n;
  int dev = 0;
  check_cuda(cudaGetDevice(&dev), "get device");
  cudaDeviceProp prop;
  check_cuda(cudaGetDeviceProperties(&prop, dev), "device properties");
  if (prop.major < 10) fail(SFAIRSC_ERR_UNSUPPORTED, "needs a Blackwell (sm_10x) GPU");
  c->sms = prop.multiProcessorCount;

  c->row_ptr = to_device(c, row_ptr, (size_t)n + 1);
  c->col = to_device(c, col_idx, (size_t)c->nnz);
  c->val_orig = to_device(c, static_cast<const unsigned char*>(values), (size_t)c->nnz, dtype_size(c->vdt_orig));
  const int32_t* lab_in = nullptr;
  if (dense) {
    int32_t* zl = c->dalloc<int32_t>(n);
    check_cuda(cudaMemsetAsync(zl, 0, sizeof(int32_t) * n, s), "memset");
    lab_in = zl;
    c->Fd64 = to_device(c, F, (size_t)n * (c->h - 1));
  } else {
    lab_in = to_device(c, labels, (size_t)n);
  }

  unsigned* flags = c->dalloc<unsigned>(4);
  check_cuda(cudaMemsetAsync(flags, 0, 4 * sizeof(unsigned), s), "memset");
  if (c->opts.validate > 0)
    launch_validate(n, c->nnz, c->row_ptr, c->col, c->val_orig, c->vdt_orig, lab_in, hl, c->opts.validate >= 2,
                    flags, s);
  unsigned hf = 0;
  check_cuda(cudaMemcpyAsync(&hf, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "d2h");
  check_cuda(cudaStreamSynchronize(s), "validate");
  if (hf & ((1u << 0) | (1u << 1) | (1u << 2) | (1u << 6) | (1u << 7)))
    fail(SFAIRSC_ERR_BAD_CSR, "CSR structure invalid (row_ptr, column range, self loop or symmetry)");
  if (hf & (1u << 4)) fail(SFAIRSC_ERR_NONFINITE, "non-finite edge weight");
  if (hf & (1u << 3)) fail(SFAIRSC_ERR_BAD_CSR, "negative edge weight");
  if (hf & (1u << 5)) fail(SFAIRSC_ERR_INVALID_ARG, "group label outside [0, h)");

  // degrees, D^{-1/2}, group sums
  c->lab = c->dalloc<uint8_t>(n);
  c->deg = c->dalloc<double>(n);
  c->dinv64 = c->dalloc<double>(n);
  c->dinv32 = c->dalloc<float>(n);
  const int nb = degrees_blocks(n);
  double* bsum = c->dalloc<double>((size_t)nb * 2 * hl);
  check_cuda(cudaMemsetAsync(flags, 0, sizeof(unsigned), s), "memset");
  launch_degrees(n, c->row_ptr, c->val_orig, c->vdt_orig, lab_in, c->lab, c->deg, c->dinv64, c->dinv32, bsum, nb, hl,
                 c->normalized, flags, s);
  std::vector<double> hb((size_t)nb * 2 * hl);
  check_cuda(cudaMemcpyAsync(hb.data(), bsum, hb.size() * sizeof(double), cudaMemcpyDeviceToHost, s), "d2h");
  check_cuda(cudaMemcpyAsync(&hf, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "d2h");
  check_cuda(cudaStreamSynchronize(s), "degrees");
  if (hf & (1u << 8)) fail(SFAIRSC_ERR_ISOLATED_VERTEX, "a vertex has zero degree (D must be positive definite)");
  const int h = c->h;
  std::vector<double> cnt(h, 0.0), S(h, 0.0);
  for (int b = 0; b < nb; ++b)
    for (int g = 0; g < hl; ++g) {
      cnt[g] += hb[((size_t)b * hl + g) * 2 + 0];
      S[g] += hb[((size_t)b * hl + g) * 2 + 1];
    }
  if (!dense)
    for (int g = 0; g < h; ++g)
      if (cnt[g] < 0.5) fail(SFAIRSC_ERR_EMPTY_GROUP, "group " + std::to_string(g) + " is empty");
  if (c->k > n - h + 1) fail(SFAIRSC_ERR_K_TOO_LARGE, "k exceeds n - h + 1");

  // C^T C in closed form and its Cholesky factor (Lemma 2.1: SPD)
  c->z.assign(h, 0.0);
  double Ssum = 0.0;
  if (!dense)
    for (int g = 0; g < h; ++g) {
      c->z[g] = cnt[g] / (double)n;
      Ssum += S[g];
    }
  c->params_host = static_cast<double*>(pinned_get(sizeof(double) * kParams));
  double* P = c->params_host;
  std::fill(P, P + kParams, 0.0);
  for (int g = 0; g < h; ++g) P[kPZ + g] = c->z[g];
  const int p = h - 1;
  std::vector<double> M((size_t)std::max(p, 1) * std::max(p, 1), 0.0);
  if (dense && p > 0) {
    // C^T C = F^T D^{-1} F (F^T F unnormalized) by a device reduction, summed here in block order
    const int cb = std::max(1, std::min(2 * c->sms, (n + 63) / 64));
    double* part = c->dalloc<double>((size_t)cb * p * p);
    launch_dense_ctc(n, p, c->Fd64, c->deg, c->normalized, part, cb, s);
    std::vector<double> hp((size_t)cb * p * p);
    check_cuda(cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, s), "d2h");
    check_cuda(cudaStreamSynchronize(s), "C^T C");
    for (int b = 0; b < cb; ++b)
      for (int q = 0; q < p * p; ++q) M[q] += hp[(size_t)b * p * p + q];
    for (double v : M)
      if (!std::isfinite(v)) fail(SFAIRSC_ERR_NONFINITE, "non-finite entry in F");
  } else {
    for (int a = 0; a < p; ++a)
      for (int b = 0; b < p; ++b)
        M[(size_t)a * p + b] = (a == b ? S[a] : 0.0) - c->z[b] * S[a] - c->z[a] * S[b] + c->z[a] * c->z[b] * Ssum;
  }
  for (int a = 0; a < p; ++a) {
    for (int b = 0; b <= a; ++b) {
      double sum = M[(size_t)a * p + b];
      for (int q = 0; q < b; ++q) sum -= P[kPL + a * kLStride + q] * P[kPL + b * kLStride + q];
      if (a == b) {
        if (!(sum > 0.0))
          fail(dense ? SFAIRSC_ERR_INVALID_ARG : SFAIRSC_ERR_EMPTY_GROUP,
               dense ? "F does not have full column rank (C^T C is not positive definite)"
                     : "C^T C is not positive definite");
        P[kPL + a * kLStride + a] = std::sqrt(sum);
      } else {
        P[kPL + a * kLStride + b] = sum / P[kPL + b * kLStride + b];
      }
    }
  }
  // sigma = ||L_n||_1 unless given
  if (std::isnan(c->opts.sigma)) {
    double* bmax = c->dalloc<double>((n + 255) / 256);
    launch_sigma_rows(n, c->row_ptr, c->col, c->val_orig, c->vdt_orig, c->dinv64, c->deg, c->normalized, bmax,
                      (n + 255) / 256, s);
    std::vector<double> hm((n + 255) / 256);
    check_cuda(cudaMemcpyAsync(hm.data(), bmax, hm.size() * sizeof(double), cudaMemcpyDeviceToHost, s), "d2h");
    check_cuda(cudaStreamSynchronize(s), "sigma");
    c->sigma = *std::max_element(hm.begin(), hm.end());
  } else {
    c->sigma = c->opts.sigma;
  }
  P[kPSigma] = c->sigma;
  for (int a = 0; a + 1 < h; ++a) P[kPLinv + a] = 1.0 / P[kPL + a * kLStride + a];
  fill_group_map(P, h, dense);
  c->params = c->dalloc<double>(kParams);
  check_cuda(cudaMemcpyAsync(c->params, P, sizeof(double) * kParams, cudaMemcpyHostToDevice, s), "h2d");

  // values read by the operator: FP32 copy of FP64 values in the mixed path
  c->val = c->val_orig;
  c->vdt = c->vdt_orig;
  if (c->vt == VecType::F32 && c->vdt_orig == SFAIRSC_F64) {
    float* v32 = c->dalloc<float>((size_t)c->nnz);
    f64_to_f32_kernel<<<1024, 256, 0, s>>>(c->nnz, (const double*)c->val_orig, v32);
    check_cuda(cudaGetLastError(), "value conversion");
    c->val = v32;
    c->vdt = SFAIRSC_F32;
  }

  // operator plans
  const int threads = 1024;
  const size_t smem_f = operator_smem_bytes(threads, h, 4, c->vt);
  const size_t smem_d = operator_smem_bytes(threads, h, 4, VecType::F64);
  const int gmax = std::min(operator_max_grid(c->vt, c->vdt, 4, threads, smem_f),
                            operator_max_grid(VecType::F64, c->vdt_orig, 4, threads, smem_d));
  if (gmax < 1) fail(SFAIRSC_ERR_UNSUPPORTED, "operator kernel does not fit on this device");
  const long long work = c->nnz + 16ll * n;
  const int grid = (int)std::max(1ll, std::min<long long>(gmax, (work + 16383) / 16384));
  c->cta_rows = c->dalloc<int32_t>(grid + 1);
  launch_row_partition(n, c->row_ptr, grid, 16, c->cta_rows, s);
  // rows per warp batch: enough batches for every warp of a CTA, at most 32
  const int batch_rows = (int)std::max(1ll, std::min(32ll, (long long)n / grid / 64));
  const size_t vs = c->vt == VecType::F64 ? 8 : 4;
  c->ytil = c->dalloc<unsigned char>((size_t)n * 4 * vs);
  // FP64 ytil (n x 4); for the MIXED final check also the double-float ytil of 8 vectors (n x 8 pairs)
  c->ytil64 = c->dalloc<double>((size_t)n * (c->vt == VecType::F32 ? 8 : 4));
  c->dfT = c->vt == VecType::F32 ? c->dalloc<double>((size_t)n * 8) : nullptr;
  c->op_partial = c->dalloc<double>((size_t)grid * kMaxGroups * 4);
  // words: [0..1] the operator's 64-bit barrier counter, [2] error word,
  // [4..7] operator work counters, [8..9] the Gram-Schmidt kernel's counter
  c->barrier = c->dalloc<unsigned>(16);
  c->err = c->barrier + 2;
  c->brk_step = c->dalloc<int>(1);
  c->sweeps = c->dalloc<int>(1);
  check_cuda(cudaMemsetAsync(c->barrier, 0, 16 * sizeof(unsigned), s), "memset");
  OpPlan& o = c->op;
  o.n = n;
  o.h = h;
  o.normalized = c->normalized;
  o.grid = grid;
  o.threads = threads;
  o.batch_rows = batch_rows;
  // lanes per row of the SpMV: each lane holds 8 (FP32) or 4 (FP64) entries of its row per pass
  const double avg_deg = (double)c->nnz / std::max(n, 1);
  auto lanes_for = [&](double per_lane) {
    return std::min(32, std::max(2, next_pow2((int)std::ceil(avg_deg / per_lane))));
  };
  o.lanes_per_row = lanes_for(c->vt == VecType::F64 ? 4.0 : 8.0);
  o.row_ptr = c->row_ptr;
  o.col = c->col;
  o.val = c->val;
  o.val_dtype = c->vdt;
  o.lab = c->lab;
  o.dinv = c->vt == VecType::F64 ? (const void*)c->dinv64 : (const void*)c->dinv32;
  o.deg = c->deg;
  o.params = c->params;
  o.ytil = c->ytil;
  o.partial = c->op_partial;
  o.cta_rows = c->cta_rows;
  o.barrier = reinterpret_cast<unsigned long long*>(c->barrier);
  o.err = c->err;
  o.work = c->barrier + 4;
  const unsigned long long wait_ns =
      c->opts.wait_limit_us > 0 ? (unsigned long long)c->opts.wait_limit_us * 1000ull : 2000000000ull;
  o.wait_ns = wait_ns;
  c->fault_pending = c->opts.fault_inject != 0;
  c->op64 = o;
  c->op64.val = c->val_orig;
  c->op64.val_dtype = c->vdt_orig;
  c->op64.dinv = c->dinv64;
  c->op64.ytil = c->ytil64;
  c->op64.lanes_per_row = lanes_for(4.0);
  if (dense && c->h > 1) {
    if (c->vt == VecType::F32) {
      float* f32 = c->dalloc<float>((size_t)n * (c->h - 1));
      launch_f64_to_f32((int64_t)n * (c->h - 1), c->Fd64, f32, s);
      c->Fd32 = f32;
      c->op.Fd = f32;
    } else {
      c->op.Fd = c->Fd64;
    }
    c->op64.Fd = c->Fd64;
  }
  // K (C^T t from the projected input, before the SpMV): the operator then writes its rows in
  // final form with two grid barriers fewer
  if (h > 1) {
    const int kpad = (h + 3) & ~3;
    double* K64 = c->dalloc<double>((size_t)n * kpad);
    float* K32 = c->vt == VecType::F32 ? c->dalloc<float>((size_t)n * kpad) : nullptr;
    launch_kmat(n, c->row_ptr, c->col, c->val_orig, c->vdt_orig, c->lab, dense ? c->Fd64 : nullptr,
                dense ? h - 1 : 0, h, c->dinv64, c->deg, c->normalized, K64, K32, s);
    double* part2 = c->dalloc<double>((size_t)grid * (kMaxGroups + 1) * 4);
    c->op.Kp = K32 ? (const void*)K32 : (const void*)K64;
    c->op.partial2 = part2;
    c->op64.Kp = K64;
    c->op64.partial2 = part2;
  }
  c->proj64 = c->op64;
  c->proj64.mode = 1;
  // shared-memory windows of the SpMV input, one table per block size, for both precisions
  if (c->opts.spmv_window == 1) {
    std::vector<int32_t> rows_h(grid + 1);
    check_cuda(cudaMemcpyAsync(rows_h.data(), c->cta_rows, sizeof(int32_t) * (grid + 1), cudaMemcpyDeviceToHost, s),
               "d2h");
    check_cuda(cudaStreamSynchronize(s), "row partition");
    auto alloc = [](void* ctx, size_t bytes) -> void* { return static_cast<sfairsc_ctx*>(ctx)->dalloc<unsigned char>(bytes); };
    const int bs[3] = {1, 2, 4};
    for (int i = 0; i < 3; ++i) {
      const int vs = c->vt == VecType::F64 ? 8 : 4;
      const size_t base = operator_smem_bytes(threads, h, bs[i], c->vt);
      c->op.win[i] = build_window_table(n, c->row_ptr, c->col, rows_h, window_rows_for(bs[i], vs, base), bs[i] * vs,
                                        alloc, c, s);
      if (c->vt == VecType::F64) {
        c->op64.win[i] = c->op.win[i];
      } else {
        const size_t base64 = operator_smem_bytes(threads, h, bs[i], VecType::F64);
        c->op64.win[i] = build_window_table(n, c->row_ptr, c->col, rows_h, window_rows_for(bs[i], 8, base64),
                                            bs[i] * 8, alloc, c, s);
      }
    }
  }

  // Krylov basis
  c->B = std::max(1, std::min(SFAIRSC_MAX_BLOCK, c->opts.block));
  if (c->B == 3) c->B = 4;
  // default basis: max(2k, 20) (the eigs default), and at least 10 b so that a block cycle still
  // adds several blocks after a thick restart
  int m = c->opts.basis > 0 ? c->opts.basis : std::max({2 * c->k, 20, 10 * c->B});
  m = std::max(m, c->k + c->B);
  m = (m + c->B - 1) / c->B * c->B;
  const int mcap = (n / c->B) * c->B - c->B;
  if (m > mcap) m = mcap;
  if (m < c->k + c->B || m + c->B > 256) {
    if (m + c->B > 256) fail(SFAIRSC_ERR_UNSUPPORTED, "Krylov basis larger than 252 columns");
    fail(SFAIRSC_ERR_K_TOO_LARGE, "graph too small for k and the block size");
  }
  c->m = m;
  c->ldv = (m + c->B + 3) / 4 * 4;
  c->ldh = m + c->B;
  c->V = c->dalloc<unsigned char>((size_t)n * c->ldv * vs);
  c->U = c->dalloc<unsigned char>((size_t)n * 4 * vs);
  c->Q = c->dalloc<unsigned char>((size_t)n * 4 * vs);
  check_cuda(cudaMemsetAsync(c->U, 0, (size_t)n * 4 * vs, s), "memset");
  check_cuda(cudaMemsetAsync(c->Q, 0, (size_t)n * 4 * vs, s), "memset");
  c->Hd = c->dalloc<double>((size_t)c->ldh * m);
  c->Yd = c->dalloc<double>((size_t)m * m);
  if (c->vt == VecType::F32) c->Ytc = c->dalloc<float>(2 * (size_t)((c->ldv + 7) / 8 * 8) * 256);
  const int ogmax = orth_max_grid(c->vt, c->B, 512);
  const int ogrid = std::max(1, std::min(ogmax, (n + 511) / 512));
  const int stride = 2 * 128 * 4 + 4 + 32;
  c->orth_partial = c->dalloc<double>((size_t)ogrid * stride);
  c->orth_coef = c->dalloc<double>(2 * 128 * 4);
  c->cta_rows_orth = c->dalloc<int32_t>(ogrid + 1);
  std::vector<int32_t> orows(ogrid + 1);
  for (int t = 0; t <= ogrid; ++t) orows[t] = (int32_t)((long long)t * n / ogrid);
  check_cuda(cudaMemcpyAsync(c->cta_rows_orth, orows.data(), sizeof(int32_t) * (ogrid + 1), cudaMemcpyHostToDevice, s),
             "h2d");
  OrthPlan& q = c->orth;
  q.n = n;
  q.grid = ogrid;
  q.threads = 512;
  q.ldv = c->ldv;
  q.V = c->V;
  q.U = c->U;
  q.Q = c->Q;
  q.H = c->Hd;
  q.ldh = c->ldh;
  q.partial = c->orth_partial;
  q.coef = c->orth_coef;
  q.cta_rows = c->cta_rows_orth;
  q.barrier = reinterpret_cast<unsigned long long*>(c->barrier + 8);
  q.err = c->err;
  q.brk_step = c->brk_step;
  q.sweeps = c->sweeps;
  q.wait_ns = wait_ns;
  q.pend = c->dalloc<double>(256 * 4);
  c->hh_bytes = sizeof(double) * c->ldh * m;
  c->yh_bytes = c->ys_bytes = sizeof(double) * m * m;
  c->Hh = static_cast<double*>(pinned_get(c->hh_bytes));
  c->Yh = static_cast<double*>(pinned_get(c->yh_bytes));
  c->Ystage = pinned_get(c->ys_bytes);

  // final-stage buffers
  const int k = c->k;
  c->X64 = c->dalloc<double>((size_t)n * k);
  c->AX64 = c->dalloc<double>((size_t)n * k);
  c->Hres = c->dalloc<double>((size_t)n * k);
  c->lam_d = c->dalloc<double>(k);
  c->stat_blocks = std::max(1, std::min(2 * c->sms, (n + 1023) / 1024));
  c->stat_partial = c->dalloc<double>((size_t)c->stat_blocks * k * 3);
  c->colkey = c->dalloc<unsigned long long>(2 * (size_t)k);
  c->diag_blocks = std::max(1, std::min(2 * c->sms, (n + 1023) / 1024));
  c->diag_partial = c->dalloc<double>((size_t)c->diag_blocks * ((size_t)h * k + (size_t)k * k));
  if (dense && h > 1) c->fth_partial = c->dalloc<double>((size_t)c->diag_blocks * (h - 1) * k);
  c->bw_blocks = std::max(1, std::min(8 * c->sms, (n + 7) / 8));
  c->bw_partial = c->dalloc<double>(c->bw_blocks);
  c->bw_A = c->dalloc<double>(n);
  c->bw_Hp = c->dalloc<double>((size_t)n * backward_padded_width(k));
  c->labels_d = c->dalloc<int32_t>(n);
  check_cuda(cudaStreamSynchronize(s), "create");
}

void check_err_word(sfairsc_ctx* c) {
  unsigned e = 0;
  check_cuda(cudaMemcpyAsync(&e, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream), "d2h");
  check_cuda(cudaStreamSynchronize(c->stream), "sync");
  if (e) {
    check_cuda(cudaMemsetAsync(c->barrier, 0, 16 * sizeof(unsigned), c->stream), "memset");
    check_cuda(cudaStreamSynchronize(c->stream), "sync");
    if (e & kErrBarrierTimeout) fail(SFAIRSC_ERR_DEVICE_TIMEOUT, "a grid barrier timed out");
  }
}

void apply_op(sfairsc_ctx* c, bool fp64, const void* w, int64_t wrs, int64_t wcs, void* out, int64_t ors, int64_t ocs,
              int nvec) {
  OpPlan p = fp64 ? c->op64 : c->op;
  if (c->fault_pending) {  // testing hook: word 12 of the counter block is zero and nothing writes it
    p.stall_flag = c->barrier + 12;
    c->fault_pending = false;
  }
  const bool timed = c->opts.profile && !fp64;
  cudaEvent_t a = nullptr, b = nullptr;
  if (timed) {
    a = c->take_event();
    b = c->take_event();
    check_cuda(cudaEventRecord(a, c->stream), "event record");
  }
  launch_operator(p, fp64 ? VecType::F64 : c->vt, w, wrs, wcs, out, ors, ocs, nvec, c->stream);
  c->n_launches += (nvec + 3) / 4 + ((nvec & 3) == 3 ? 1 : 0);
  if (timed) {
    check_cuda(cudaEventRecord(b, c->stream), "event record");
    c->ev_op.emplace_back(a, b);
  }
}

void orth(sfairsc_ctx* c, int J, int j, bool pend_in = false, bool defer = false) {
  const bool timed = c->opts.profile != 0;
  cudaEvent_t a = nullptr, b = nullptr;
  if (timed) {
    a = c->take_event();
    b = c->take_event();
    check_cuda(cudaEventRecord(a, c->stream), "event record");
  }
  launch_orth(c->orth, c->vt, J, j, c->B, pend_in, defer, c->stream);
  c->n_launches += 1;
  if (timed) {
    check_cuda(cudaEventRecord(b, c->stream), "event record");
    c->ev_orth.emplace_back(a, b);
  }
}

// Sum and recycle the recorded event pairs (the stream must be synchronised).
float drain_events(sfairsc_ctx* c, std::vector<std::pair<cudaEvent_t, cudaEvent_t>>& v) {
  float tot = 0.f;
  for (auto& pr : v) {
    float ms = 0.f;
    check_cuda(cudaEventElapsedTime(&ms, pr.first, pr.second), "event time");
    tot += ms;
    c->ev_pool.push_back(pr.first);
    c->ev_pool.push_back(pr.second);
  }
  v.clear();
  return tot;
}

struct Timer {
  cudaEvent_t a, b;
  explicit Timer(cudaStream_t s) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s);
  }
  float stop(cudaStream_t s) {
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms;
  }
};

// Y[:, 0:cols] (host, c->Yh, column-major mv x cols) to the device, row-major
// (row q = basis column q, cols entries) in the basis precision: c->Yd holds
// doubles, or floats in its first half for the FP32 basis.
void upload_y(sfairsc_ctx* c, int mv, int cols) {
  const size_t cnt = (size_t)mv * cols;
  if (c->vt == VecType::F64) {
    double* st = static_cast<double*>(c->Ystage);
    for (int q = 0; q < mv; ++q)
      for (int i = 0; i < cols; ++i) st[(size_t)q * cols + i] = c->Yh[(size_t)i * mv + q];
    check_cuda(cudaMemcpyAsync(c->Yd, st, sizeof(double) * cnt, cudaMemcpyHostToDevice, c->stream), "h2d");
  } else {
    float* st = static_cast<float*>(c->Ystage);
    for (int q = 0; q < mv; ++q)
      for (int i = 0; i < cols; ++i) st[(size_t)q * cols + i] = (float)c->Yh[(size_t)i * mv + q];
    check_cuda(cudaMemcpyAsync(c->Yd, st, sizeof(float) * cnt, cudaMemcpyHostToDevice, c->stream), "h2d");
  }
}

// FP64 Ritz vectors X = V[:, 0:mv] Y[:, 0:k] -> project X <- P X (exact F^T H = 0)
// -> AX = L_n^sigma X with the FP64 operator -> Rayleigh quotients and explicit
// residual norms ||A x - lambda x|| / ||x||.  V is left untouched.
double final_check(sfairsc_ctx* c, int mv, const std::vector<double>& T, std::vector<double>& xx) {
  cudaStream_t s = c->stream;
  const int n = (int)c->n, k = c->k;
  for (int i = 0; i < k; ++i)
    for (int q = 0; q < mv; ++q) c->Yh[(size_t)i * mv + q] = T[(size_t)i * mv + q];
  upload_y(c, mv, k);
  launch_ritz(c->vt, n, c->V, c->ldv, mv, k, c->Yd, c->AX64, s);
  c->n_launches += 3 + (k + 3) / 4;
  for (int i = 0; i < k; i += 4) {
    const int nv = std::min(4, k - i);
    launch_operator(c->proj64, VecType::F64, c->AX64 + (size_t)i * n, 1, n, c->X64 + (size_t)i * n, 1, n, nv, s);
  }
  if (c->vt == VecType::F32) {
    // X lies in null(C^T) (projected just above), so A X = P (L_n X): the SpMV in double-float on
    // the FP32 pipe (FP64-grade), then the FP64 projection
    // eight vectors per SpMV (one pass over the edges and one gather per entry for eight columns),
    // the FP64 projection four at a time
    for (int i = 0; i < k;) {
      const int nv = k - i >= 8 ? 8 : std::min(4, k - i);
      launch_df_spmv(n, c->row_ptr, c->col, c->val_orig, c->vdt_orig, c->dinv64, c->deg, c->normalized,
                     c->op64.lanes_per_row, c->X64 + (size_t)i * n, nv, c->ytil64, c->dfT, c->sms, s);
      for (int q = 0; q < nv; q += 4)
        launch_operator(c->proj64, VecType::F64, c->dfT + (size_t)q * n, 1, n, c->AX64 + (size_t)(i + q) * n, 1, n,
                        std::min(4, nv - q), s);
      c->n_launches += 2 + (nv + 3) / 4;
      i += nv;
    }
  } else {
    for (int i = 0; i < k; i += 4) {
      const int nv = std::min(4, k - i);
      apply_op(c, true, c->X64 + (size_t)i * n, 1, n, c->AX64 + (size_t)i * n, 1, n, nv);
    }
  }
  launch_column_stats(n, k, c->X64, c->AX64, nullptr, c->stat_partial, c->stat_blocks, nullptr, s);
  std::vector<double> st((size_t)c->stat_blocks * k * 3);
  check_cuda(cudaMemcpyAsync(st.data(), c->stat_partial, st.size() * sizeof(double), cudaMemcpyDeviceToHost, s), "d2h");
  check_err_word(c);
  std::vector<double> xay(k, 0.0);
  xx.assign(k, 0.0);
  for (int b = 0; b < c->stat_blocks; ++b)
    for (int i = 0; i < k; ++i) {
      xay[i] += st[((size_t)b * k + i) * 3 + 0];
      xx[i] += st[((size_t)b * k + i) * 3 + 1];
    }
  // A unit Ritz vector that keeps less than half of its norm under P lies
  // mostly in range(C), the eigenspace of sigma (Prop. 3.2): sigma is not above
  // the wanted eigenvalues (Prop. 3.3).  Its eigenvalue is reported as sigma.
  c->lam_h.assign(k, 0.0);
  c->shift_found = false;
  std::vector<char> in_range_c(k, 0);
  for (int i = 0; i < k; ++i) {
    if (xx[i] < 0.25) {
      in_range_c[i] = 1;
      c->shift_found = true;
      xay[i] = c->sigma;
      xx[i] = 1.0;
    }
    c->lam_h[i] = xay[i] / xx[i];
  }
  check_cuda(cudaMemcpyAsync(c->lam_d, c->lam_h.data(), sizeof(double) * k, cudaMemcpyHostToDevice, s), "h2d");
  launch_column_resid(n, k, c->X64, c->AX64, c->lam_d, c->stat_partial, c->stat_blocks, s);
  std::vector<double> rp((size_t)c->stat_blocks * k);
  check_cuda(cudaMemcpyAsync(rp.data(), c->stat_partial, rp.size() * sizeof(double), cudaMemcpyDeviceToHost, s), "d2h");
  check_cuda(cudaStreamSynchronize(s), "residual");
  double maxres = 0.0;
  for (int i = 0; i < k; ++i) {
    if (in_range_c[i]) continue;
    double r2 = 0.0;
    for (int b = 0; b < c->stat_blocks; ++b) r2 += rp[(size_t)b * k + i];
    maxres = std::max(maxres, std::sqrt(r2 / xx[i]) / c->sigma);
  }
  return maxres;
}

int solve_impl(sfairsc_ctx* c, double* eigenvalues, double* Hout, int32_t* labels, sfairsc_info* info) {
  cudaStream_t s = c->stream;
  const int n = (int)c->n, k = c->k, B = c->B, m = c->m, ldh = c->ldh;
  const int kNoBreak = std::numeric_limits<int>::max();
  sfairsc_info inf{};
  inf.sigma = c->sigma;
  Timer tsolve(s);
  c->n_launches = 0;
  int n_op = 0, n_orth = 0, orth_cols = 0, eig_fallbacks = 0;
  float ms_op = 0.f, ms_orth = 0.f, ms_restart = 0.f;
  double ms_eig = 0.0;
  check_cuda(cudaMemsetAsync(c->sweeps, 0, sizeof(int), s), "memset");
  launch_random_block(c->vt, n, c->U, 4, B, c->opts.seed, s);
  orth(c, 0, -1);
  c->n_launches += 1;
  check_cuda(cudaMemsetAsync(c->Hd, 0, sizeof(double) * ldh * m, s), "memset");
  int j0 = 0, restarts = 0, matvecs = 0, since_break = 1 << 20;
  uint64_t fresh = 0;  // counter for replacement start blocks
  std::vector<double> T, theta, resid, xx;
  double maxres = 0.0;
  bool converged = false;
  const double tol = c->opts.tol * c->sigma;
  for (;;) {
    check_cuda(cudaMemcpyAsync(c->brk_step, &kNoBreak, sizeof(int), cudaMemcpyHostToDevice, s), "h2d");
    // deferred second projection (opts.orth_mode 0): each step's new block is stored before its
    // second projection; the next step applies it in its first sweep, the restart to the carried block
    const bool defer = c->opts.orth_mode == 0;
    for (int j = j0; j < m; j += B) {
      apply_op(c, false, c->Q, 4, 1, c->U, 4, 1, B);  // Q holds V[:, j:j+B]
      orth(c, j + B, j, defer && j > j0, defer);
      orth_cols += j + B;
      matvecs += B;
      ++n_op;
      ++n_orth;
    }
    int brk = kNoBreak;
    check_cuda(cudaMemcpyAsync(c->Hh, c->Hd, sizeof(double) * ldh * m, cudaMemcpyDeviceToHost, s), "d2h");
    check_cuda(cudaMemcpyAsync(&brk, c->brk_step, sizeof(int), cudaMemcpyDeviceToHost, s), "d2h");
    check_err_word(c);  // synchronises; a breakdown is handled below, not raised
    if (c->opts.profile) {
      ms_op += drain_events(c, c->ev_op);
      ms_orth += drain_events(c, c->ev_orth);
      ms_restart += drain_events(c, c->ev_restart);
    }
    const bool broke = brk != kNoBreak;
    // basis columns 0..mv-1 are valid: a block that lost rank at step brk is dropped
    const int mv = broke ? std::max(B, std::min(m, brk + B)) : m;
    since_break = broke ? 0 : since_break + 1;
    T.assign((size_t)mv * mv, 0.0);
    theta.assign(mv, 0.0);
    resid.assign(mv, 0.0);
    for (int jj = 0; jj < mv; ++jj)
      for (int ii = 0; ii <= jj; ++ii) {
        const double v = c->Hh[(size_t)jj * ldh + ii];
        T[(size_t)jj * mv + ii] = v;
        T[(size_t)ii * mv + jj] = v;
      }
    {
      const auto t0 = std::chrono::steady_clock::now();
      const std::vector<double> T0 = T;
      if (!host_symmetric_eig(mv, T.data(), theta.data())) {
        // the QR iteration hit its sweep limit: solve the projected problem again by Jacobi
        T = T0;
        if (!host_symmetric_eig_jacobi(mv, T.data(), theta.data()))
          fail(SFAIRSC_ERR_NONFINITE, "the projected matrix holds a non-finite entry");
        ++eig_fallbacks;
      }
      ms_eig += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    for (int i = 0; i < mv; ++i) {
      double acc = 0.0;
      for (int r = 0; r < B; ++r) {
        double sr = 0.0;
        for (int q = 0; q < mv; ++q) sr += c->Hh[(size_t)q * ldh + mv + r] * T[(size_t)i * mv + q];
        acc += sr * sr;
      }
      resid[i] = std::sqrt(acc);
    }
    int nconv = 0;
    for (int i = 0; i < std::min(k, mv); ++i) nconv += resid[i] <= tol;
    const bool estimate_ok = mv >= k && nconv == k && since_break >= 1;
    const bool out_of_restarts = restarts >= c->opts.max_restarts;
    if ((estimate_ok || out_of_restarts) && mv >= k) {
      Timer tfin(s);
      maxres = final_check(c, mv, T, xx);
      inf.ms_final += tfin.stop(s);
      if (maxres <= c->opts.tol || out_of_restarts || c->shift_found) {
        converged = maxres <= c->opts.tol;
        break;
      }
      since_break = 0;  // the estimate was optimistic: verify again after another cycle
    }
    // thick restart: keep the K smallest Ritz vectors
    int K = k + (m - k) / 2;
    K = std::max(K / B * B, ((k + B - 1) / B) * B);
    K = std::min({K, m - B, mv});
    for (int i = 0; i < K; ++i)
      for (int q = 0; q < mv; ++q) c->Yh[(size_t)i * mv + q] = T[(size_t)i * mv + q];
    upload_y(c, mv, K);
    {
      cudaEvent_t ea = nullptr, eb = nullptr;
      if (c->opts.profile) {
        ea = c->take_event();
        eb = c->take_event();
        check_cuda(cudaEventRecord(ea, s), "event record");
      }
      const double* E = (c->opts.orth_mode == 0 && !broke) ? c->orth.pend : nullptr;
      if (c->vt == VecType::F32 && c->opts.restart_mode == 0 && restart_tc_fits(n, c->ldv, mv, K, B)) {
        launch_restart_tc(n, static_cast<float*>(c->V), c->ldv, mv, K, B, reinterpret_cast<const float*>(c->Yd),
                          static_cast<float*>(c->Q), E, c->Ytc, c->sms, c->err, c->orth.wait_ns, s);
        ++inf.restarts_tc;
        c->n_launches += 1;  // the split of [Y | -E]
      } else
        launch_restart(c->vt, n, c->V, c->ldv, mv, K, B, c->Yd, c->Q, E, s);
      if (c->opts.profile) {
        check_cuda(cudaEventRecord(eb, s), "event record");
        c->ev_restart.emplace_back(ea, eb);
      }
    }
    c->n_launches += 1;
    std::vector<double> Hn((size_t)ldh * m, 0.0);
    for (int i = 0; i < K; ++i) Hn[(size_t)i * ldh + i] = theta[i];
    if (broke) {
      // fresh random block orthogonal to the kept Ritz vectors (invariant subspace found)
      launch_random_block(c->vt, n, c->U, 4, B, c->opts.seed + 0x9E3779B97F4A7C15ull * (++fresh), s);
      orth(c, K, -1);
      c->n_launches += 1;
      ++n_orth;
      orth_cols += K;
    } else {
      for (int r = 0; r < B; ++r)
        for (int i = 0; i < K; ++i) {
          double sr = 0.0;
          for (int q = 0; q < mv; ++q) sr += c->Hh[(size_t)q * ldh + mv + r] * T[(size_t)i * mv + q];
          Hn[(size_t)i * ldh + K + r] = sr;
        }
    }
    std::memcpy(c->Hh, Hn.data(), sizeof(double) * ldh * m);
    check_cuda(cudaMemcpyAsync(c->Hd, c->Hh, sizeof(double) * ldh * m, cudaMemcpyHostToDevice, s), "h2d");
    j0 = K;
    ++restarts;
  }
  // order by Rayleigh quotient (Ritz order up to rounding)
  std::vector<int> ord(k);
  for (int i = 0; i < k; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return c->lam_h[a] < c->lam_h[b]; });
  bool perm = false;
  for (int i = 0; i < k; ++i) perm |= ord[i] != i;
  if (perm) {
    check_cuda(cudaMemcpyAsync(c->AX64, c->X64, sizeof(double) * n * k, cudaMemcpyDeviceToDevice, s), "d2d");
    for (int i = 0; i < k; ++i)
      check_cuda(cudaMemcpyAsync(c->X64 + (size_t)i * n, c->AX64 + (size_t)ord[i] * n, sizeof(double) * n,
                                 cudaMemcpyDeviceToDevice, s), "d2d");
    std::vector<double> l2(k), x2(k);
    for (int i = 0; i < k; ++i) {
      l2[i] = c->lam_h[ord[i]];
      x2[i] = xx[ord[i]];
    }
    c->lam_h = l2;
    xx = x2;
  }
  inf.ms_solve = tsolve.stop(s);
  inf.restarts = restarts;
  inf.matvecs = matvecs;
  inf.max_resid = maxres;
  inf.ms_operator = ms_op;
  inf.ms_orth = ms_orth;
  inf.ms_restart = ms_restart;
  inf.ms_host_eig = (float)ms_eig;
  inf.n_operator = n_op;
  inf.host_eig_fallbacks = eig_fallbacks;
  {
    const WindowTable& wt = c->op.win[B == 1 ? 0 : B == 2 ? 1 : 2];
    inf.spmv_segments = wt.nseg;
    inf.spmv_windowed = wt.windowed;
    inf.spmv_in_window = c->nnz > 0 ? (float)((double)wt.in_window / (double)c->nnz) : 0.f;
  }
  inf.n_orth = n_orth;
  inf.orth_cols = orth_cols;
  {
    int sw = 0;
    check_cuda(cudaMemcpy(&sw, c->sweeps, sizeof(int), cudaMemcpyDeviceToHost), "d2h");
    inf.orth_sweeps = sw;
  }
  inf.basis = m;
  inf.block = B;
  int status = converged ? SFAIRSC_OK : SFAIRSC_ERR_NOT_CONVERGED;
  for (int i = 0; i < k; ++i)
    if (c->lam_h[i] >= c->sigma * (1.0 - 1e-8)) status = SFAIRSC_ERR_SHIFT;
  // unit-norm columns in FP64, then H = D^{-1/2} X with the sign convention
  {
    std::vector<double> scale(k);
    for (int i = 0; i < k; ++i) scale[i] = 1.0 / std::sqrt(xx[i]);
    check_cuda(cudaMemcpyAsync(c->AX64, scale.data(), sizeof(double) * k, cudaMemcpyHostToDevice, s), "h2d");
    launch_scale_columns(n, k, c->X64, c->AX64, s);
    check_cuda(cudaStreamSynchronize(s), "sync");
  }
  launch_embed(n, k, c->X64, c->dinv64, c->normalized, c->Hres, c->colkey, s);
  c->n_launches += 6;  // scale, colkey init, colmax, argmax, embed, diagnostics
  check_cuda(cudaMemcpyAsync(c->lam_d, c->lam_h.data(), sizeof(double) * k, cudaMemcpyHostToDevice, s), "h2d");
  // diagnostics: max |F^T H| and max |H^T D H - I|
  {
    const int h = c->h;
    const bool dense = c->Fd64 != nullptr;
    const int hd = dense ? 1 : h;  // dense constraints: the label sums are unused, F^T H comes below
    launch_diagnostics(n, k, hd, c->Hres, c->deg, c->lab, c->params, c->diag_partial, c->diag_blocks, nullptr, s,
                       c->vt == VecType::F64);
    const size_t P = (size_t)hd * k + (size_t)k * k;
    std::vector<double> dg((size_t)c->diag_blocks * P);
    check_cuda(cudaMemcpyAsync(dg.data(), c->diag_partial, dg.size() * sizeof(double), cudaMemcpyDeviceToHost, s), "d2h");
    std::vector<double> fth;
    if (dense && h > 1) {
      launch_dense_fth(n, h - 1, k, c->Fd64, c->Hres, c->fth_partial, c->diag_blocks, s);
      fth.resize((size_t)c->diag_blocks * (h - 1) * k);
      check_cuda(cudaMemcpyAsync(fth.data(), c->fth_partial, fth.size() * sizeof(double), cudaMemcpyDeviceToHost, s),
                 "d2h");
    }
    check_cuda(cudaStreamSynchronize(s), "diagnostics");
    std::vector<double> acc(P, 0.0);
    for (int b = 0; b < c->diag_blocks; ++b)
      for (size_t i = 0; i < P; ++i) acc[i] += dg[(size_t)b * P + i];
    double ferr = 0.0, derr = 0.0;
    if (dense) {
      const size_t q = (size_t)(h - 1) * k;
      for (size_t i = 0; i < q; ++i) {
        double t = 0.0;
        for (int b = 0; b < c->diag_blocks; ++b) t += fth[(size_t)b * q + i];
        ferr = std::max(ferr, std::fabs(t));
      }
    } else {
      for (int i = 0; i < k; ++i) {
        double tot = 0.0;
        for (int g = 0; g < h; ++g) tot += acc[(size_t)g * k + i];
        for (int g = 0; g + 1 < h; ++g) ferr = std::max(ferr, std::fabs(acc[(size_t)g * k + i] - c->z[g] * tot));
      }
    }
    for (int a = 0; a < k; ++a)
      for (int b = a; b < k; ++b) {
        const double v = acc[(size_t)hd * k + (size_t)a * k + b];
        derr = std::max(derr, std::fabs(v - (a == b ? 1.0 : 0.0)));
      }
    inf.fairness_err = ferr;
    inf.dorth_err = derr;
  }
  if (eigenvalues) {
    if (is_device_ptr(eigenvalues))
      check_cuda(cudaMemcpyAsync(eigenvalues, c->lam_d, sizeof(double) * k, cudaMemcpyDeviceToDevice, s), "copy");
    else
      std::memcpy(eigenvalues, c->lam_h.data(), sizeof(double) * k);
  }
  // H to host memory on a side stream, so the copy runs under the k-means (which only reads H)
  cudaEvent_t h_copied = nullptr;
  if (Hout && !is_device_ptr(Hout) && labels) {
    if (!c->side) check_cuda(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking), "side stream");
    cudaEvent_t h_ready = c->take_event();
    h_copied = c->take_event();
    check_cuda(cudaEventRecord(h_ready, s), "event record");
    check_cuda(cudaStreamWaitEvent(c->side, h_ready, 0), "stream wait");
    check_cuda(cudaMemcpyAsync(Hout, c->Hres, sizeof(double) * n * k, cudaMemcpyDeviceToHost, c->side), "copy H");
    check_cuda(cudaEventRecord(h_copied, c->side), "event record");
    c->ev_pool.push_back(h_ready);  // reusable once recorded work completes (the stream is synchronised below)
  } else if (Hout) {
    check_cuda(cudaMemcpyAsync(Hout, c->Hres, sizeof(double) * n * k,
                               is_device_ptr(Hout) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s), "copy H");
  }
  if (labels) {
    Timer tk(s);
    const KmeansResult kr = run_kmeans(n, k, c->Hres, k, c->opts.kmeans_seed, c->opts.kmeans_n_init,
                                       c->opts.kmeans_max_iter, c->labels_d, nullptr, s);
    inf.kmeans_inertia = kr.inertia;
    inf.kmeans_iters = kr.iterations;
    c->n_launches += kr.launches;
    check_cuda(cudaMemcpyAsync(labels, c->labels_d, sizeof(int32_t) * n,
                               is_device_ptr(labels) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s), "copy labels");
    inf.ms_kmeans = tk.stop(s);
  }
  if (h_copied) {
    check_cuda(cudaStreamWaitEvent(s, h_copied, 0), "stream wait");
    c->ev_pool.push_back(h_copied);
  }
  check_cuda(cudaStreamSynchronize(s), "solve end");
  c->solved = true;
  inf.status = status;
  inf.ms_total = inf.ms_solve + inf.ms_kmeans;
  inf.n_launches = c->n_launches;
  if (info) *info = inf;
  return status;
}

}  // namespace

extern "C" {

const char* sfairsc_strerror(int status) {
  switch (status) {
    case SFAIRSC_OK: return "ok";
    case SFAIRSC_ERR_INVALID_ARG: return "invalid argument";
    case SFAIRSC_ERR_BAD_CSR: return "invalid CSR structure";
    case SFAIRSC_ERR_ISOLATED_VERTEX: return "isolated vertex (zero degree)";
    case SFAIRSC_ERR_EMPTY_GROUP: return "empty group";
    case SFAIRSC_ERR_K_TOO_LARGE: return "k too large for the graph";
    case SFAIRSC_ERR_NONFINITE: return "non-finite input";
    case SFAIRSC_ERR_NOT_CONVERGED: return "eigensolver did not converge";
    case SFAIRSC_ERR_SHIFT: return "shift sigma not above the wanted eigenvalues";
    case SFAIRSC_ERR_CUDA: return "CUDA error";
    case SFAIRSC_ERR_OOM: return "out of memory";
    case SFAIRSC_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
    case SFAIRSC_ERR_UNSUPPORTED: return "unsupported configuration";
    case SFAIRSC_ERR_BREAKDOWN: return "Krylov block lost rank";
    default: return "unknown status";
  }
}

const char* sfairsc_last_error(void) { return g_last_error.c_str(); }

int sfairsc_opts_default(sfairsc_opts* o) {
  if (!o) return SFAIRSC_ERR_INVALID_ARG;
  std::memset(o, 0, sizeof(*o));
  o->sigma = std::numeric_limits<double>::quiet_NaN();
  o->tol = 1e-6;
  o->max_restarts = 200;
  o->basis = 0;
  o->prec = SFAIRSC_PREC_MIXED;
  o->block = 1;
  o->seed = 1;
  o->kmeans_seed = 0;
  o->kmeans_n_init = 1;
  o->kmeans_max_iter = 100;
  o->validate = 1;
  return SFAIRSC_OK;
}

static bool valid_opts(const sfairsc_opts& o) {
  return o.tol > 0.0 && o.max_restarts >= 0 && o.block >= 1 && o.block <= SFAIRSC_MAX_BLOCK && o.kmeans_n_init >= 1 &&
         o.kmeans_max_iter >= 1 && (o.prec == 0 || o.prec == 1) && o.wait_limit_us >= 0 &&
         (o.fault_inject == 0 || o.fault_inject == 1) && (o.spmv_window == 0 || o.spmv_window == 1) &&
         (o.orth_mode == 0 || o.orth_mode == 1) && (o.restart_mode == 0 || o.restart_mode == 1);
}

int sfairsc_create(sfairsc_ctx** out, int64_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx,
                   const void* values, int32_t value_dtype, const int32_t* group_labels, int32_t h, int32_t k,
                   int32_t normalized, const sfairsc_opts* opts, void* cuda_stream) {
  if (!out) return SFAIRSC_ERR_INVALID_ARG;
  *out = nullptr;
  if (n < 2 || n > (1ll << 30) || nnz < 1 || nnz > 0x7fffffffll || !row_ptr || !col_idx || !values || !group_labels ||
      h < 1 || k < 1 || (value_dtype != SFAIRSC_F64 && value_dtype != SFAIRSC_F32 && value_dtype != SFAIRSC_BF16)) {
    g_last_error = "invalid argument to sfairsc_create";
    return SFAIRSC_ERR_INVALID_ARG;
  }
  if (h > SFAIRSC_MAX_GROUPS) {
    g_last_error = "h exceeds 32 groups";
    return SFAIRSC_ERR_UNSUPPORTED;
  }
  std::unique_ptr<sfairsc_ctx> c(new (std::nothrow) sfairsc_ctx());
  if (!c) return SFAIRSC_ERR_OOM;
  sfairsc_opts_default(&c->opts);
  if (opts) c->opts = *opts;
  if (!valid_opts(c->opts)) {
    g_last_error = "invalid options";
    return SFAIRSC_ERR_INVALID_ARG;
  }
  c->n = n;
  c->nnz = nnz;
  c->h = h;
  c->k = k;
  c->normalized = normalized ? 1 : 0;
  c->vdt_orig = value_dtype;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->vt = c->opts.prec == SFAIRSC_PREC_FP64 ? VecType::F64 : VecType::F32;
  const int rc = guarded([&] { build_context(c.get(), row_ptr, col_idx, values, group_labels); });
  if (rc != SFAIRSC_OK) return rc;
  *out = c.release();
  return SFAIRSC_OK;
}

int sfairsc_create_dense(sfairsc_ctx** out, int64_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx,
                         const void* values, int32_t value_dtype, const double* F, int32_t p, int32_t k,
                         int32_t normalized, const sfairsc_opts* opts, void* cuda_stream) {
  if (!out) return SFAIRSC_ERR_INVALID_ARG;
  *out = nullptr;
  if (n < 2 || n > (1ll << 30) || nnz < 1 || nnz > 0x7fffffffll || !row_ptr || !col_idx || !values || p < 0 ||
      (p > 0 && !F) || k < 1 ||
      (value_dtype != SFAIRSC_F64 && value_dtype != SFAIRSC_F32 && value_dtype != SFAIRSC_BF16)) {
    g_last_error = "invalid argument to sfairsc_create_dense";
    return SFAIRSC_ERR_INVALID_ARG;
  }
  if (p + 1 > SFAIRSC_MAX_GROUPS) {
    g_last_error = "more than 31 constraint columns";
    return SFAIRSC_ERR_UNSUPPORTED;
  }
  std::unique_ptr<sfairsc_ctx> c(new (std::nothrow) sfairsc_ctx());
  if (!c) return SFAIRSC_ERR_OOM;
  sfairsc_opts_default(&c->opts);
  if (opts) c->opts = *opts;
  if (!valid_opts(c->opts)) {
    g_last_error = "invalid options";
    return SFAIRSC_ERR_INVALID_ARG;
  }
  c->n = n;
  c->nnz = nnz;
  c->h = p + 1;
  c->k = k;
  c->normalized = normalized ? 1 : 0;
  c->vdt_orig = value_dtype;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->vt = c->opts.prec == SFAIRSC_PREC_FP64 ? VecType::F64 : VecType::F32;
  static const double kNoColumns = 0.0;
  const int rc = guarded([&] { build_context(c.get(), row_ptr, col_idx, values, nullptr, p > 0 ? F : &kNoColumns); });
  if (rc != SFAIRSC_OK) return rc;
  *out = c.release();
  return SFAIRSC_OK;
}

int sfairsc_destroy(sfairsc_ctx* ctx) {
  if (!ctx) return SFAIRSC_OK;
  cudaStreamSynchronize(ctx->stream);
  delete ctx;
  return SFAIRSC_OK;
}

int sfairsc_get_sigma(const sfairsc_ctx* ctx, double* sigma) {
  if (!ctx || !sigma) return SFAIRSC_ERR_INVALID_ARG;
  *sigma = ctx->sigma;
  return SFAIRSC_OK;
}

int sfairsc_apply_operator(sfairsc_ctx* ctx, const void* w, void* out, int32_t nvec) {
  if (!ctx || !w || !out || nvec < 1 || nvec > SFAIRSC_MAX_BLOCK) return SFAIRSC_ERR_INVALID_ARG;
  return guarded([&] {
    const size_t vs = ctx->vt == VecType::F64 ? 8 : 4;
    const size_t bytes = (size_t)ctx->n * nvec * vs;
    const bool wd = is_device_ptr(w), od = is_device_ptr(out);
    const void* win = w;
    void* wout = out;
    void* tmp_in = nullptr;
    void* tmp_out = nullptr;
    if (!wd) {
      check_cuda(cudaMallocAsync(&tmp_in, bytes, ctx->stream), "allocation");
      check_cuda(cudaMemcpyAsync(tmp_in, w, bytes, cudaMemcpyHostToDevice, ctx->stream), "h2d");
      win = tmp_in;
    }
    if (!od) {
      check_cuda(cudaMallocAsync(&tmp_out, bytes, ctx->stream), "allocation");
      wout = tmp_out;
    }
    apply_op(ctx, false, win, 1, ctx->n, wout, 1, ctx->n, nvec);
    if (!od) check_cuda(cudaMemcpyAsync(out, tmp_out, bytes, cudaMemcpyDeviceToHost, ctx->stream), "d2h");
    if (tmp_in) cudaFreeAsync(tmp_in, ctx->stream);
    if (tmp_out) cudaFreeAsync(tmp_out, ctx->stream);
    if (!wd || !od) check_err_word(ctx);
  });
}

int sfairsc_solve(sfairsc_ctx* ctx, double* eigenvalues, double* H, int32_t* labels, sfairsc_info* info) {
  if (!ctx) return SFAIRSC_ERR_INVALID_ARG;
  int status = SFAIRSC_OK;
  const int rc = guarded([&] { status = solve_impl(ctx, eigenvalues, H, labels, info); });
  if (rc != SFAIRSC_OK) {
    if (info) info->status = rc;
    return rc;
  }
  return status;
}

int sfairsc_kmeans(int64_t n, int32_t d, const double* X, int32_t kc, uint64_t seed, int32_t n_init, int32_t max_iter,
                   int32_t* labels, double* centroids, double* inertia, int32_t* iterations, void* cuda_stream) {
  if (!X || !labels || n < 1 || d < 1 || kc < 1 || kc > n || n_init < 1 || max_iter < 1) return SFAIRSC_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  return guarded([&] {
    std::vector<void*> tmp;
    auto dev = [&](size_t bytes) {
      void* p = nullptr;
      check_cuda(cudaMallocAsync(&p, std::max<size_t>(bytes, 1), s), "allocation");
      tmp.push_back(p);
      return p;
    };
    const double* Xd = X;
    if (!is_device_ptr(X)) {
      void* p = dev(sizeof(double) * n * d);
      check_cuda(cudaMemcpyAsync(p, X, sizeof(double) * n * d, cudaMemcpyHostToDevice, s), "h2d");
      Xd = static_cast<const double*>(p);
    }
    const bool ld = is_device_ptr(labels);
    int32_t* Ld = ld ? labels : static_cast<int32_t*>(dev(sizeof(int32_t) * n));
    const bool cd = centroids && is_device_ptr(centroids);
    double* Cd = centroids ? (cd ? centroids : static_cast<double*>(dev(sizeof(double) * kc * d))) : nullptr;
    const KmeansResult r = run_kmeans(n, d, Xd, kc, seed, n_init, max_iter, Ld, Cd, s);
    if (!ld) check_cuda(cudaMemcpyAsync(labels, Ld, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s), "d2h");
    if (centroids && !cd) check_cuda(cudaMemcpyAsync(centroids, Cd, sizeof(double) * kc * d, cudaMemcpyDeviceToHost, s), "d2h");
    check_cuda(cudaStreamSynchronize(s), "k-means");
    for (void* p : tmp) cudaFreeAsync(p, s);
    check_cuda(cudaStreamSynchronize(s), "k-means free");
    if (inertia) *inertia = r.inertia;
    if (iterations) *iterations = r.iterations;
  });
}

int sfairsc_backward(sfairsc_ctx* ctx, const double* grad_lambda, double* grad_values, double bandwidth,
                     double* grad_bandwidth) {
  if (!ctx || !grad_lambda || !grad_values) return SFAIRSC_ERR_INVALID_ARG;
  if (!ctx->solved) {
    g_last_error = "sfairsc_backward needs a prior sfairsc_solve";
    return SFAIRSC_ERR_INVALID_ARG;
  }
  return guarded([&] {
    cudaStream_t s = ctx->stream;
    const int k = ctx->k;
    std::vector<void*> tmp;
    const double* gd = grad_lambda;
    if (!is_device_ptr(grad_lambda)) {
      void* p = nullptr;
      check_cuda(cudaMallocAsync(&p, sizeof(double) * k, s), "allocation");
      tmp.push_back(p);
      check_cuda(cudaMemcpyAsync(p, grad_lambda, sizeof(double) * k, cudaMemcpyHostToDevice, s), "h2d");
      gd = static_cast<const double*>(p);
    }
    const bool od = is_device_ptr(grad_values);
    double* G = grad_values;
    if (!od) {
      void* p = nullptr;
      check_cuda(cudaMallocAsync(&p, sizeof(double) * ctx->nnz, s), "allocation");
      tmp.push_back(p);
      G = static_cast<double*>(p);
    }
    const double bw = grad_bandwidth ? bandwidth : 0.0;
    launch_backward((int)ctx->n, ctx->row_ptr, ctx->col, ctx->val_orig, ctx->vdt_orig, k, ctx->Hres, ctx->lam_d, gd, G,
                    bw, ctx->bw_partial, ctx->bw_blocks, ctx->bw_A, ctx->bw_Hp, ctx->normalized, s);
    if (!od) check_cuda(cudaMemcpyAsync(grad_values, G, sizeof(double) * ctx->nnz, cudaMemcpyDeviceToHost, s), "d2h");
    std::vector<double> part(ctx->bw_blocks);
    check_cuda(cudaMemcpyAsync(part.data(), ctx->bw_partial, sizeof(double) * ctx->bw_blocks, cudaMemcpyDeviceToHost, s),
               "d2h");
    check_cuda(cudaStreamSynchronize(s), "backward");
    for (void* p : tmp) cudaFreeAsync(p, s);
    if (grad_bandwidth) {
      double acc = 0.0;
      for (double v : part) acc += v;
      *grad_bandwidth = bw > 0.0 ? acc / bw : 0.0;  // the kernel sums g_e w_e (-2 ln w_e); dw/ds has the 1/s
    }
    check_cuda(cudaStreamSynchronize(s), "backward end");
  });
}

int sfairsc_backward_vectors(sfairsc_ctx* ctx, const double* grad_H, const double* grad_lambda, double* grad_values,
                             double bandwidth, double* grad_bandwidth, int32_t max_iter, double rtol,
                             int32_t* iterations, double* max_rel_resid) {
  if (!ctx || !grad_H || !grad_values) return SFAIRSC_ERR_INVALID_ARG;
  if (!ctx->solved) {
    g_last_error = "sfairsc_backward_vectors needs a prior sfairsc_solve";
    return SFAIRSC_ERR_INVALID_ARG;
  }
  if (ctx->k > 64 || !ctx->normalized) {
    g_last_error = "the eigenvector-level backward supports the normalized problem with k <= 64";
    return SFAIRSC_ERR_UNSUPPORTED;
  }
  if (ctx->opts.prec != SFAIRSC_PREC_FP64) {
    // the solves below deflate with the computed eigenvectors: FP32-accurate ones leave components of
    // lower eigenvectors in the complement, where A - lambda_i I is then indefinite
    g_last_error = "the eigenvector-level backward needs the eigenvectors of an FP64 solve";
    return SFAIRSC_ERR_UNSUPPORTED;
  }
  int status = SFAIRSC_OK;
  const int rc = guarded([&] {
    cudaStream_t s = ctx->stream;
    const int n = (int)ctx->n, k = ctx->k;
    const int iters_max = max_iter > 0 ? max_iter : 1000;
    const double tol = rtol > 0.0 ? rtol : 1e-10;
    const std::vector<double>& lam = ctx->lam_h;
    for (int i = 0; i < k; ++i)
      for (int j = i + 1; j < k; ++j)
        if (std::fabs(lam[i] - lam[j]) <= 1e-12 * ctx->sigma)
          fail(SFAIRSC_ERR_INVALID_ARG, "repeated eigenvalue: its eigenvectors are not differentiable");
    std::vector<void*> tmp;
    auto dev = [&](size_t bytes) {
      void* p = nullptr;
      check_cuda(cudaMallocAsync(&p, std::max<size_t>(bytes, 8), s), "allocation");
      tmp.push_back(p);
      return static_cast<double*>(p);
    };
    const size_t nk = (size_t)n * k;
    const double* G = grad_H;
    if (!is_device_ptr(grad_H)) {
      double* d = dev(sizeof(double) * nk);
      check_cuda(cudaMemcpyAsync(d, grad_H, sizeof(double) * nk, cudaMemcpyHostToDevice, s), "h2d");
      G = d;
    }
    double* glam = nullptr;
    if (grad_lambda) {
      glam = dev(sizeof(double) * k);
      check_cuda(cudaMemcpyAsync(glam, grad_lambda, sizeof(double) * k,
                                 is_device_ptr(grad_lambda) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s),
                 "copy");
    }
    double *X = dev(8 * nk), *B0 = dev(8 * nk), *Bp = dev(8 * nk), *Zc = dev(8 * nk), *Y = dev(8 * nk),
           *R = dev(8 * nk), *P = dev(8 * nk), *Q = dev(8 * nk);
    const int nb = std::max(1, std::min(2 * ctx->sms, (n + 63) / 64));
    double* part = dev(sizeof(double) * nb * k * k);
    double* small = dev(sizeof(double) * (3 * k + k * k));  // alpha / beta / ones, k x k coefficients
    std::vector<double> hpart((size_t)nb * k * k);
    auto gram = [&](const double* A, const double* Bm) {  // A^T Bm (k x k, [i][j] = A_i . Bm_j), summed in block order
      launch_col_gram(n, k, A, k, Bm, part, nb, s);
      check_cuda(cudaMemcpyAsync(hpart.data(), part, sizeof(double) * nb * k * k, cudaMemcpyDeviceToHost, s), "d2h");
      check_cuda(cudaStreamSynchronize(s), "gram");
      std::vector<double> T((size_t)k * k, 0.0);
      for (int b = 0; b < nb; ++b)
        for (int q = 0; q < k * k; ++q) T[q] += hpart[(size_t)b * k * k + q];
      return T;
    };
    auto dots = [&](const double* A, const double* Bm) {
      launch_col_dots(n, k, A, Bm, part, nb, s);
      check_cuda(cudaMemcpyAsync(hpart.data(), part, sizeof(double) * nb * k, cudaMemcpyDeviceToHost, s), "d2h");
      check_cuda(cudaStreamSynchronize(s), "dots");
      std::vector<double> d(k, 0.0);
      for (int b = 0; b < nb; ++b)
        for (int i = 0; i < k; ++i) d[i] += hpart[(size_t)b * k + i];
      return d;
    };
    auto upload = [&](const std::vector<double>& v, double* dst) {
      check_cuda(cudaMemcpyAsync(dst, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice, s), "h2d");
    };
    auto right_mul = [&](const double* A, const std::vector<double>& C, double beta, double* out) {
      std::vector<double> Cc(C);
      upload(Cc, small + 3 * k);
      launch_col_gemm(n, k, A, k, small + 3 * k, beta, out, s);
      check_cuda(cudaStreamSynchronize(s), "right product");  // the coefficient slot is reused next
    };
    // X = D^{1/2} H (unit columns, the returned signs); B0 = D^{-1/2} Gbar; Bp = P B0
    launch_rows_to_cols_scaled(n, k, ctx->Hres, ctx->dinv64, 1, X, s);
    launch_rows_to_cols_scaled(n, k, G, ctx->dinv64, 0, B0, s);
    launch_operator(ctx->proj64, VecType::F64, B0, 1, n, Bp, 1, n, k, s);
    // the computed eigenvectors' part: z_i = sum_{j != i} x_j (x_j^T b_i) / (lambda_i - lambda_j)
    std::vector<double> T = gram(X, Bp);  // T[j][i] = x_j . b_i
    std::vector<double> Ck((size_t)k * k, 0.0), mT((size_t)k * k);
    for (int j = 0; j < k; ++j)
      for (int i = 0; i < k; ++i) {
        if (i != j) Ck[(size_t)j * k + i] = T[(size_t)j * k + i] / (lam[i] - lam[j]);
        mT[(size_t)j * k + i] = -T[(size_t)j * k + i];
      }
    right_mul(X, Ck, 0.0, Zc);
    // the rest: (A - lambda_i) y_i = (I - X X^T) b_i on the complement, where it is positive definite
    check_cuda(cudaMemcpyAsync(R, Bp, 8 * nk, cudaMemcpyDeviceToDevice, s), "copy");
    right_mul(X, mT, 1.0, R);
    check_cuda(cudaMemsetAsync(Y, 0, 8 * nk, s), "memset");
    check_cuda(cudaMemcpyAsync(P, R, 8 * nk, cudaMemcpyDeviceToDevice, s), "copy");
    std::vector<double> rho = dots(R, R), bnorm(k), coef(k);
    for (int i = 0; i < k; ++i) bnorm[i] = std::sqrt(rho[i]);
    upload(lam, small + 2 * k);  // the shifts
    std::vector<char> done(k, 0);
    int it = 0;
    double worst = 0.0;
    for (; it < iters_max; ++it) {
      worst = 0.0;
      bool all = true;
      for (int i = 0; i < k; ++i) {
        const double rr = bnorm[i] > 0.0 ? std::sqrt(rho[i]) / bnorm[i] : 0.0;
        done[i] = rr <= tol;
        worst = std::max(worst, rr);
        all = all && done[i];
      }
      if (all) break;
      apply_op(ctx, true, P, 1, n, Q, 1, n, k);
      launch_col_shift(n, k, Q, P, small + 2 * k, s);
      std::vector<double> Tq = gram(X, Q);
      for (double& v : Tq) v = -v;
      right_mul(X, Tq, 1.0, Q);
      std::vector<double> pq = dots(P, Q);
      for (int i = 0; i < k; ++i) coef[i] = (done[i] || !(pq[i] > 0.0)) ? 0.0 : rho[i] / pq[i];
      upload(coef, small);
      launch_cg_update(n, k, Y, R, P, Q, small, s);
      std::vector<double> rn = dots(R, R);
      for (int i = 0; i < k; ++i) {
        coef[i] = done[i] || rho[i] == 0.0 ? 0.0 : rn[i] / rho[i];
        rho[i] = rn[i];
      }
      upload(coef, small + k);
      launch_cg_direction(n, k, P, R, small + k, s);
    }
    check_err_word(ctx);
    // z_i = known part - y_i; c_i = gbar_i . h_i = b0_i . x_i
    std::vector<double> ones(k, 1.0);
    upload(ones, small);
    launch_col_shift(n, k, Zc, Y, small, s);
    std::vector<double> cvec = dots(B0, X);
    upload(cvec, small + k);
    const int kp = (2 * k + 3) / 4 * 4;
    double *A = dev(8 * (size_t)n), *Qp = dev(8 * (size_t)n * kp), *Gp = dev(8 * (size_t)n * kp);
    launch_vector_vertex(n, k, kp, ctx->Hres, Zc, ctx->dinv64, ctx->lam_d, glam, small + k, A, Qp, Gp, s);
    const bool od = is_device_ptr(grad_values);
    double* gout = od ? grad_values : dev(8 * (size_t)ctx->nnz);
    const double bw = grad_bandwidth ? bandwidth : 0.0;
    launch_sddmm_rows(n, ctx->row_ptr, ctx->col, ctx->val_orig, ctx->vdt_orig, kp, Qp, Gp, A, gout, bw,
                      ctx->bw_partial, ctx->bw_blocks, s);
    if (!od) check_cuda(cudaMemcpyAsync(grad_values, gout, 8 * (size_t)ctx->nnz, cudaMemcpyDeviceToHost, s), "d2h");
    std::vector<double> bp(ctx->bw_blocks);
    check_cuda(cudaMemcpyAsync(bp.data(), ctx->bw_partial, sizeof(double) * bp.size(), cudaMemcpyDeviceToHost, s),
               "d2h");
    check_cuda(cudaStreamSynchronize(s), "vector backward");
    for (void* p : tmp) cudaFreeAsync(p, s);
    check_cuda(cudaStreamSynchronize(s), "vector backward free");
    if (grad_bandwidth) {
      double acc = 0.0;
      for (double v : bp) acc += v;
      *grad_bandwidth = bw > 0.0 ? acc / bw : 0.0;
    }
    if (iterations) *iterations = it;
    if (max_rel_resid) *max_rel_resid = worst;
    if (!(worst <= tol)) status = SFAIRSC_ERR_NOT_CONVERGED;
  });
  if (rc != SFAIRSC_OK) return rc;
  if (status != SFAIRSC_OK)
    g_last_error = "conjugate gradient did not reach rtol (eigenvectors not accurate enough, or a tiny gap)";
  return status;
}

}  // extern "C"
