// Internal declarations of the s-FairSC library: the context, parameter
// layout and the host-side launchers of every kernel.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sfairsc.h"

namespace sfairsc {

// Device parameter block (doubles): z_s, the Cholesky factor of C^T C and sigma.
constexpr int kPZ = 0;                 // z_s = |V_s| / n, s < 32
constexpr int kPL = 32;                // lower Cholesky factor of C^T C, row-major, stride 31
constexpr int kLStride = 31;
constexpr int kPSigma = kPL + 31 * 31; // sigma
constexpr int kPLinv = kPSigma + 1;    // reciprocals of the factor's diagonal, 31 entries
constexpr int kPG = 1056;               // h x h map from the group sums to the correction coefficients
constexpr int kParams = kPG + 32 * 32;

enum class VecType { F64 = 0, F32 = 1 };

struct CudaError {
  cudaError_t err;
  const char* what;
};

// Throwing wrappers used inside the library; the C entry points catch and map to status codes.
struct Status {
  int code;
  std::string msg;
};
void check_cuda(cudaError_t e, const char* what);
[[noreturn]] void fail(int code, const std::string& msg);
// What fail() and check_cuda() throw inside the library; entry points map it to a status.
struct SfError {
  int code;
  std::string msg;
};
// Record the detail message returned by sfairsc_last_error() on this thread.
void set_last_error(const std::string& msg);

// Shared-memory windows of the SpMV input (one table per block size b): each
// CTA's rows are cut into segments; a segment with ws >= 0 stages rows
// [ws, ws + win_rows) of ytil (b values each) in shared memory and gathers
// from there the entries whose column falls inside, and from L2 the others.
struct WindowTable {
  int win_rows = 0;                // rows per window (0: no windows)
  const int32_t* seg_row = nullptr;  // int32[nseg + 1]: first row of each segment
  const int32_t* seg_ws = nullptr;   // int32[nseg]: window start row, or -1 (no window)
  const int32_t* cta_seg = nullptr;  // int32[grid + 1]: first segment of each CTA
  int nseg = 0;
  int windowed = 0;                // segments with a window
  long long in_window = 0;         // stored entries whose column falls in their segment's window
};

// Operator launch description (everything the fused kernel needs).
struct OpPlan {
  int n = 0;
  int h = 1;
  int normalized = 1;
  int grid = 0;          // cooperative CTAs
  int threads = 1024;
  int batch_rows = 32;   // unused (kept for the plan layout)
  int lanes_per_row = 8; // SpMV lanes per row (power of two, 2..32): 8 FP32 / 4 FP64 entries per lane per pass
  int mode = 0;          // 0: L_n^sigma w, 1: P w
  const int32_t* row_ptr = nullptr;
  const int32_t* col = nullptr;
  const void* val = nullptr;
  int val_dtype = 0;
  const uint8_t* lab = nullptr;
  const void* dinv = nullptr;  // VT[n]
  const double* deg = nullptr; // double[n] (unnormalized path)
  const double* params = nullptr;
  void* ytil = nullptr;        // VT[n * 4]
  double* partial = nullptr;   // double[grid * 32 * 4]
  const int32_t* cta_rows = nullptr;  // int32[grid + 1]
  unsigned long long* barrier = nullptr;  // grid barrier arrival counter (64-bit)
  unsigned* err = nullptr;
  unsigned* work = nullptr;    // 1 word: dynamic row-block counter of the SpMV
  unsigned long long wait_ns = 2000000000ull;  // bound of every device-side wait
  const unsigned* stall_flag = nullptr;  // non-null: the launch first waits for this word (never set) to become nonzero
  WindowTable win[3];  // by block size b = 1, 2, 4 (index 0, 1, 2)
  const void* Fd = nullptr;  // dense constraints F (n x (h - 1), row-major, vector type) instead of labels
  // C^T t from y (vector type, n x kpad in 4-column panels, kpad = h rounded up to 4) and the
  // per-CTA sums it needs (grid x 33 x 4 doubles); nullptr: a pass over t after the SpMV
  const void* Kp = nullptr;
  double* partial2 = nullptr;
};

// Rows of ytil (b values of vs bytes) a window may hold next to the kernel's other shared memory.
int window_rows_for(int b, int vs, size_t base_smem);
// Choose the windows of the CTA row ranges cta_rows (host copy, grid + 1 entries) for windows of
// win_rows rows: a device pass histograms each 256-row chunk's columns, the host merges chunks
// into segments.  Allocations go through alloc (device memory owned by the caller).
WindowTable build_window_table(int n, const int32_t* row_ptr, const int32_t* col, const std::vector<int32_t>& cta_rows,
                               int win_rows, int bytes_per_row, void* (*alloc)(void*, size_t), void* alloc_ctx,
                               cudaStream_t s);

// Launch out = L_n^sigma w for nvec vectors; element (r, v) of w is w[r*wrs + v*wcs]
// and of out is out[r*ors + v*ocs].
void launch_operator(const OpPlan& p, VecType vt, const void* w, int64_t wrs, int64_t wcs, void* out, int64_t ors,
                     int64_t ocs, int nvec, cudaStream_t s);
// T = L_n X (or L X unnormalized) for b <= 4 or b = 8 FP64 columns (column-major, ld n) with
// FP64-grade accuracy on the FP32 pipe (double-float); ytil_pairs: workspace of n * b float pairs.
void launch_df_spmv(int n, const int32_t* row_ptr, const int32_t* col, const void* val, int val_dtype,
                    const double* dinv64, const double* deg, int normalized, int lanes, const double* X, int b,
                    void* ytil_pairs, double* T, int sms, cudaStream_t s);
// Largest co-resident grid of the operator kernel for this instantiation.
int operator_max_grid(VecType vt, int val_dtype, int nvec, int threads, size_t smem);
size_t operator_smem_bytes(int threads, int h, int nvec, VecType vt);
// The linear map tot -> coef of the operator's small solve ((C^T C)^{-1} and, for group labels, the
// shift by z), as an h x h row-major matrix at P[kPG], from z, the Cholesky factor and its inverse
// diagonal already in P: the kernels then form every coefficient in parallel.
void fill_group_map(double* P, int h, bool dense);
// K_c = d_c^{-1/2} (F_c - sum_r w_cr F_r / d_r) (normalized) or d_c F_c - sum_r w_cr F_r, row c of the
// n x kpad matrix in 4-column panels (zero past the constraint columns), in FP64 and FP32 (either
// output may be null); F is the group indicator (Fd = nullptr) or the dense F (n x p, row-major).
void launch_kmat(int n, const int32_t* row_ptr, const int32_t* col, const void* val, int val_dtype, const uint8_t* lab,
                 const double* Fd, int p, int h, const double* dinv64, const double* deg, int normalized,
                 double* K64, float* K32, cudaStream_t s);

// Setup kernels.
void launch_validate(int n, int64_t nnz, const int32_t* row_ptr, const int32_t* col, const void* val, int val_dtype,
                     const int32_t* labels, int h, int check_symmetry, unsigned* flags, cudaStream_t s);
void launch_degrees(int n, const int32_t* row_ptr, const void* val, int val_dtype, const int32_t* labels_in,
                    uint8_t* lab, double* deg, double* dinv64, float* dinv32, double* blocksums, int nblocks,
                    int h, int normalized, unsigned* flags, cudaStream_t s);
int degrees_blocks(int n);
void launch_sigma_rows(int n, const int32_t* row_ptr, const int32_t* col, const void* val, int val_dtype,
                       const double* dinv64, const double* deg, int normalized, double* blockmax, int nblocks,
                       cudaStream_t s);
void launch_row_partition(int n, const int32_t* row_ptr, int grid, int row_weight, int32_t* cta_rows, cudaStream_t s);
// Dense constraint matrix F (n x p row-major FP64): per-block partial sums of C^T C (p x p) and of
// F^T H (p x k, H n x k row-major); an FP64 -> FP32 copy.
void launch_dense_ctc(int n, int p, const double* F, const double* deg, int normalized, double* partial, int nblocks,
                      cudaStream_t s);
void launch_dense_fth(int n, int p, int k, const double* F, const double* H, double* partial, int nblocks,
                      cudaStream_t s);
void launch_f64_to_f32(int64_t count, const double* in, float* out, cudaStream_t s);

// Krylov kernels.
struct OrthPlan {
  int n = 0;
  int grid = 0;
  int threads = 1024;
  int64_t ldv = 0;
  void* V = nullptr;          // VT, ldv/4 panels of 4 columns, each n x 4 row-major
  void* U = nullptr;          // VT, n x 4 row-major: the block being orthogonalised
  void* Q = nullptr;          // VT, n x 4 row-major: copy of the newest basis block (operator input)
  double* H = nullptr;        // projected matrix, column-major, ld ldh
  int ldh = 0;
  double* partial = nullptr;  // grid * (mmax + 4) * 4
  double* coef = nullptr;     // (mmax + 4) * 4 reduced coefficients
  const int32_t* cta_rows = nullptr;
  unsigned long long* barrier = nullptr;  // grid barrier arrival counter (64-bit)
  unsigned* err = nullptr;
  int* brk_step = nullptr;    // smallest step j whose new block lost rank (atomicMin)
  int* sweeps = nullptr;      // accumulates the number of passes over V
  unsigned long long wait_ns = 2000000000ull;  // bound of every device-side wait
  double* pend = nullptr;     // 256 x 4: pending second-projection correction of the newest block
};
// Orthogonalise the B columns in U against V[:, 0:J] (CGS2), record the
// coefficients in H[0:J, j:j+B], orthonormalise the block (CholQR), store it
// as V[:, J:J+B] and its R factor in H[J:J+B, j:j+B].
// pend_in: V[:, j:j+B] still owes its second projection (correction p.pend, j x B), applied in the
// first sweep.  defer: leave the new block's second projection pending (p.pend, J x B) instead of
// a third sweep; the next launch, or the restart, applies it.
void launch_orth(const OrthPlan& p, VecType vt, int J, int j, int B, bool pend_in, bool defer, cudaStream_t s);
int orth_max_grid(VecType vt, int B, int threads);
// V[:, 0:K] = V[:, 0:m] Y (Y: m x K row-major on device, in the basis precision), then V[:, K:K+B] =
// V[:, m:m+B] - V[:, 0:m] E when E (m x B row-major FP64, the carried block's pending correction) is
// given, else V[:, m:m+B].  V is stored as ldv/4 panels of n x 4 (panel p = columns 4p..4p+3).
// Q (n x 4 row-major) receives the carried block too.
void launch_restart(VecType vt, int n, void* V, int64_t ldv, int m, int K, int B, const void* Y, void* Q,
                    const double* E, cudaStream_t s);
// Fill V[:, 0:B] with a seeded pseudo-random block.
void launch_random_block(VecType vt, int n, void* V, int64_t ldv, int B, uint64_t seed, cudaStream_t s);
// X64 = V[:, 0:m] Y (Y: m x k row-major, in the basis precision), X64 n x k column-major FP64; V unchanged.
// thick restart on the tensor cores (FP32 basis, blocks of 4; see restart_tc.cu): whether the
// shape fits its shared-memory plan, and the launch (Yt: 2 x 8-rounded ldv x 256 floats of scratch)
bool restart_tc_fits(int n, int64_t ldv, int m, int K, int B);
void launch_restart_tc(int n, float* V, int64_t ldv, int m, int K, int B, const float* Y, float* Q, const double* E,
                       float* Yt, int sms, unsigned* err, unsigned long long wait_ns, cudaStream_t s);
void launch_ritz(VecType vt, int n, const void* V, int64_t ldv, int m, int k, const void* Y, double* X64,
                 cudaStream_t s);
// partial[b][c] = sum over block b's rows of (AX_c - lam_c X_c)^2.
void launch_column_resid(int n, int k, const double* X, const double* AX, const double* lam, double* partial,
                         int nblocks, cudaStream_t s);
// FP64 copy / conversion of the first k columns of V to X64 (n x k column-major).
void launch_to_f64(VecType vt, int n, const void* V, int64_t ldv, int k, double* X, cudaStream_t s);
// Column norms and Rayleigh data: out[c] = <X_c, AX_c>, out[k + c] = <X_c, X_c>, out[2k + c] = ||AX_c - l_c X_c||^2.
void launch_column_stats(int n, int k, const double* X, const double* AX, const double* lam, double* partial,
                         int nblocks, double* out, cudaStream_t s);
// X[:, c] *= scale[c] (X column-major n x k).
void launch_scale_columns(int n, int k, double* X, const double* scale, cudaStream_t s);
// Embedding H = D^{-1/2} X (row-major n x k), sign per column; sign_partial workspace.
void launch_embed(int n, int k, const double* X, const double* dinv64, int normalized, double* H,
                  unsigned long long* colkey, cudaStream_t s);
// Fairness and D-orthogonality diagnostics of H.
void launch_diagnostics(int n, int k, int h, const double* H, const double* deg, const uint8_t* lab,
                        const double* params, double* partial, int nblocks, double* out, cudaStream_t s, bool fp64);

// Backward SDDMM.
// grad[e] for every stored entry; partial[b] = per-block sum of the bandwidth terms; A = n-vector
// workspace; Hp = n x backward_padded_width(k) workspace (H with rows padded to a multiple of 4).
int backward_padded_width(int k);
void launch_backward(int n, const int32_t* row_ptr, const int32_t* col, const void* val, int val_dtype, int k,
                     const double* H, const double* lam, const double* gbar, double* grad, double bandwidth,
                     double* partial, int nblocks, double* A, double* Hp, int normalized, cudaStream_t s);

void launch_sddmm_rows(int n, const int32_t* row_ptr, const int32_t* col, const void* val, int val_dtype, int kp,
                       const double* Qp, const double* Gp, const double* A, double* grad, double bandwidth,
                       double* partial, int nblocks, cudaStream_t s);
// Eigenvector-level backward helpers (column-major n x k blocks, FP64).
void launch_rows_to_cols_scaled(int n, int k, const double* G, const double* s, int divide, double* out,
                                cudaStream_t st);
void launch_col_gram(int n, int k1, const double* X, int k2, const double* Y, double* partial, int nblocks,
                     cudaStream_t s);
void launch_col_gemm(int n, int k1, const double* X, int k2, const double* C, double beta, double* out, cudaStream_t s);
void launch_col_dots(int n, int k, const double* A, const double* B, double* partial, int nblocks, cudaStream_t s);
void launch_col_shift(int n, int k, double* Q, const double* P, const double* shift, cudaStream_t s);
void launch_cg_update(int n, int k, double* Y, double* R, const double* P, const double* Q, const double* alpha,
                      cudaStream_t s);
void launch_cg_direction(int n, int k, double* P, const double* R, const double* beta, cudaStream_t s);
void launch_vector_vertex(int n, int k, int kp, const double* H, const double* Zc, const double* dinv,
                          const double* lam, const double* glam, const double* cvec, double* A, double* Qp, double* Gp,
                          cudaStream_t s);

// k-means (device part).  Returns inertia and iterations of the winner.
struct KmeansResult {
  double inertia = 0.0;
  int iterations = 0;
  int launches = 0;
};
KmeansResult run_kmeans(int64_t n, int d, const double* X, int kc, uint64_t seed, int n_init, int max_iter,
                        int32_t* labels, double* centroids, cudaStream_t s);

// Host FP64 symmetric eigensolver (Householder tridiagonalisation + implicit QR).
// A: m x m column-major symmetric (overwritten with eigenvectors), w: eigenvalues ascending.
// Returns false when the QR iteration used up max_sweeps (default 60 m) before
// every off-diagonal entry deflated: A and w then hold an unconverged result.
bool host_symmetric_eig(int m, double* A, double* w, int max_sweeps = -1);
// Cyclic Jacobi (FP64) for the same problem: always converges for finite
// input; slower, the fallback when the QR iteration gives up.  Returns false
// if A holds a non-finite entry.
bool host_symmetric_eig_jacobi(int m, double* A, double* w);

}  // namespace sfairsc
