/*
 * sfairsc.h -- C ABI of the GB300 s-FairSC library (libsfairsc.so).
 *
 * s-FairSC (Wang, Lu, Davidson and Bai, "Scalable Spectral Clustering with
 * Group Fairness Constraints", AISTATS 2023, Algorithm 3) solves the fair
 * spectral clustering problem (eq. normal-prob-fair)
 *
 *     min tr(H^T L H)  s.t.  H^T D H = I_k,  F^T H = 0
 *
 * by computing the k smallest eigenpairs of
 *
 *     L_n^sigma = P L_n P + sigma (I - P)                    (eq. asigma)
 *
 * with L_n = D^{-1/2} (D - W) D^{-1/2}, C = D^{-1/2} F, F the first h-1
 * columns of F0 = G - 1 z^T (Lemma 2.1), P = I - C (C^T C)^{-1} C^T
 * (eq. mv-Pw) and sigma = ||L_n||_1 (App. C), touching the operator only
 * through w -> P(L_n(P w)) - sigma P w + sigma w (Sec. 3.4 (i)).  The
 * embedding is H = D^{-1/2} X and the cluster labels come from k-means on
 * the rows of H (Algorithm 3 step 4).
 *
 * Conventions shared by every entry point
 *  - Pointers may be device pointers (cudaMalloc, torch CUDA tensors,
 *    managed memory) or host pointers (pageable or pinned); the library
 *    detects which with cudaPointerGetAttributes.  Host inputs are copied to
 *    library-owned device buffers; host outputs are filled by a copy back.
 *  - Integer arrays are int32, floating arrays are FP64 unless a dtype says
 *    otherwise.  Matrices are row-major n x k unless stated.
 *  - Every call returns an sfairsc_status (0 = success, negative = error).
 *    No C++ exception crosses the ABI.  sfairsc_strerror() names a status.
 *  - A context is not thread-safe; distinct contexts are independent.
 *  - All device work is ordered on the stream given at create
 *    (NULL = the legacy default stream).  sfairsc_solve, sfairsc_kmeans and
 *    sfairsc_backward return after that work completes.
 *    sfairsc_apply_operator on device buffers returns once its kernel is
 *    enqueued.
 */
#ifndef SFAIRSC_H
#define SFAIRSC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define SFAIRSC_API __attribute__((visibility("default")))
#else
#define SFAIRSC_API
#endif

#define SFAIRSC_ABI_VERSION 2
#define SFAIRSC_MAX_GROUPS 32   /* h <= 32: groups are reduced with one warp lane each */
#define SFAIRSC_MAX_BLOCK 4     /* Krylov block size b in 1..4 */

typedef enum {
  SFAIRSC_OK = 0,
  SFAIRSC_ERR_INVALID_ARG = -1,     /* null pointer, size out of range, bad enum */
  SFAIRSC_ERR_BAD_CSR = -2,         /* row_ptr not monotone, column out of range, self loop, negative weight */
  SFAIRSC_ERR_ISOLATED_VERTEX = -3, /* some d_i = 0: D must be positive definite (Sec. 2.1) */
  SFAIRSC_ERR_EMPTY_GROUP = -4,     /* some |V_s| = 0: F would lose rank h-1 (Lemma 2.1) */
  SFAIRSC_ERR_K_TOO_LARGE = -5,     /* k > n - h + 1, the dimension of null(C^T) */
  SFAIRSC_ERR_NONFINITE = -6,       /* NaN or Inf in the input weights */
  SFAIRSC_ERR_NOT_CONVERGED = -7,   /* max_restarts reached; outputs hold the best Ritz pairs so far */
  SFAIRSC_ERR_SHIFT = -8,           /* a returned eigenvalue reached sigma: sigma <= lambda_k (Prop. 3.3) */
  SFAIRSC_ERR_CUDA = -9,            /* a CUDA runtime call failed */
  SFAIRSC_ERR_OOM = -10,            /* device or pinned-host allocation failed */
  SFAIRSC_ERR_DEVICE_TIMEOUT = -11, /* a bounded device-side wait gave up (the kernel returned early) */
  SFAIRSC_ERR_UNSUPPORTED = -12,    /* a valid request outside the library's limits (h > 32, no sm_103a device) */
  SFAIRSC_ERR_BREAKDOWN = -13       /* the Krylov block lost rank (exactly invariant subspace) */
} sfairsc_status;

typedef enum { SFAIRSC_F64 = 0, SFAIRSC_F32 = 1, SFAIRSC_BF16 = 2 } sfairsc_dtype;

/* FP64: every vector, value and reduction in FP64.
 * MIXED: Krylov vectors and SpMV in FP32 (values stored as given: FP32 or
 * BF16); group sums, Gram-Schmidt inner products (compensated FP32 pairs),
 * the (h-1)x(h-1) Cholesky of C^T C and the projected eigenproblem in FP64. */
typedef enum { SFAIRSC_PREC_FP64 = 0, SFAIRSC_PREC_MIXED = 1 } sfairsc_prec;

typedef struct {
  double sigma;            /* Hotelling shift; NaN => ||L_n||_1 (App. C) */
  double tol;              /* converged when ||A x - lambda x|| <= tol * sigma; default 1e-6 */
  int32_t max_restarts;    /* default 200 */
  int32_t basis;           /* Krylov basis size m; 0 => max(2k, 20, 10 b) rounded to the block b */
  int32_t prec;            /* sfairsc_prec; default MIXED */
  int32_t block;           /* Krylov block size 1..4; default 1 */
  uint64_t seed;           /* start block of the eigensolver; default 1 */
  uint64_t kmeans_seed;    /* splitmix64 seed of k-means++; default 0 */
  int32_t kmeans_n_init;   /* replicates, best inertia wins; default 1 */
  int32_t kmeans_max_iter; /* Lloyd assignments per replicate; default 100 */
  int32_t validate;        /* 0: none, 1: structure checks (default), 2: also symmetry (sorted columns) */
  int32_t profile;         /* 1: time the operator and orthogonalisation kernels with CUDA events (info.ms_*) */
  int32_t wait_limit_us;   /* bound of every device-side wait (grid barriers, copy completions) in
                              microseconds; a wait that runs out sets an error word, the kernel returns
                              and the call reports DEVICE_TIMEOUT; 0 => 2,000,000 (2 s) */
  int32_t fault_inject;    /* testing hook, 0 normally.  1: the first operator launch of the next
                              sfairsc_solve / sfairsc_apply_operator call waits on a device flag that
                              nothing sets, so that call ends in DEVICE_TIMEOUT after wait_limit_us
                              (no fault, no hang); the hook is then cleared and later calls run normally */
  int32_t spmv_window;     /* 0 (default): the operator's SpMV takes row blocks dynamically and gathers
                              its input from L2.  1: each CTA keeps its own row range and, per row
                              segment, stages a slice of the input vector in shared memory where that
                              serves enough of the segment's gathers (chosen at create from the column
                              distribution), gathering the rest from L2 */
  int32_t orth_mode;       /* reorthogonalisation of each new Krylov block.  0: classical Gram-Schmidt
                              twice with the second projection deferred -- the block is stored after one
                              projection and corrected during the next step's first pass over the basis
                              (two passes over the basis per step); 1: the DGKS test of ARPACK, a third
                              pass when a column kept less than 1/sqrt(2) of its norm */
  int32_t restart_mode;    /* the thick-restart product V <- V Y.  0 (default): on the tensor cores
                              (tcgen05, TF32 in three passes hi*hi + hi*lo + lo*hi, FP32 accumulation) for
                              a MIXED basis with blocks of 4 whose tile plan fits in shared memory, on the
                              CUDA cores (FP32 FMA) otherwise; 1: always on the CUDA cores */
  int32_t reserved[3];
} sfairsc_opts;

typedef struct {
  int32_t status;          /* same value the call returned */
  int32_t restarts;        /* thick restarts performed */
  int32_t matvecs;         /* operator applications (counting each of the b block columns) */
  int32_t kmeans_iters;    /* Lloyd assignments of the winning replicate */
  double sigma;            /* shift used */
  double max_resid;        /* max_i ||A x_i - lambda_i x_i||_2 / sigma, FP64 operator, ||x_i|| = 1 */
  double fairness_err;     /* max |F^T H| over entries */
  double dorth_err;        /* max |H^T D H - I| over entries */
  double kmeans_inertia;   /* sum of squared distances of the winning replicate */
  float ms_setup, ms_solve, ms_kmeans, ms_total;
  float ms_operator;       /* with opts.profile: summed device time of the fused operator launches */
  float ms_orth;           /* with opts.profile: summed device time of the CGS2 orthogonalisation launches */
  int32_t n_operator;      /* fused operator launches in the solve (main precision) */
  int32_t n_orth;          /* orthogonalisation launches in the solve */
  int32_t n_launches;      /* all kernels this call launched */
  int32_t orth_cols;       /* sum over orthogonalisation launches of the basis columns J swept */
  int32_t basis;           /* Krylov basis size m in use */
  int32_t block;           /* Krylov block size b in use */
  int32_t orth_sweeps;     /* passes over the basis V in all orthogonalisation launches (2 or 3 each) */
  float ms_restart;        /* with opts.profile: device time of the thick-restart GEMMs */
  float ms_host_eig;       /* host time of the projected eigenproblems (one per restart) */
  float ms_final;          /* device time of the final FP64 check, projection and embedding */
  int32_t host_eig_fallbacks; /* projected eigenproblems whose QR iteration hit its sweep limit and were
                                 solved again by cyclic Jacobi */
  int32_t spmv_segments;   /* row segments of the operator's SpMV at the solve's block size */
  int32_t spmv_windowed;   /* of those, segments that stage a shared-memory window of the input */
  float spmv_in_window;    /* fraction of the stored entries whose gather is served by a window */
  int32_t restarts_tc;     /* thick restarts taken on the tensor cores (opts.restart_mode) */
  int32_t reserved[3];
} sfairsc_info;

typedef struct sfairsc_ctx sfairsc_ctx;

/* Human-readable name of a status code; never NULL. */
SFAIRSC_API const char* sfairsc_strerror(int status);

/* Detail message of the last failing call on this thread ("" after a
 * success); valid until the next call on this thread.  Never NULL. */
SFAIRSC_API const char* sfairsc_last_error(void);

/* Fill *opts with the defaults listed above.  Errors: INVALID_ARG if opts is NULL. */
SFAIRSC_API int sfairsc_opts_default(sfairsc_opts* opts);

/*
 * Build a solver context for one graph (Algorithm 3 steps 1-2).
 *
 * n, nnz        vertices and stored entries (both triangles of the symmetric W)
 * row_ptr       int32[n+1], row_ptr[0] = 0, nondecreasing, row_ptr[n] = nnz
 * col_idx       int32[nnz], column of each entry, in [0, n), no diagonal
 * values        nnz weights w_ij >= 0 of dtype value_dtype (sfairsc_dtype);
 *               W must be symmetric (checked only with validate = 2)
 * group_labels  int32[n], group of each vertex in [0, h) (eq. group-vec);
 *               F is built from them per Lemma 2.1 and never stored
 * h             number of groups, 1..32 (h = 1: plain SC, Algorithm 1)
 * k             number of eigenpairs and clusters, 1 <= k <= n - h + 1
 * normalized    1: the paper's normalized problem.  0: an extension the
 *               paper does not define: L = D - W, P = I - F (F^T F)^{-1} F^T,
 *               sigma = ||L||_1, H = X.
 * opts          NULL for defaults
 * cuda_stream   cudaStream_t to order all work on (NULL = default stream)
 *
 * Ownership: device inputs are borrowed and must stay valid and unchanged
 * until sfairsc_destroy; host inputs are copied.  The context owns its
 * workspace (Krylov basis, projected matrix, scratch), allocated here.
 * Computes the degrees d_i = sum_j w_ij (Sec. 2.1), d^{-1/2}, the group
 * sizes and sums S_s = sum_{i in V_s} 1/d_i, C^T C in closed form from them,
 * its Cholesky factor, and sigma.
 * Errors: INVALID_ARG, BAD_CSR, ISOLATED_VERTEX, EMPTY_GROUP, K_TOO_LARGE,
 * NONFINITE, UNSUPPORTED, CUDA, OOM.  On error *out is NULL.
 */
SFAIRSC_API int sfairsc_create(sfairsc_ctx** out, int64_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx,
                   const void* values, int32_t value_dtype, const int32_t* group_labels, int32_t h, int32_t k,
                   int32_t normalized, const sfairsc_opts* opts, void* cuda_stream);

/*
 * A context for the fair SC problem with a general constraint matrix F in place of group labels
 * (eq. normal-prob-fair: min tr(H^T L H), H^T D H = I, F^T H = 0, for any F of full column rank;
 * the random-Laplacian experiment of Sec. 4 uses a random dense F).  Everything else is as in
 * sfairsc_create: C = D^{-1/2} F (F for normalized = 0), C^T C = F^T D^{-1} F is formed by a
 * device reduction and factored in FP64 (Sec. 3.4 (ii), eq. mv-Pw), and the fused operator
 * applies P w = w - C (C^T C)^{-1} C^T w as a pair of tall-skinny products (C^T w reduced over
 * the rows, then C a per row) around the SpMV.  sfairsc_solve, sfairsc_apply_operator,
 * sfairsc_backward work on the context unchanged; info.fairness_err is max |F^T H|.
 *
 * F  double[n * p], row-major (row i holds F's row i), DEVICE or host memory; borrowed if on
 *    the device (keep it alive and unchanged until destroy), copied if on the host.  Finite.
 * p  columns of F, 0..31 (0: no constraint, plain SC, Algorithm 1); k <= n - p.
 * Errors: as sfairsc_create; INVALID_ARG also when F lacks full column rank (its C^T C is not
 * positive definite), NONFINITE when F holds a non-finite entry; UNSUPPORTED for p > 31.
 */
SFAIRSC_API int sfairsc_create_dense(sfairsc_ctx** out, int64_t n, int64_t nnz, const int32_t* row_ptr,
                                     const int32_t* col_idx, const void* values, int32_t value_dtype, const double* F,
                                     int32_t p, int32_t k, int32_t normalized, const sfairsc_opts* opts,
                                     void* cuda_stream);

/* Release the context and its workspace.  NULL is accepted.  Returns OK or CUDA. */
SFAIRSC_API int sfairsc_destroy(sfairsc_ctx* ctx);

/* The shift sigma in use (Sec. 3.4 (iii), App. C).  Errors: INVALID_ARG. */
SFAIRSC_API int sfairsc_get_sigma(const sfairsc_ctx* ctx, double* sigma);

/*
 * out = L_n^sigma w for nvec vectors at once (Sec. 3.4 (i)-(ii)):
 * P(L_n(P w)) - sigma P w + sigma w, in one fused kernel.
 * w, out: n x nvec COLUMN-major (each vector contiguous), FP64 when the
 * context precision is FP64 and FP32 when it is MIXED; nvec in 1..4.
 * w and out must not overlap.  Errors: INVALID_ARG, CUDA, DEVICE_TIMEOUT.
 */
SFAIRSC_API int sfairsc_apply_operator(sfairsc_ctx* ctx, const void* w, void* out, int32_t nvec);

/*
 * Algorithm 3 steps 3-4: the k smallest eigenpairs of L_n^sigma by a
 * thick-restart block Lanczos with CGS2 reorthogonalisation, then
 * H = D^{-1/2} X and seeded k-means on the rows of H.
 * eigenvalues  double[k], ascending (FP64 Rayleigh quotients of the final vectors)
 * H            double[n*k] row-major, H^T D H = I; each column's largest-magnitude
 *              entry (lowest row on ties) is positive.  May be NULL.
 * labels       int32[n] cluster of each vertex in [0, k).  May be NULL (no k-means).
 * info         may be NULL.
 * Errors: INVALID_ARG, NOT_CONVERGED (outputs still written), SHIFT, CUDA,
 * DEVICE_TIMEOUT, BREAKDOWN.
 */
SFAIRSC_API int sfairsc_solve(sfairsc_ctx* ctx, double* eigenvalues, double* H, int32_t* labels, sfairsc_info* info);

/*
 * Seeded k-means on the rows of an n x d FP64 row-major matrix (Algorithm 3
 * step 4), exactly reproducible: float32 distances in dimension order,
 * splitmix64 counter draws, k-means++ with integer-quantised D^2 weights,
 * Lloyd with fixed-point exact centroid sums (the full rule set is stated
 * in the library's k-means source).
 * labels int32[n]; centroids double[kc*d] (may be NULL); inertia double[1] (may be NULL).
 * Errors: INVALID_ARG, CUDA, OOM.
 */
SFAIRSC_API int sfairsc_kmeans(int64_t n, int32_t d, const double* X, int32_t kc, uint64_t seed, int32_t n_init,
                   int32_t max_iter, int32_t* labels, double* centroids, double* inertia, int32_t* iterations,
                   void* cuda_stream);

/*
 * Gradient of f = sum_i gbar_i lambda_i with respect to the stored weights,
 * after a successful sfairsc_solve on this context:
 *   d lambda_i / d w_ab = (h_ai - h_bi)^2 - lambda_i (h_ai^2 + h_bi^2)
 * for the undirected weight w_ab = w_ba (first-order perturbation of the
 * pencil (Z^T L Z, Z^T D Z) of Algorithm 2, whose Z does not depend on W);
 * each CSR entry receives half, so summing over both entries gives the
 * undirected derivative.  One pass over W's sparsity pattern (SDDMM).
 * grad_lambda   double[k] (gbar)
 * grad_values   double[nnz] output
 * bandwidth     s > 0 when the weights are w = exp(-r^2/(2 s^2)); then
 *               *grad_bandwidth = sum_e g_e w_e (-2 ln w_e) / s.  Pass
 *               bandwidth <= 0 or grad_bandwidth = NULL to skip it.
 * Errors: INVALID_ARG (no solve yet), CUDA.
 */
SFAIRSC_API int sfairsc_backward(sfairsc_ctx* ctx, const double* grad_lambda, double* grad_values, double bandwidth,
                     double* grad_bandwidth);

/*
 * Gradient of a loss on the embedding H (and optionally on the eigenvalues) with respect to the
 * stored weights, after a successful sfairsc_solve on this context (normalized problem, k <= 64,
 * simple eigenvalues).  The columns of H are the generalized eigenvectors of the pencil
 * (Z^T L Z, Z^T D Z) of Algorithm 2 (Z spans null(F^T) and does not depend on W), with H^T D H = I
 * and the sign convention of sfairsc_solve; first-order perturbation gives, per undirected weight,
 *   d loss / d w_ab = sum_i (v_ia - v_ib)(h_ia - h_ib) - lambda_i (v_ia h_ia + v_ib h_ib)
 *                           - c_i (h_ia^2 + h_ib^2) / 2
 *                   + sum_i gbar_lambda_i ((h_ia - h_ib)^2 - lambda_i (h_ia^2 + h_ib^2)),
 * v_i = sum_{j != i} h_j (h_j^T gbar_i) / (lambda_i - lambda_j) over every eigenpair of the pencil,
 * c_i = gbar_i^T h_i.  The j <= k part of v_i comes from the computed eigenvectors; the rest from k
 * conjugate-gradient solves (A - lambda_i I) y = (I - X X^T) P D^{-1/2} gbar_i on the FP64 operator
 * A = L_n^sigma, positive definite on that complement; then one SDDMM over W's pattern.
 * Each CSR entry receives half of the undirected derivative.
 * grad_H        double[n * k] row-major (d loss / d H), device or host
 * grad_lambda   double[k] or NULL
 * grad_values   double[nnz] output, device or host
 * bandwidth, grad_bandwidth   as in sfairsc_backward
 * max_iter      conjugate-gradient iterations (0: 1000); rtol relative residual (<= 0: 1e-10)
 * iterations, max_rel_resid   (nullable) iterations taken and the largest final relative residual
 * The solves deflate with the computed eigenvectors, so they must come from an FP64 solve at a
 * tolerance near rtol (for example opts.tol = 1e-12); a looser solve leaves parts of lower
 * eigenvectors in the complement, where A - lambda_i I is indefinite, and the solves stall.
 * Errors: INVALID_ARG (no solve, repeated eigenvalue), UNSUPPORTED (k > 64, normalized = 0, a MIXED
 * context), NOT_CONVERGED (some relative residual above rtol after max_iter; outputs written from the
 * last iterate), CUDA, OOM, DEVICE_TIMEOUT.
 */
SFAIRSC_API int sfairsc_backward_vectors(sfairsc_ctx* ctx, const double* grad_H, const double* grad_lambda,
                                         double* grad_values, double bandwidth, double* grad_bandwidth,
                                         int32_t max_iter, double rtol, int32_t* iterations, double* max_rel_resid);

/*
 * One application of L_n^sigma (same result as sfairsc_apply_operator in
 * MIXED precision) that allocates no memory at all.  The paper has no
 * counterpart.  It serves callers that cannot call cudaMalloc: plug-ins that
 * run inside a host runtime which owns the device allocator or refuses new
 * allocations once it has started, and deployments whose device memory budget
 * is fixed at start-up.  No context is needed: degrees, D^{-1/2}, the C^T C
 * factor and sigma = ||L_n||_1 are recomputed on every call from the inputs.
 *
 * n, nnz, row_ptr, col_idx   CSR of the symmetric W as in sfairsc_create
 * values                      FP32 weights; group_labels int32 in [0, h)
 * w, out                      FP32, n x nvec COLUMN-major, nvec in 1..4; must not overlap
 * Every pointer must be DEVICE memory (host data would need a staging
 * buffer).  Limits: n <= 524,288, h <= 32, normalized problem only.
 *
 * Scratch is one file-scope device array of about 20 MB that every GPU that
 * loads the library holds until the process exits.  The first call on a
 * device resolves that array's address (cudaGetSymbolAddress) with the
 * device current; make that first call before any stream capture.  All calls
 * share the array and it keeps the last call's contents (each call clears the
 * words that must start at zero): calls that overlap on the GPU race, so do
 * not run two at once on one device.  Calls from different host threads are
 * serialised.  Each call waits on cuda_stream for its set-up reductions and
 * returns after out is written.
 * Errors: INVALID_ARG (null or host pointer, bad size), UNSUPPORTED (n or h
 * above the limits), BAD_CSR, ISOLATED_VERTEX, EMPTY_GROUP, NONFINITE,
 * DEVICE_TIMEOUT, CUDA.
 */
SFAIRSC_API int sfairsc_apply_operator_static(int64_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx,
                                              const float* values, const int32_t* group_labels, int32_t h,
                                              const float* w, float* out, int32_t nvec, void* cuda_stream);

/* ------------------------------------------------------------------ batched form
 * Many independent problems of Algorithm 3 (steps 2-4: setup, the k smallest
 * eigenpairs of L_n^sigma, H = D^{-1/2} X) solved by ONE persistent
 * cooperative kernel launch.  Each graph is the normalized s-FairSC problem
 * of Sec. 3.4 with its own W (FP32 weights), group labels, h and k.  The
 * eigensolver is the block (b = 4) form of the restarted Lanczos method: the
 * operator of Sec. 3.4 (i)-(ii) is applied to 4 vectors at once (an SpMM that
 * reads the CSR once per 4 vectors), Krylov vectors and the operator run in
 * FP32, inner products carry in FP64, the projected problem (Rayleigh-Ritz)
 * and the final residual check run in FP64.  A graph is converged when every
 * returned pair has ||A x - lambda x|| <= tol * sigma with the FP64 operator.
 * k-means (step 5) is not part of the batch: call sfairsc_kmeans on H.
 *
 * Every pointer in a graph description is DEVICE memory owned by the
 * caller; row_ptr, col_idx, values and group_labels are read only and must
 * stay alive and unchanged until sfairsc_batch_destroy.  Outputs (device):
 * eigenvalues (k doubles, ascending) and, when H is not NULL, H (n x k
 * doubles, row-major, each column's largest-magnitude entry of X made
 * positive).  Limits per graph: 16 <= n < 2^30, nnz < 2^31, 1 <= h <= 32,
 * k <= 28 and k <= n - h + 1.
 */
typedef struct {
  int64_t n, nnz;
  const int32_t* row_ptr;       /* n + 1 */
  const int32_t* col_idx;       /* nnz, both triangles, no self loops */
  const float* values;          /* nnz, w_ij >= 0 */
  const int32_t* group_labels;  /* n, in [0, h) */
  int32_t h, k;
  double* eigenvalues;          /* out: k */
  double* H;                    /* out: n x k row-major, or NULL */
} sfairsc_batch_graph;

typedef struct {
  int32_t status;       /* first non-OK graph status, DEVICE_TIMEOUT, or OK */
  int32_t converged;    /* graphs that reached tol */
  int32_t breakdowns;   /* Krylov blocks that lost rank (restarted with fresh vectors) */
  int32_t grid;         /* CTAs of the launch */
  int64_t restarts;     /* summed over graphs */
  int64_t matvecs;      /* operator applications summed over graphs (4 per block) */
  double max_resid;     /* max over graphs of max_i ||A x_i - lambda_i x_i|| / sigma */
  double split;         /* schedule: load fraction above which a graph gets a larger team */
  float ms_solve;       /* device time of the launch */
  float ms_autotune;    /* host time spent in sfairsc_batch_autotune */
  int32_t ctas_per_sm;  /* schedule: resident CTAs per SM (1 or 2) */
  int32_t max_team;     /* schedule: largest team (CTAs working on one graph) */
  int32_t autotuned;    /* 1 after sfairsc_batch_autotune */
  int32_t cuda_graph;   /* 1 when the launch sequence replays a captured CUDA graph */
  int32_t smem_bytes;   /* dynamic shared memory per CTA */
  int32_t teams[5];     /* teams of 1, 2, 4, 8, 16 CTAs */
  int32_t reserved[6];
} sfairsc_batch_info;

typedef struct sfairsc_batch sfairsc_batch;

/* Plan a batch: checks the descriptions, allocates every graph's workspace
 * (one device arena, about n * (4 (m + 4) + 140) bytes per graph with m the
 * basis size max(2k + 8, 20)), and builds the schedule from a cost model:
 * graphs queue largest first, and graphs large against the mean per-CTA load
 * get teams of 2..16 CTAs that split their rows.  opts: tol, max_restarts,
 * basis, seed, validate are used (validate 2 also checks symmetry and sorted
 * columns); NULL gives the defaults.  Errors: INVALID_ARG, K_TOO_LARGE, OOM,
 * UNSUPPORTED, CUDA.  Per-graph input errors (BAD_CSR, ISOLATED_VERTEX,
 * EMPTY_GROUP, NONFINITE) are found on the device and reported per graph by
 * sfairsc_batch_solve. */
SFAIRSC_API int sfairsc_batch_create(sfairsc_batch** out, int32_t count, const sfairsc_batch_graph* graphs,
                                     const sfairsc_opts* opts, void* cuda_stream);

/* Autotuner: times every candidate schedule (resident CTAs per SM, largest
 * team, team threshold) with one full solve each and keeps the fastest; the
 * outputs hold the last candidate's (identical up to rounding) results. */
SFAIRSC_API int sfairsc_batch_autotune(sfairsc_batch* batch);

/* Set the schedule by hand: ctas_per_sm 1 or 2 (resident CTAs per SM),
 * max_team a power of two in 1..16, split >= 0 (a graph moves to the next
 * larger team while its cost exceeds split x the mean per-CTA load x the team
 * size; 0 puts every graph on the largest team).  UNSUPPORTED if the kernel
 * does not fit that many CTAs per SM. */
SFAIRSC_API int sfairsc_batch_schedule(sfairsc_batch* batch, int32_t ctas_per_sm, int32_t max_team, double split);

/* Solve every graph with one cooperative launch (captured into a CUDA graph
 * on first use and replayed).  status (host, count entries, nullable)
 * receives each graph's status.  Returns OK when every graph converged, else
 * the first failing graph's status (NOT_CONVERGED leaves the best pairs found),
 * or DEVICE_TIMEOUT if a bounded device wait gave up. */
SFAIRSC_API int sfairsc_batch_solve(sfairsc_batch* batch, int32_t* status, sfairsc_batch_info* info);

/* Per-graph results of the last sfairsc_batch_solve (host arrays of count
 * entries, each nullable): thick restarts, operator applications (4 per block
 * step) and max_i ||A x_i - lambda_i x_i|| / sigma. */
SFAIRSC_API int sfairsc_batch_stats(const sfairsc_batch* batch, int32_t* restarts, int32_t* matvecs, double* resid);

SFAIRSC_API int sfairsc_batch_destroy(sfairsc_batch* batch);

/* create + solve + destroy in one call. */
SFAIRSC_API int sfairsc_solve_batched(int32_t count, const sfairsc_batch_graph* graphs, const sfairsc_opts* opts,
                                      int32_t* status, sfairsc_batch_info* info, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* SFAIRSC_H */
