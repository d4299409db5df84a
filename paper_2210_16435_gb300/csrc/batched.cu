// Batched s-FairSC eigensolve: many independent graphs in ONE persistent
// cooperative launch (the batching form of Algorithm 3 steps 2-4).
//
// The CTAs of the launch are partitioned into teams of 1, 2, 4, 8 or 16
// CTAs.  Every team pulls graphs from the queue of its size class (largest
// graphs first) and solves each one start to finish:
//   setup     degrees, D^{-1/2}, |V_s|, S_s, C^T C and its Cholesky factor in
//             closed form, sigma = ||L_n||_1 (Sec. 2.1, Sec. 3.3, App. C);
//   Lanczos   thick-restart block Lanczos, block size 4, on
//             L_n^sigma = P L_n P + sigma (I - P) (Sec. 3.4), the operator
//             applied to 4 vectors at once as an SpMM (Sec. 3.4 (i)-(ii):
//             y = P w, t = L_n y, out = t - C(b - sigma a)); classical
//             Gram-Schmidt with the DGKS refinement test and Cholesky QR
//             twice; FP32 vectors, FP64 inner-product carries;
//   RR        the projected matrix in FP64, diagonalised inside the CTA by
//             the parallel (round-robin) cyclic Jacobi method;
//   check     Ritz vectors, projection, Rayleigh quotients and explicit
//             residuals with an FP64 operator; H = D^{-1/2} X (Algorithm 3 step 4).
// Rows of a graph are split over the team's CTAs; their partial sums meet in
// global memory behind a team barrier (acquire/release, bounded wait) and are
// added in rank order, so every CTA of a team holds bit-identical small
// matrices and the result does not depend on which team solved the graph.
// The basis V is stored as 4-column panels (panel p = columns 4p..4p+3, an
// n x 4 row-major array), so a CTA's rows of the first J columns are J/4
// contiguous pieces that stream through a shared-memory ring by bulk copies.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace sfairsc {
namespace bat {

constexpr int kT = 512;  // threads per CTA
constexpr int kW = kT / 32;
constexpr int kB = 4;        // Krylov block size
constexpr int kMaxM = 60;    // basis columns
constexpr int kMaxH = 32;
constexpr int kStages = 4;
constexpr int kJacobiSweeps = 24;
constexpr int kBadOff = kMaxH * kB;  // offset of the validation counters in a reduction slot
constexpr unsigned long long kWaitNs = 2000000000ull;

// Result of one graph.
struct Stat {
  int status, restarts, matvecs, breakdowns;
  double max_resid, sigma;
};

struct Job {
  int n, nnz, h, k, m, ldv, lanes, pad;
  const int32_t* row_ptr;
  const int32_t* col;
  const float* val;
  const int32_t* labels;
  double* lam;    // k
  double* H;      // n x k row-major (may be null)
  float* V;       // ldv/4 panels of n x 4
  float* U;       // n x 4
  float* ytil;    // n x 4
  float* dinv;    // n
  double* dinv64; // n
  uint8_t* lab;   // n
  double* X;      // n x 4
  double* AX;     // n x 4
  double* ytil64; // n x 4
};

struct Params {
  double tol;
  int max_restarts;
  int validate;
  unsigned long long seed;
};

// Shared-memory carve-up (byte offsets), computed on the host from the
// batch's largest basis and the ring's stage size.
struct Layout {
  int red, loc, tot, hm, A, E, yf, cf, lc, ring, total;
  int slot;  // doubles per warp partial and per team slot
  int mmax, jmax;
  int stage_floats, stage_rows;
};

struct Sched {
  const Job* jobs;
  Stat* stats;
  const int* order;        // graph indices grouped by class, largest first within a class
  const int* class_begin;  // [ncls + 1]
  unsigned* class_next;    // [ncls] queue heads
  const int* cta_team0;    // first CTA of each CTA's team
  const int* cta_size;
  const int* cta_class;
  unsigned* bar;           // 2 words per CTA (a team uses its first CTA's pair)
  double* part;            // 2 slots per CTA
  unsigned* mailbox;       // per CTA (a team uses its first CTA's word)
  unsigned* err;
  Params prm;
  Layout L;
};

struct Sm {
  double *red, *loc, *tot, *Hm, *A, *E, *Lc;
  float *Yf, *cf;
  double *z, *coefA, *coefD, *av, *cs, *theta, *gram, *R1, *R2, *Rd, *misc;
  float *coefAf, *coefDf, *Rdf;  // FP32 copies used in the per-row loops
  int* pq;
  unsigned char* ring;
  uint64_t *full, *empty;
  int* ints;  // [0] dead, [1] mailbox copy, [2] r0, [3] r1, [4] chol ok, [5] scratch flag, [6] ring abort
};

struct Team {
  int rank, size;
  unsigned* bar;
  double* part;  // this team's slots: part[(rank * 2 + parity) * slot]
  unsigned* err;
  int slot;
  int parity;
};

// ------------------------------------------------------------------ team sync
// Barrier over the team's CTAs (all co-resident: cooperative launch).  The
// wait is bounded; a timeout sets kErrBarrierTimeout and marks the CTA dead,
// after which every barrier and ring stream of this CTA returns at once.
__device__ bool team_barrier(Team& T, Sm& S) {
  __syncthreads();
  if (T.size == 1) return S.ints[0] == 0;
  if (threadIdx.x == 0 && S.ints[0] == 0) {
    const unsigned gen = ld_acquire_gpu(T.bar + 1);
    __threadfence();
    const unsigned arrived = atom_add_acqrel_gpu(T.bar, 1u);
    if (arrived == (unsigned)T.size - 1u) {
      T.bar[0] = 0u;
      __threadfence();
      st_release_gpu(T.bar + 1, gen + 1u);
    } else {
      const unsigned long long t0 = globaltimer_ns();
      while (ld_acquire_gpu(T.bar + 1) == gen) {
        __nanosleep(32);
        if (globaltimer_ns() - t0 > kWaitNs) {
          atomicOr(T.err, kErrBarrierTimeout);
          S.ints[0] = 1;
          break;
        }
      }
    }
  }
  __syncthreads();
  return S.ints[0] == 0;
}

// S.loc[0..cnt) of every CTA of the team -> S.tot[0..cnt), combined in rank order.
// mode 0: sum; 1: max; 2: argmax pairs (values [0, cnt/2), rows [cnt/2, cnt):
// larger value wins, then the lower row).
__device__ void team_reduce(Team& T, Sm& S, int cnt, int mode = 0) {
  if (T.size == 1) {
    for (int i = threadIdx.x; i < cnt; i += kT) S.tot[i] = S.loc[i];
    __syncthreads();
    return;
  }
  double* mine = T.part + (size_t)(T.rank * 2 + T.parity) * T.slot;
  for (int i = threadIdx.x; i < cnt; i += kT) mine[i] = S.loc[i];
  team_barrier(T, S);
  if (mode == 2) {
    const int half = cnt / 2;
    for (int i = threadIdx.x; i < half; i += kT) {
      double bv = -1.0, br = 0.0;
      for (int r = 0; r < T.size; ++r) {
        const double* p = T.part + (size_t)(r * 2 + T.parity) * T.slot;
        const double v = __ldcg(p + i), row = __ldcg(p + half + i);
        if (v > bv || (v == bv && row < br)) {
          bv = v;
          br = row;
        }
      }
      S.tot[i] = bv;
      S.tot[half + i] = br;
    }
  } else {
    for (int i = threadIdx.x; i < cnt; i += kT) {
      double s = mode == 1 ? -INFINITY : 0.0;
      for (int r = 0; r < T.size; ++r) {
        const double v = __ldcg(T.part + (size_t)(r * 2 + T.parity) * T.slot + i);
        s = mode == 1 ? fmax(s, v) : s + v;
      }
      S.tot[i] = s;
    }
  }
  T.parity ^= 1;
  __syncthreads();
}

// Per-warp partials red[w][0..cnt) -> S.loc (fixed order over warps).
__device__ void warps_to_loc(Sm& S, int slot, int cnt) {
  __syncthreads();
  for (int i = threadIdx.x; i < cnt; i += kT) {
    double s = 0.0;
    for (int w = 0; w < kW; ++w) s += S.red[w * slot + i];
    S.loc[i] = s;
  }
  __syncthreads();
}

// The same for red entries holding packed FP32 (sum, carry) pairs (Comp::slot):
// the warps' pairs are added by TwoSum in FP32 and converted to FP64 once.
__device__ void warps_to_loc_pairs(Sm& S, int slot, int cnt) {
  __syncthreads();
  for (int i = threadIdx.x; i < cnt; i += kT) S.loc[i] = comp32_slot_sum(S.red + i, kW, slot);
  __syncthreads();
}

__device__ void zero_red(Sm& S, int slot, int cnt) {
  __syncthreads();
  for (int i = threadIdx.x; i < kW * slot; i += kT)
    if (i % slot < cnt) S.red[i] = 0.0;
  __syncthreads();
}

// Sum of one value per thread over the CTA (fixed order), broadcast.
__device__ double cta_sum(Sm& S, double v) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_allsum(v);
  __syncthreads();
  if (lane == 0) S.red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < kW; ++w) s += S.red[w];
  __syncthreads();
  return s;
}

// ------------------------------------------------------------------ small solves
// Given tot[s*4+v] = sum_{i in V_s} d_i^{-1/2} x_i, the normal equations
// a = (C^T C)^{-1} C^T x with (C^T x)_s = T_s - z_s sum T, and the row
// coefficients coef[s*4+v] = a_s - z.a (a_{h-1} := 0), so that (C a)_i =
// d_i^{-1/2} coef[g_i] (Sec. 3.4 (i)).  a_out (nullable) receives a.
__device__ void solve_groups(const Sm& S, const double* tot, int h, double* a_out, double* coef,
                             float* coef_f = nullptr) {
  const int v = threadIdx.x;
  if (v < kB) {
    const int p = h - 1;
    double sum = 0.0;
    for (int s = 0; s < h; ++s) sum += tot[s * kB + v];
    double y[kMaxH];
    for (int s = 0; s < p; ++s) {
      double r = tot[s * kB + v] - S.z[s] * sum;
      for (int q = 0; q < s; ++q) r -= S.Lc[s * kMaxH + q] * y[q];
      y[s] = r / S.Lc[s * kMaxH + s];
    }
    for (int s = p - 1; s >= 0; --s) {
      double r = y[s];
      for (int q = s + 1; q < p; ++q) r -= S.Lc[q * kMaxH + s] * y[q];
      y[s] = r / S.Lc[s * kMaxH + s];
    }
    double za = 0.0;
    for (int s = 0; s < p; ++s) za += S.z[s] * y[s];
    for (int s = 0; s < p; ++s) {
      if (a_out) a_out[s * kB + v] = y[s];
      coef[s * kB + v] = y[s] - za;
      if (coef_f) coef_f[s * kB + v] = (float)(y[s] - za);
    }
    coef[p * kB + v] = -za;
    if (coef_f) coef_f[p * kB + v] = (float)-za;
  }
  __syncthreads();
}

// Row coefficients of C(b - sigma a) (a nullable: C b).
__device__ void deflate_coef(const Sm& S, int h, double sigma, const double* b, const double* a, double* coef,
                             float* coef_f = nullptr) {
  const int v = threadIdx.x;
  if (v < kB) {
    const int p = h - 1;
    double zu = 0.0;
    double u[kMaxH];
    for (int q = 0; q < p; ++q) {
      u[q] = b[q * kB + v] - (a ? sigma * a[q * kB + v] : 0.0);
      zu += S.z[q] * u[q];
    }
    for (int q = 0; q < p; ++q) {
      coef[q * kB + v] = u[q] - zu;
      if (coef_f) coef_f[q * kB + v] = (float)(u[q] - zu);
    }
    coef[p * kB + v] = -zu;
    if (coef_f) coef_f[p * kB + v] = (float)-zu;
  }
  __syncthreads();
}

// ------------------------------------------------------------------ compensated FP32 sums
// Per-row sums run in FP32 with an error-free TwoSum carry (Knuth): s + c
// holds the running sum to about twice FP32 precision.  This replaces FP64
// accumulation in every per-row loop: this GPU's FP64 rate is a small
// fraction of its FP32 rate.
struct Comp {
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
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
  // the pair packed into 8 bytes (see warps_to_loc_pairs)
  __device__ __forceinline__ double slot() const {
    return __longlong_as_double((long long)(((unsigned long long)__float_as_uint(c) << 32) | __float_as_uint(s)));
  }
};

// Sum over the lanes whose ids differ only in bits >= `from` (xor tree, TwoSum
// at every level); every lane of a group ends with the same pair.
__device__ __forceinline__ void comp_reduce(Comp& a, int from) {
  for (int o = from; o < 32; o <<= 1) {
    const float os = __shfl_xor_sync(0xffffffffu, a.s, o), oc = __shfl_xor_sync(0xffffffffu, a.c, o);
    float t, e;
    two_sum(a.s, os, t, e);
    a.s = t;
    a.c = __fadd_rn(__fadd_rn(a.c, oc), e);
  }
}

// ------------------------------------------------------------------ group sums
// red[w][s*4+v] = sum over warp w's rows i in V_s of f(i)_v, for s < h.
// Thread per row; groups are taken 4 per pass with predicated adds (no
// per-row shuffles).  FP32 windows of 16 rows carried by TwoSum.  f is called
// once per row in total (in the pass that holds the row's group).
template <typename F>
__device__ void group_sums_f32(Sm& S, int slot, int r0, int r1, int h, const uint8_t* lab, F&& f) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int s0 = 0; s0 < h; s0 += 4) {
    float win[4][kB];
    Comp acc[4][kB];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int v = 0; v < kB; ++v) {
        win[j][v] = 0.f;
        acc[j][v].zero();
      }
    int cnt = 0;
    for (int r = r0 + threadIdx.x; r < r1; r += kT) {
      const int g = (int)lab[r] - s0;
      if (g >= 0 && g < 4) {
        float x[kB];
        f(r, x);
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
          for (int v = 0; v < kB; ++v) win[j][v] += g == j ? x[v] : 0.f;
      }
      if (++cnt == 16) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
          for (int v = 0; v < kB; ++v) {
            acc[j][v].add(win[j][v]);
            win[j][v] = 0.f;
          }
        cnt = 0;
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int v = 0; v < kB; ++v) {
        acc[j][v].add(win[j][v]);
        comp_reduce(acc[j][v], 1);
      }
    if (lane == 0)
      for (int j = 0; j < 4 && s0 + j < h; ++j)
#pragma unroll
        for (int v = 0; v < kB; ++v) S.red[warp * slot + (s0 + j) * kB + v] = acc[j][v].slot();
  }
}

// The same in FP64 (setup and the final check): thread per row, 4 groups per pass.
template <typename F>
__device__ void group_sums_f64(Sm& S, int slot, int r0, int r1, int h, const uint8_t* lab, F&& f) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int s0 = 0; s0 < h; s0 += 4) {
    double acc[4][kB];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int v = 0; v < kB; ++v) acc[j][v] = 0.0;
    for (int r = r0 + threadIdx.x; r < r1; r += kT) {
      const int g = (int)lab[r] - s0;
      if (g >= 0 && g < 4) {
        double x[kB];
        f(r, x);
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (g == j)
#pragma unroll
            for (int v = 0; v < kB; ++v) acc[j][v] += x[v];
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int v = 0; v < kB; ++v) acc[j][v] = warp_allsum(acc[j][v]);
    if (lane == 0)
      for (int j = 0; j < 4 && s0 + j < h; ++j)
#pragma unroll
        for (int v = 0; v < kB; ++v) S.red[warp * slot + (s0 + j) * kB + v] = acc[j][v];
  }
}

// ------------------------------------------------------------------ ring streaming
// Streams rows [r0, r1) of panels 0..np-1 of V (and of U when withU) through
// the ring of shared-memory stages, one bulk copy per panel and stage, and
// calls consume(rg, nr, st) in every warp once per stage: the stage holds
// rows rg..rg+nr-1, V[rg+i][4p+j] at st[p*ps + 4i + j] and U[rg+i][j] at
// st[uoff + 4i + j] (ps = 4 stage_rows + 4, uoff = (jmax/4) ps).  Every wait
// is bounded; a timeout marks the CTA dead and drains the copies in flight.
template <typename F>
__device__ bool stream_rows(const Job& J, Sm& S, const Layout& L, unsigned* err, long& seq, int r0, int r1, int np,
                            bool withU, F&& consume) {
  if (S.ints[0]) return false;
  const int SR = L.stage_rows;
  const int ps = SR * 4 + 4;
  const int uoff = (L.jmax / 4) * ps;
  const int lane = threadIdx.x & 31;
  const int nchunks = (r1 - r0 + SR - 1) / SR;
  float* ring = reinterpret_cast<float*>(S.ring);
  const size_t panel = (size_t)J.n * 4;
  auto issue = [&](int g) {
    const int s = (int)((seq + g) % kStages);
    const int rg = r0 + g * SR;
    const int nr = min(SR, r1 - rg);
    const unsigned bytes = (unsigned)nr * 16u;
    float* st = ring + (size_t)s * L.stage_floats;
    mbar_arrive_expect_tx(&S.full[s], bytes * (unsigned)(np + (withU ? 1 : 0)));
    for (int p = 0; p < np; ++p) bulk_g2s(st + (size_t)p * ps, J.V + p * panel + (size_t)rg * 4, bytes, &S.full[s]);
    if (withU) bulk_g2s(st + uoff, J.U + (size_t)rg * 4, bytes, &S.full[s]);
  };
  // this CTA's generic-proxy writes of V and U must be ordered before the bulk reads
  fence_proxy_async();
  __syncthreads();
  if (threadIdx.x == 0) {
    S.ints[6] = 0;
    for (int g = 0; g < min(kStages, nchunks); ++g) issue(g);
  }
  __syncthreads();
  int g = 0;
  for (; g < nchunks; ++g) {
    const long q = seq + g;
    const int s = (int)(q % kStages);
    const unsigned par = (unsigned)((q / kStages) & 1);
    if (!mbar_wait(&S.full[s], par, err)) atomicExch(&S.ints[6], 1);
    if (*(volatile int*)&S.ints[6]) break;
    const int rg = r0 + g * SR;
    consume(rg, min(SR, r1 - rg), ring + (size_t)s * L.stage_floats);
    __syncwarp();
    if (lane == 0) mbar_arrive(&S.empty[s]);
    if (threadIdx.x == 0 && g + kStages < nchunks) {
      if (mbar_wait(&S.empty[s], par, err)) issue(g + kStages);
      else atomicExch(&S.ints[6], 1);
    }
  }
  __syncthreads();
  const bool aborted = S.ints[6] != 0;
  if (aborted && threadIdx.x == 0) {
    // drain every copy already issued (bounded), then give up on this CTA
    const int issued = min(nchunks, g + kStages);
    for (int gg = g; gg < issued; ++gg) {
      const long q = seq + gg;
      mbar_wait(&S.full[q % kStages], (unsigned)((q / kStages) & 1), err);
    }
    S.ints[0] = 1;
  }
  seq += nchunks;
  __syncthreads();
  return !aborted;
}

// Lanes per row for a row-group sweep over np panels (a power of two >= np).
__device__ __forceinline__ int lanes_for(int np) { return np <= 1 ? 1 : np <= 2 ? 2 : np <= 4 ? 4 : np <= 8 ? 8 : 16; }

// ------------------------------------------------------------------ operator pieces
template <typename VT>
__device__ __forceinline__ void load4(const VT* p, bool l2, VT (&y)[4]) {
  if constexpr (sizeof(VT) == 4) {
    const float4 t = l2 ? __ldcg(reinterpret_cast<const float4*>(p)) : *reinterpret_cast<const float4*>(p);
    y[0] = t.x;
    y[1] = t.y;
    y[2] = t.z;
    y[3] = t.w;
  } else {
    const double2* q = reinterpret_cast<const double2*>(p);
    const double2 a = l2 ? __ldcg(q) : q[0];
    const double2 b = l2 ? __ldcg(q + 1) : q[1];
    y[0] = a.x;
    y[1] = a.y;
    y[2] = b.x;
    y[3] = b.y;
  }
}

// ytil = D^{-1/2} P w for own rows, given the row coefficients of C a in S.coefA.
template <typename VT>
__device__ void op_ytil(const Job& J, const VT* cA, int r0, int r1, const VT* w, VT* ytil, const VT* dinv) {
  for (int r = r0 + threadIdx.x; r < r1; r += kT) {
    const int g = J.lab[r];
    const VT d = dinv[r];
#pragma unroll
    for (int v = 0; v < kB; ++v) ytil[(size_t)r * 4 + v] = d * (w[(size_t)r * 4 + v] - d * cA[g * kB + v]);
  }
}

// t = y - D^{-1/2} W ytil for own rows.  `lanes` lanes per row; each lane
// holds up to U (column, weight) pairs of its row per pass.  The FP32 path is
// software-pipelined over the warp's row groups: the pairs of the next group
// and the row bounds of the group after it are loaded while this group's
// ytil rows are gathered, so a group costs about one memory round trip.
// Other CTAs' ytil rows are read through L2 (team) or L1.
template <typename VT>
__device__ __forceinline__ void spmm_row_tail(const Job& J, bool team, const VT* ytil, int e, int e1, int Lr,
                                              VT (&s)[kB]) {
  for (; e < e1; e += Lr) {
    const int c = __ldg(J.col + e);
    const VT w = (VT)__ldg(J.val + e);
    VT y[4];
    load4(ytil + (size_t)c * 4, team, y);
#pragma unroll
    for (int v = 0; v < kB; ++v) s[v] += w * y[v];
  }
}

template <typename VT>
__device__ void op_spmm(const Job& J, const VT* cA, int r0, int r1, bool team, const VT* w, const VT* ytil,
                        const VT* dinv, VT* t_out) {
  constexpr int U = sizeof(VT) == 4 ? 8 : 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int Lr = J.lanes;
  const int sub = lane & (Lr - 1);
  const int rpw = 32 / Lr;
  const int stride = kW * rpw;
  auto bounds = [&](int rb, int& e, int& e1) {
    const int r = rb + lane / Lr;
    if (r < r1) {
      e = __ldg(J.row_ptr + r) + sub;
      e1 = __ldg(J.row_ptr + r + 1);
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
      c[u] = in ? __ldg(J.col + ee) : -1;
      wv[u] = in ? (VT)__ldg(J.val + ee) : VT(0);
    }
  };
  int rb = r0 + warp * rpw;
  int e_cur = 0, e1_cur = 0, e_nx = 0, e1_nx = 0;
  int c_cur[U];
  VT w_cur[U];
  bounds(rb, e_cur, e1_cur);
  fetch(e_cur, e1_cur, c_cur, w_cur);
  bounds(rb + stride, e_nx, e1_nx);
  for (; rb < r1; rb += stride) {
    int c_nx[U];
    VT w_nx[U];
    fetch(e_nx, e1_nx, c_nx, w_nx);  // next group's pairs, in flight during this group's gathers
    int e_nn, e1_nn;
    bounds(rb + 2 * stride, e_nn, e1_nn);
    VT s[kB] = {VT(0), VT(0), VT(0), VT(0)};
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (c_cur[u] >= 0) {
        VT y[4];
        load4(ytil + (size_t)c_cur[u] * 4, team, y);
#pragma unroll
        for (int v = 0; v < kB; ++v) s[v] += w_cur[u] * y[v];
      }
    }
    if (e_cur + U * Lr < e1_cur) spmm_row_tail(J, team, ytil, e_cur + U * Lr, e1_cur, Lr, s);
    for (int o = Lr >> 1; o > 0; o >>= 1)
#pragma unroll
      for (int v = 0; v < kB; ++v) s[v] += __shfl_xor_sync(0xffffffffu, s[v], o);
    const int r = rb + lane / Lr;
    if (r < r1 && sub == 0) {
      const int g = J.lab[r];
      const VT d = dinv[r];
#pragma unroll
      for (int v = 0; v < kB; ++v) {
        const VT y = w[(size_t)r * 4 + v] - d * cA[g * kB + v];
        t_out[(size_t)r * 4 + v] = y - d * s[v];
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

// ------------------------------------------------------------------ Cholesky QR helpers
// Upper Cholesky factor of the 4x4 Gram S.gram into R, and S.Rd, the divisor
// of U R^{-1}.  A pivot below 1e-10 of its reference (the column's norm
// before the projection, or its Gram diagonal) is a rank loss: that column
// is left unscaled and the call returns false.
__device__ bool chol4(Sm& S, double* R, const double* ref) {
  if (threadIdx.x == 0) {
    int ok = 1;
    for (int i = 0; i < 16; ++i) R[i] = S.Rd[i] = 0.0;
    for (int c = 0; c < kB; ++c) {
      double d = S.gram[c * kB + c];
      for (int q = 0; q < c; ++q) d -= R[q * kB + c] * R[q * kB + c];
      const double rf = ref ? ref[c] : S.gram[c * kB + c];
      if (!(d > 1e-10 * rf) || !(d > 0.0)) {
        ok = 0;
        R[c * kB + c] = d > 0.0 ? sqrt(d) : 0.0;
        S.Rd[c * kB + c] = 1.0;
        continue;
      }
      const double rc = sqrt(d);
      R[c * kB + c] = rc;
      S.Rd[c * kB + c] = rc;
      for (int q = c + 1; q < kB; ++q) {
        double s = S.gram[c * kB + q];
        for (int p = 0; p < c; ++p) s -= R[p * kB + c] * R[p * kB + q];
        R[c * kB + q] = s / rc;
        S.Rd[c * kB + q] = s / rc;
      }
    }
    S.ints[4] = ok;
    for (int i = 0; i < 16; ++i) S.Rdf[i] = (float)S.Rd[i];
    for (int v = 0; v < kB; ++v) S.Rdf[16 + v] = (float)(1.0 / S.Rd[v * kB + v]);
  }
  __syncthreads();
  return S.ints[4] != 0;
}

// u <- u R^{-1} (forward substitution over the 4 columns).
__device__ __forceinline__ void apply_rinv(const Sm& S, float (&u)[4]) {
#pragma unroll
  for (int v = 0; v < kB; ++v) {
    float s = u[v];
#pragma unroll
    for (int q = 0; q < v; ++q) s -= u[q] * S.Rdf[q * kB + v];
    u[v] = s * S.Rdf[16 + v];
  }
}

// FP32 window of the 10 unique Gram entries of one row.
__device__ __forceinline__ void gram_add(float (&g)[10], const float (&u)[4]) {
  int i = 0;
#pragma unroll
  for (int a = 0; a < kB; ++a)
#pragma unroll
    for (int b = a; b < kB; ++b) {
      g[i] = fmaf(u[a], u[b], g[i]);
      ++i;
    }
}

__device__ void gram_unpack(Sm& S, const double* t10) {
  if (threadIdx.x == 0) {
    int i = 0;
    for (int a = 0; a < kB; ++a)
      for (int b = a; b < kB; ++b) {
        S.gram[a * kB + b] = t10[i];
        S.gram[b * kB + a] = t10[i];
        ++i;
      }
  }
  __syncthreads();
}

// Gram (10 unique entries) of U's own rows, thread per row, after u <- u R^{-1}
// when `apply`; team-reduced into S.gram.
__device__ void gram_pass(const Job& J, Sm& S, Team& T, const Layout& L, int r0, int r1, bool apply) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float gw[10];
  Comp ga[10];
#pragma unroll
  for (int e = 0; e < 10; ++e) {
    gw[e] = 0.f;
    ga[e].zero();
  }
  int cnt = 0;
  for (int r = r0 + threadIdx.x; r < r1; r += kT) {
    const float4 t = *reinterpret_cast<const float4*>(J.U + (size_t)r * 4);
    float u[kB] = {t.x, t.y, t.z, t.w};
    if (apply) {
      apply_rinv(S, u);
      *reinterpret_cast<float4*>(J.U + (size_t)r * 4) = make_float4(u[0], u[1], u[2], u[3]);
    }
    gram_add(gw, u);
    if (++cnt == 16) {
#pragma unroll
      for (int e = 0; e < 10; ++e) {
        ga[e].add(gw[e]);
        gw[e] = 0.f;
      }
      cnt = 0;
    }
  }
#pragma unroll
  for (int e = 0; e < 10; ++e) {
    ga[e].add(gw[e]);
    comp_reduce(ga[e], 1);
  }
  __syncthreads();
  if (lane == 0)
    for (int e = 0; e < 10; ++e) S.red[warp * L.slot + e] = ga[e].slot();
  warps_to_loc_pairs(S, L.slot, 10);
  team_reduce(T, S, 10);
  gram_unpack(S, S.tot);
}

// Orthogonalise the block in U against V[:, 0:Jc] and append it as panel Jc/4.
// When `fin` is set U holds t = L_n y and is first finished as U - d coefD[g]
// (the last term of the operator).  Coefficients go to Hm[0:Jc, jcol:jcol+4]
// and the R factor to Hm[Jc:Jc+4, jcol:jcol+4] when jcol >= 0.  Leaves the
// group solve of D^{-1/2} times the new block in S.av / S.coefA for the next
// operator.  Returns false on a rank loss.
//
// The V sweeps take 32-row blocks per warp in two phases.  Phase A, one lane
// per row: finish or update the row of U (the update reads the row's Jc
// columns of V and the coefficients), store it, and add its Gram entries.
// Phase B, LPR lanes per row (lane p holds panel p, columns 4p..4p+3): add
// the row's products to the new coefficients V^T u.  Both phases read V and
// U with plain coalesced loads (phase B mostly from L1); sums accumulate in
// FP32 windows carried by TwoSum and are combined over lanes by a TwoSum tree.
__device__ bool orth_block(const Job& J, Sm& S, Team& T, const Layout& L, long& seq, int r0, int r1, int Jc, int jcol,
                           bool fin, int& sweeps) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int slot = L.slot, ldh = L.mmax + kB;
  const int h = J.h;
  const int np = Jc / 4;
  const int x0 = L.jmax * kB;  // extras offset in a slot
  const size_t pan = (size_t)J.n * 4;
  float* U = J.U;
  bool ok = true;
  (void)seq;
  if (Jc > 0) {
    const int LPR = lanes_for(np), RPW = 32 / LPR;
    const int p = lane & (LPR - 1), ri = lane / LPR;
    const bool own = p < np;
    float* uw = reinterpret_cast<float*>(S.red + warp * slot);  // this warp's 32 updated rows (phase A -> B)
    // sweep(kind): kind 1: finish (fin) + c = V^T u + norms;  kind 2: u -= V cf, c = V^T u, Gram;
    // kind 3: u -= V cf, Gram.  Leaves the coefficient sums in red[w][c*4+v] and the extras at x0.
    auto sweep = [&](int kind) {
      const bool upd = kind >= 2, want_c = kind <= 2;
      float win[4][kB], gw[10];
      Comp acc[4][kB], ga[10];
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int v = 0; v < kB; ++v) {
          win[j][v] = 0.f;
          acc[j][v].zero();
        }
#pragma unroll
      for (int e = 0; e < 10; ++e) {
        gw[e] = 0.f;
        ga[e].zero();
      }
      int nb = 0;
      for (int rb = r0 + warp * 32; rb < r1; rb += kW * 32) {
        // ---- phase A: lane = row
        const int r = rb + lane;
        float u[kB] = {0.f, 0.f, 0.f, 0.f};
        if (r < r1) {
          const float4 t = *reinterpret_cast<const float4*>(U + (size_t)r * 4);
          u[0] = t.x;
          u[1] = t.y;
          u[2] = t.z;
          u[3] = t.w;
          if (kind == 1 && fin) {
            const int g = J.lab[r];
            const float d = J.dinv[r];
#pragma unroll
            for (int v = 0; v < kB; ++v) u[v] -= d * S.coefDf[g * kB + v];
          }
          if (upd) {
            float q[kB] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
            for (int pp = 0; pp < np; ++pp) {
              const float4 x = *reinterpret_cast<const float4*>(J.V + pp * pan + (size_t)r * 4);
              const float xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const float4 c4 = *reinterpret_cast<const float4*>(S.cf + (4 * pp + j) * kB);
                q[0] = fmaf(xs[j], c4.x, q[0]);
                q[1] = fmaf(xs[j], c4.y, q[1]);
                q[2] = fmaf(xs[j], c4.z, q[2]);
                q[3] = fmaf(xs[j], c4.w, q[3]);
              }
            }
#pragma unroll
            for (int v = 0; v < kB; ++v) u[v] -= q[v];
          } else {
            // warm L1 with the row's panels for phase B
            for (int pp = 0; pp < np; ++pp)
              asm volatile("prefetch.global.L1 [%0];" ::"l"(J.V + pp * pan + (size_t)r * 4));
          }
          if (upd || fin) *reinterpret_cast<float4*>(U + (size_t)r * 4) = make_float4(u[0], u[1], u[2], u[3]);
        }
        if (kind == 1) {
          // input norms only: the Gram diagonal
          gw[0] = fmaf(u[0], u[0], gw[0]);
          gw[4] = fmaf(u[1], u[1], gw[4]);
          gw[7] = fmaf(u[2], u[2], gw[7]);
          gw[9] = fmaf(u[3], u[3], gw[9]);
        } else {
          gram_add(gw, u);
        }
        if (want_c) *reinterpret_cast<float4*>(uw + lane * 4) = make_float4(u[0], u[1], u[2], u[3]);
        __syncwarp();
        // ---- phase B: LPR lanes per row, lane p = panel p
        if (want_c && own) {
          const int nrow = min(32, r1 - rb);
          for (int s0 = 0; s0 < LPR; s0 += 4) {
            float4 xv[4], uv[4];
#pragma unroll
            for (int s = 0; s < 4; ++s) {
              const int i = ri + RPW * (s0 + s);
              const bool in = s0 + s < LPR && i < nrow;
              xv[s] = in ? *reinterpret_cast<const float4*>(J.V + p * pan + (size_t)(rb + i) * 4)
                         : make_float4(0.f, 0.f, 0.f, 0.f);
              uv[s] = in ? *reinterpret_cast<const float4*>(uw + i * 4) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int s = 0; s < 4; ++s) {
              const float xs[4] = {xv[s].x, xv[s].y, xv[s].z, xv[s].w};
              const float us[4] = {uv[s].x, uv[s].y, uv[s].z, uv[s].w};
#pragma unroll
              for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int v = 0; v < kB; ++v) win[j][v] = fmaf(xs[j], us[v], win[j][v]);
            }
          }
        }
        __syncwarp();
        if (++nb == 8) {
#pragma unroll
          for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int v = 0; v < kB; ++v) {
              acc[j][v].add(win[j][v]);
              win[j][v] = 0.f;
            }
#pragma unroll
          for (int e = 0; e < 10; ++e) {
            ga[e].add(gw[e]);
            gw[e] = 0.f;
          }
          nb = 0;
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int v = 0; v < kB; ++v) {
          acc[j][v].add(win[j][v]);
          comp_reduce(acc[j][v], LPR);
        }
#pragma unroll
      for (int e = 0; e < 10; ++e) {
        ga[e].add(gw[e]);
        comp_reduce(ga[e], 1);
      }
      zero_red(S, slot, x0 + 10);
      if (want_c && ri == 0 && own)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
          for (int v = 0; v < kB; ++v) S.red[warp * slot + (4 * p + j) * kB + v] = acc[j][v].slot();
      if (lane == 0)
#pragma unroll
        for (int e = 0; e < 10; ++e) S.red[warp * slot + x0 + e] = ga[e].slot();
      warps_to_loc_pairs(S, slot, x0 + 10);
      team_reduce(T, S, x0 + 10);
      ++sweeps;
    };
    // ---- sweep 1: (finish the operator) + c1 = V^T u + input norms
    sweep(1);
    gram_unpack(S, S.tot + x0);
    if (threadIdx.x < kB) S.misc[threadIdx.x] = S.gram[threadIdx.x * (kB + 1)];
    for (int i = threadIdx.x; i < Jc * kB; i += kT) {
      S.cf[i] = (float)S.tot[i];
      if (jcol >= 0) S.Hm[(size_t)(i / kB) + (size_t)ldh * (jcol + i % kB)] = S.tot[i];
    }
    __syncthreads();
    // ---- sweep 2 (u -= V c1; c2 = V^T u; Gram) and, on the DGKS test, sweep 3 (u -= V c2; Gram)
    for (int round = 0; round < 2; ++round) {
      sweep(round == 0 ? 2 : 3);
      gram_unpack(S, S.tot + x0);
      int again = 0;
      for (int v = 0; v < kB; ++v)
        if (S.gram[v * kB + v] < 0.5 * S.misc[v]) again = 1;  // DGKS: lost more than 1/sqrt(2) of its norm
      if (!again || round == 1) break;
      for (int i = threadIdx.x; i < Jc * kB; i += kT) {
        S.cf[i] = (float)S.tot[i];
        if (jcol >= 0) S.Hm[(size_t)(i / kB) + (size_t)ldh * (jcol + i % kB)] += S.tot[i];
      }
      __syncthreads();
    }
  } else {
    gram_pass(J, S, T, L, r0, r1, false);
  }
  // ---- Cholesky QR, twice
  ok = chol4(S, S.R1, Jc > 0 ? S.misc : nullptr);
  gram_pass(J, S, T, L, r0, r1, true);
  ok = chol4(S, S.R2, nullptr) && ok;
  // ---- final scaling into panel Jc/4 and the group sums of D^{-1/2} q for the next operator
  float* Vp = J.V + (size_t)(Jc / 4) * J.n * 4;
  group_sums_f32(S, slot, r0, r1, h, J.lab, [&](int r, float(&x)[kB]) {
    const float4 t = *reinterpret_cast<const float4*>(U + (size_t)r * 4);
    float u[kB] = {t.x, t.y, t.z, t.w};
    apply_rinv(S, u);
    *reinterpret_cast<float4*>(Vp + (size_t)r * 4) = make_float4(u[0], u[1], u[2], u[3]);
    const float d = J.dinv[r];
#pragma unroll
    for (int v = 0; v < kB; ++v) x[v] = d * u[v];
  });
  warps_to_loc_pairs(S, slot, h * kB);
  team_reduce(T, S, h * kB);
  if (h > 1) {
    solve_groups(S, S.tot, h, S.av, S.coefA, S.coefAf);
  } else {
    for (int i = threadIdx.x; i < kMaxH * kB; i += kT) {
      S.coefA[i] = S.av[i] = 0.0;
      S.coefAf[i] = 0.f;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && jcol >= 0) {
    for (int q = 0; q < kB; ++q)
      for (int v = 0; v < kB; ++v) {
        double s = 0.0;
        for (int pp = 0; pp < kB; ++pp) s += S.R2[q * kB + pp] * S.R1[pp * kB + v];
        S.Hm[(size_t)(Jc + q) + (size_t)ldh * (jcol + v)] = q <= v ? s : 0.0;
      }
  }
  __syncthreads();
  return ok;
}

// L_n^sigma on panel `pin` of V (FP32): U receives t = L_n y, S.coefD the row
// coefficients of C(b - sigma a); orth_block's first sweep subtracts them.
__device__ void operator_f32(const Job& J, Sm& S, Team& T, const Layout& L, int r0, int r1, int pin, double sigma) {
  const float* w = J.V + (size_t)pin * J.n * 4;
  op_ytil<float>(J, S.coefAf, r0, r1, w, J.ytil, J.dinv);
  team_barrier(T, S);
  op_spmm<float>(J, S.coefAf, r0, r1, T.size > 1, w, J.ytil, J.dinv, J.U);
  __syncthreads();
  if (J.h > 1) {
    group_sums_f32(S, L.slot, r0, r1, J.h, J.lab, [&](int r, float(&x)[kB]) {
      const float4 t = *reinterpret_cast<const float4*>(J.U + (size_t)r * 4);
      const float d = J.dinv[r];
      x[0] = d * t.x;
      x[1] = d * t.y;
      x[2] = d * t.z;
      x[3] = d * t.w;
    });
    warps_to_loc_pairs(S, L.slot, J.h * kB);
    team_reduce(T, S, J.h * kB);
    solve_groups(S, S.tot, J.h, S.coefD, S.cs);                   // b into coefD
    deflate_coef(S, J.h, sigma, S.coefD, S.av, S.coefD, S.coefDf);  // same thread reads b before writing
  } else {
    for (int i = threadIdx.x; i < kMaxH * kB; i += kT) {
      S.coefD[i] = 0.0;
      S.coefDf[i] = 0.f;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ Jacobi
// Round-robin pairing of the parallel cyclic Jacobi method (Brent and Luk,
// 1985): in round rr of N-1, index N-1 meets rr and (rr+t) meets (rr-t) mod N-1.
__device__ __forceinline__ void rr_pair(int rr, int t, int N, int& p, int& q) {
  const int M = N - 1;
  if (t == 0) {
    p = rr;
    q = M;
  } else {
    p = (rr + t) % M;
    q = (rr - t + M) % M;
  }
  if (p > q) {
    const int s = p;
    p = q;
    q = s;
  }
}

// Parallel cyclic Jacobi sweeps on the symmetric N x N matrix A (column-major,
// element type T), rotations accumulated into E.  Stops when the squared
// off-diagonal Frobenius norm is at most tol times the total, or after maxs
// sweeps.  Rotations with |a_pq| <= skip * sqrt(|a_pp a_qq|) are skipped
// (threshold Jacobi).  Rotation angles as in Golub and Van Loan, Matrix
// Computations, Sec. 8.5.
template <typename T>
__device__ void jacobi_sweeps(Sm& S, T* A, T* E, int N, int maxs, double tol, double skip) {
  const int half = N / 2;
  for (int sweep = 0; sweep < maxs; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = threadIdx.x; i < N * N; i += kT) {
      const double x = (double)A[i] * (double)A[i];
      tot += x;
      if (i % N != i / N) off += x;
    }
    off = cta_sum(S, off);
    tot = cta_sum(S, tot);
    if (!(off > tol * tot)) break;
    for (int rr = 0; rr < N - 1; ++rr) {
      if ((int)threadIdx.x < half) {
        int p, q;
        rr_pair(rr, threadIdx.x, N, p, q);
        const T apq = A[p + q * N];
        T c = T(1), s = T(0);
        if (fabs((double)apq) > skip * sqrt(fabs((double)A[p + p * N] * (double)A[q + q * N])) + 1e-300) {
          const T tau = (A[q + q * N] - A[p + p * N]) / (T(2) * apq);
          const T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
          c = T(1) / sqrt(T(1) + t * t);
          s = t * c;
        }
        S.cs[2 * threadIdx.x] = (double)c;
        S.cs[2 * threadIdx.x + 1] = (double)s;
        S.pq[2 * threadIdx.x] = p;
        S.pq[2 * threadIdx.x + 1] = q;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < half * N; i += kT) {  // rows p and q
        const int t = i / N, col = i % N;
        const T s = (T)S.cs[2 * t + 1];
        if (s == T(0)) continue;
        const T c = (T)S.cs[2 * t];
        const int p = S.pq[2 * t], q = S.pq[2 * t + 1];
        const T xp = A[p + col * N], xq = A[q + col * N];
        A[p + col * N] = c * xp - s * xq;
        A[q + col * N] = s * xp + c * xq;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < half * N; i += kT) {  // columns p and q, of A and of E
        const int t = i / N, row = i % N;
        const T s = (T)S.cs[2 * t + 1];
        if (s == T(0)) continue;
        const T c = (T)S.cs[2 * t];
        const int p = S.pq[2 * t], q = S.pq[2 * t + 1];
        const T xp = A[row + p * N], xq = A[row + q * N];
        A[row + p * N] = row == q ? T(0) : c * xp - s * xq;
        A[row + q * N] = row == p ? T(0) : s * xp + c * xq;
        const T ep = E[row + p * N], eq = E[row + q * N];
        E[row + p * N] = c * ep - s * eq;
        E[row + q * N] = s * ep + c * eq;
      }
      __syncthreads();
    }
  }
}

// Eigen-decomposition of the symmetric N x N matrix S.A (column-major, FP64),
// N even: eigenvalues ascending in S.theta, eigenvectors in the columns of S.A.
// Jacobi sweeps first run in FP32 on a copy (this GPU's FP32 rate is far above
// its FP64 rate); the FP32 eigenvector matrix is then made orthonormal in
// FP64 (one Newton-Schulz step, E <- E (3I - E^T E) / 2), the FP64 matrix is
// transformed to E^T A E, and FP64 Jacobi sweeps finish the diagonalisation
// to FP64 accuracy.  Scratch: S.Yf (N^2 floats) and the ring (2 N^2 floats, then N^2 doubles).
__device__ void jacobi_eig(Sm& S, int N) {
  double* A = S.A;
  double* E = S.E;
  float* Af = S.Yf;
  float* Ef = reinterpret_cast<float*>(S.ring);
  double* T2 = reinterpret_cast<double*>(S.ring);
  const int NN = N * N;
  for (int i = threadIdx.x; i < NN; i += kT) {
    Af[i] = (float)A[i];
    Ef[i] = (i % N == i / N) ? 1.f : 0.f;
  }
  __syncthreads();
  jacobi_sweeps<float>(S, Af, Ef, N, 12, 1e-13, 1e-9);
  for (int i = threadIdx.x; i < NN; i += kT) E[i] = (double)Ef[i];
  __syncthreads();
  // G = E^T E, then M = (3I - G) / 2 into T2
  for (int i = threadIdx.x; i < NN; i += kT) {
    const int a = i % N, b = i / N;
    double g = 0.0;
    for (int r = 0; r < N; ++r) g = fma(E[r + a * N], E[r + b * N], g);
    T2[i] = (a == b ? 1.5 : 0.0) - 0.5 * g;
  }
  __syncthreads();
  // E <- E M, one row per warp, in place
  {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r = warp; r < N; r += kW) {
      double o0 = 0.0, o1 = 0.0;
      for (int kk = 0; kk < N; ++kk) {
        const double e = E[r + kk * N];
        if (lane < N) o0 = fma(e, T2[kk + lane * N], o0);
        if (lane + 32 < N) o1 = fma(e, T2[kk + (lane + 32) * N], o1);
      }
      __syncwarp();
      if (lane < N) E[r + lane * N] = o0;
      if (lane + 32 < N) E[r + (lane + 32) * N] = o1;
      __syncwarp();
    }
  }
  __syncthreads();
  // B = A E into T2, then A <- E^T B
  for (int i = threadIdx.x; i < NN; i += kT) {
    const int a = i % N, b = i / N;
    double x = 0.0;
    for (int kk = 0; kk < N; ++kk) x = fma(A[a + kk * N], E[kk + b * N], x);
    T2[i] = x;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NN; i += kT) {
    const int a = i % N, b = i / N;
    double x = 0.0;
    for (int kk = 0; kk < N; ++kk) x = fma(E[kk + a * N], T2[kk + b * N], x);
    A[i] = x;
  }
  __syncthreads();
  // symmetrise (E^T A E is symmetric up to rounding), then FP64 sweeps
  for (int i = threadIdx.x; i < NN; i += kT) {
    const int a = i % N, b = i / N;
    if (a < b) {
      const double m = 0.5 * (A[a + b * N] + A[b + a * N]);
      A[a + b * N] = m;
      A[b + a * N] = m;
    }
  }
  __syncthreads();
  jacobi_sweeps<double>(S, A, E, N, kJacobiSweeps, 1e-28, 1e-18);
  // ascending order, ties by index
  if ((int)threadIdx.x < N) {
    const int i = threadIdx.x;
    const double di = A[i * (N + 1)];
    int rank = 0;
    for (int j = 0; j < N; ++j) {
      const double dj = A[j * (N + 1)];
      rank += (dj < di) || (dj == di && j < i);
    }
    S.pq[i] = rank;
    S.theta[rank] = di;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NN; i += kT) {
    const int row = i % N, col = i / N;
    A[row + S.pq[col] * N] = E[row + col * N];
  }
  __syncthreads();
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Seeded start block in U (uniform in [-0.5, 0.5)), own rows.
__device__ void random_block(const Job& J, int r0, int r1, uint64_t seed) {
  for (int r = r0 + threadIdx.x; r < r1; r += kT) {
    float u[kB];
#pragma unroll
    for (int v = 0; v < kB; ++v) {
      const uint64_t z = mix64(seed + ((uint64_t)r * 4 + v + 1) * 0x9E3779B97F4A7C15ull);
      u[v] = (float)((double)(z >> 11) * 0x1.0p-53 - 0.5);
    }
    *reinterpret_cast<float4*>(J.U + (size_t)r * 4) = make_float4(u[0], u[1], u[2], u[3]);
  }
}

// First row of rank's share when rows are weighted by nnz + 16 per row.
__device__ int split_row(const Job& J, int rank, int size) {
  if (rank <= 0) return 0;
  if (rank >= size) return J.n;
  const long long total = (long long)J.nnz + 16ll * J.n;
  const long long target = total * rank / size;
  int lo = 0, hi = J.n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if ((long long)__ldg(J.row_ptr + mid) + 16ll * mid >= target) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

// ------------------------------------------------------------------ setup
// Structure checks, degrees, D^{-1/2}, labels, |V_s|, S_s, the Cholesky factor
// of C^T C and sigma.  Returns a status; on success sigma is set and S.z,
// S.Lc hold z and the factor; own rows are [S.ints[2], S.ints[3]).
__device__ int setup_graph(const Job& J, const Params& prm, Sm& S, Team& T, const Layout& L, double& sigma) {
  const int n = J.n, h = J.h, slot = L.slot, tid = threadIdx.x;
  int status = SFAIRSC_OK;
  {  // row_ptr first, on a plain row split, so that every later read is in range
    const int a0 = (int)((long long)n * T.rank / T.size), a1 = (int)((long long)n * (T.rank + 1) / T.size);
    double bad = 0.0;
    for (int r = a0 + tid; r < a1; r += kT) {
      const int p0 = __ldg(J.row_ptr + r), p1 = __ldg(J.row_ptr + r + 1);
      if (p0 < 0 || p1 < p0 || p1 > J.nnz) bad += 1.0;
      if (r == 0 && p0 != 0) bad += 1.0;
      if (r == n - 1 && p1 != J.nnz) bad += 1.0;
    }
    bad = cta_sum(S, bad);
    if (tid == 0) S.loc[0] = bad;
    __syncthreads();
    team_reduce(T, S, 1);
    if (S.tot[0] != 0.0) status = SFAIRSC_ERR_BAD_CSR;
  }
  if (tid == 0) {
    S.ints[2] = split_row(J, T.rank, T.size);
    S.ints[3] = max(S.ints[2], split_row(J, T.rank + 1, T.size));
  }
  __syncthreads();
  const int r0 = S.ints[2], r1 = S.ints[3];
  if (status != SFAIRSC_OK) return status;
  // entries: column range, self loop, negative, non-finite, label range, symmetry (validate >= 2)
  double nbad[6] = {0, 0, 0, 0, 0, 0};
  for (int r = r0 + tid; r < r1; r += kT) {
    const int p0 = __ldg(J.row_ptr + r), p1 = __ldg(J.row_ptr + r + 1);
    double d = 0.0;
    int prev = -1;
    for (int e = p0; e < p1; ++e) {
      const int c = __ldg(J.col + e);
      const float w = __ldg(J.val + e);
      if (c < 0 || c >= n) {
        nbad[0] += 1.0;
        continue;
      }
      if (c == r) nbad[1] += 1.0;
      if (!isfinite(w)) nbad[3] += 1.0;
      else if (w < 0.f) nbad[2] += 1.0;
      if (prm.validate >= 2) {
        if (c <= prev) nbad[5] += 1.0;
        prev = c;
        int lo = __ldg(J.row_ptr + c), hi = __ldg(J.row_ptr + c + 1);
        int found = -1;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          const int cm = __ldg(J.col + mid);
          if (cm == r) {
            found = mid;
            break;
          }
          if (cm < r) lo = mid + 1;
          else hi = mid;
        }
        if (found < 0 || __ldg(J.val + found) != w) nbad[5] += 1.0;
      }
      d += (double)w;
    }
    const int g = __ldg(J.labels + r);
    if (g < 0 || g >= h) nbad[4] += 1.0;
    J.lab[r] = (uint8_t)(g < 0 || g >= h ? 0 : g);
    const double di = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
    J.dinv64[r] = di;
    J.dinv[r] = (float)di;
  }
  for (int i = 0; i < 6; ++i) {
    const double s = cta_sum(S, nbad[i]);
    if (tid == 0) S.loc[kBadOff + i] = s;
  }
  __syncthreads();
  // |V_s|, S_s = sum_{i in V_s} 1/d_i, isolated vertices
  group_sums_f64(S, slot, r0, r1, h, J.lab, [&](int r, double(&x)[kB]) {
    const double di = J.dinv64[r];
    x[0] = 1.0;
    x[1] = di * di;
    x[2] = di > 0.0 ? 0.0 : 1.0;
    x[3] = 0.0;
  });
  __syncthreads();
  for (int i = tid; i < h * kB; i += kT) {
    double s = 0.0;
    for (int w = 0; w < kW; ++w) s += S.red[w * slot + i];
    S.loc[i] = s;
  }
  __syncthreads();
  team_reduce(T, S, kBadOff + 6);
  if (tid == 0) {
    const double* bad = S.tot + kBadOff;
    int code = SFAIRSC_OK;
    if (bad[0] + bad[1] > 0.0) code = SFAIRSC_ERR_BAD_CSR;
    else if (bad[3] > 0.0) code = SFAIRSC_ERR_NONFINITE;
    else if (bad[2] > 0.0 || bad[5] > 0.0) code = SFAIRSC_ERR_BAD_CSR;
    else if (bad[4] > 0.0) code = SFAIRSC_ERR_INVALID_ARG;
    double iso = 0.0, Stot = 0.0;
    for (int s = 0; s < h; ++s) {
      iso += S.tot[s * kB + 2];
      Stot += S.tot[s * kB + 1];
    }
    if (code == SFAIRSC_OK && iso > 0.0) code = SFAIRSC_ERR_ISOLATED_VERTEX;
    for (int s = 0; s < h && code == SFAIRSC_OK; ++s)
      if (S.tot[s * kB] < 0.5) code = SFAIRSC_ERR_EMPTY_GROUP;
    if (code == SFAIRSC_OK) {
      for (int s = 0; s < h; ++s) S.z[s] = S.tot[s * kB] / n;
      // (C^T C)_ab = delta_ab S_a - z_b S_a - z_a S_b + z_a z_b sum S (a, b < h-1), then Cholesky
      for (int a = 0; a < h - 1 && code == SFAIRSC_OK; ++a)
        for (int b = 0; b <= a; ++b) {
          const double Sa = S.tot[a * kB + 1], Sb = S.tot[b * kB + 1];
          double sum = (a == b ? Sa : 0.0) - S.z[b] * Sa - S.z[a] * Sb + S.z[a] * S.z[b] * Stot;
          for (int q = 0; q < b; ++q) sum -= S.Lc[a * kMaxH + q] * S.Lc[b * kMaxH + q];
          if (a == b) {
            if (!(sum > 0.0)) {
              code = SFAIRSC_ERR_EMPTY_GROUP;
              break;
            }
            S.Lc[a * kMaxH + a] = sqrt(sum);
          } else {
            S.Lc[a * kMaxH + b] = sum / S.Lc[b * kMaxH + b];
          }
        }
    }
    S.ints[5] = code;
  }
  __syncthreads();
  status = S.ints[5];
  if (status != SFAIRSC_OK) return status;
  // sigma = ||L_n||_1 = 1 + max_j d_j^{-1/2} sum_i w_ij d_i^{-1/2} (other CTAs' d^{-1/2} through L2)
  team_barrier(T, S);
  double smax = 0.0;
  for (int r = r0 + tid; r < r1; r += kT) {
    double t = 0.0;
    const int e1 = __ldg(J.row_ptr + r + 1);
    for (int e = __ldg(J.row_ptr + r); e < e1; ++e) t += (double)__ldg(J.val + e) * __ldcg(J.dinv64 + __ldg(J.col + e));
    smax = fmax(smax, 1.0 + J.dinv64[r] * t);
  }
  {
    const int lane = tid & 31, warp = tid >> 5;
    smax = warp_max(smax);
    __syncthreads();
    if (lane == 0) S.red[warp] = smax;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < kW; ++w) s = fmax(s, S.red[w]);
      S.loc[0] = s;
    }
    __syncthreads();
  }
  team_reduce(T, S, 1, 1);
  sigma = S.tot[0];
  return SFAIRSC_OK;
}

// ------------------------------------------------------------------ final FP64 check
// For Ritz vectors i0..i0+3 (Y = S.A, mv rows): x = P V y in FP64, A x with
// the FP64 operator (x in range(P), so A x = P L_n x), Rayleigh quotients,
// residuals ||A x - lambda x|| / (sigma ||x||), and H = D^{-1/2} x / ||x|| with
// the sign making the largest-magnitude entry of x positive (lowest row on ties).
// Returns the largest residual among columns < k.
__device__ double final_check4(const Job& J, Sm& S, Team& T, const Layout& L, long& seq, int r0, int r1, int mv,
                               int i0, double sigma) {
  const int h = J.h, k = J.k, slot = L.slot, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  // Y[:, i0:i0+4] as FP32 pairs hi + lo for the compensated products below
  float* Yh = S.Yf;
  float* Yl = S.Yf + mv * kB;
  for (int i = tid; i < mv * kB; i += kT) {
    const int q = i / kB, v = i % kB;
    const double y = i0 + v < k ? S.A[q + (i0 + v) * mv] : 0.0;
    const float hi = (float)y;
    Yh[i] = hi;
    Yl[i] = (float)(y - (double)hi);
  }
  __syncthreads();
  // x = V y for own rows: Dot2 on V * Yhi plus a plain FP32 sum of V * Ylo,
  // as accurate as an FP64 product of the FP32 basis with Y
  const size_t pan = (size_t)J.n * 4;
  for (int r = r0 + tid; r < r1; r += kT) {
    Dot2 acc[kB];
    float lo[kB] = {0.f, 0.f, 0.f, 0.f};
    for (int q4 = 0; q4 < mv / 4; ++q4) {
      const float4 t = *reinterpret_cast<const float4*>(J.V + q4 * pan + (size_t)r * 4);
      const float xv[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const int q = 4 * q4 + jj;
        const float4 yh = *reinterpret_cast<const float4*>(Yh + q * kB);
        const float4 yl = *reinterpret_cast<const float4*>(Yl + q * kB);
        acc[0].add_prod(xv[jj], yh.x);
        acc[1].add_prod(xv[jj], yh.y);
        acc[2].add_prod(xv[jj], yh.z);
        acc[3].add_prod(xv[jj], yh.w);
        lo[0] = fmaf(xv[jj], yl.x, lo[0]);
        lo[1] = fmaf(xv[jj], yl.y, lo[1]);
        lo[2] = fmaf(xv[jj], yl.z, lo[2]);
        lo[3] = fmaf(xv[jj], yl.w, lo[3]);
      }
    }
#pragma unroll
    for (int v = 0; v < kB; ++v) J.X[(size_t)r * 4 + v] = acc[v].value() + (double)lo[v];
  }
  __syncthreads();
  if (h > 1)
    group_sums_f64(S, slot, r0, r1, h, J.lab, [&](int r, double(&x)[kB]) {
      const double d = J.dinv64[r];
#pragma unroll
      for (int v = 0; v < kB; ++v) x[v] = d * J.X[(size_t)r * 4 + v];
    });
  warps_to_loc(S, slot, h * kB);
  team_reduce(T, S, h * kB);
  if (h > 1) {
    solve_groups(S, S.tot, h, nullptr, S.coefA);
  } else {
    for (int i = tid; i < kMaxH * kB; i += kT) S.coefA[i] = 0.0;
    __syncthreads();
  }
  for (int r = r0 + tid; r < r1; r += kT) {
    const int g = J.lab[r];
    const double d = J.dinv64[r];
#pragma unroll
    for (int v = 0; v < kB; ++v) {
      const double x = J.X[(size_t)r * 4 + v] - d * S.coefA[g * kB + v];
      J.X[(size_t)r * 4 + v] = x;
      J.ytil64[(size_t)r * 4 + v] = d * x;
    }
  }
  __syncthreads();
  for (int i = tid; i < kMaxH * kB; i += kT) S.coefA[i] = 0.0;  // y = P x = x
  team_barrier(T, S);
  op_spmm<double>(J, S.coefA, r0, r1, T.size > 1, J.X, J.ytil64, J.dinv64, J.AX);
  __syncthreads();
  if (h > 1) {
    group_sums_f64(S, slot, r0, r1, h, J.lab, [&](int r, double(&x)[kB]) {
      const double d = J.dinv64[r];
#pragma unroll
      for (int v = 0; v < kB; ++v) x[v] = d * J.AX[(size_t)r * 4 + v];
    });
    warps_to_loc(S, slot, h * kB);
    team_reduce(T, S, h * kB);
    solve_groups(S, S.tot, h, S.av, S.cs);
    deflate_coef(S, h, sigma, S.av, nullptr, S.coefD);
  } else {
    for (int i = tid; i < kMaxH * kB; i += kT) S.coefD[i] = 0.0;
    __syncthreads();
  }
  double xx[kB] = {0, 0, 0, 0}, xa[kB] = {0, 0, 0, 0};
  for (int r = r0 + tid; r < r1; r += kT) {
    const int g = J.lab[r];
    const double d = J.dinv64[r];
#pragma unroll
    for (int v = 0; v < kB; ++v) {
      const double ax = J.AX[(size_t)r * 4 + v] - d * S.coefD[g * kB + v];
      J.AX[(size_t)r * 4 + v] = ax;
      const double x = J.X[(size_t)r * 4 + v];
      xx[v] = fma(x, x, xx[v]);
      xa[v] = fma(x, ax, xa[v]);
    }
  }
  for (int v = 0; v < kB; ++v) {
    const double a = cta_sum(S, xx[v]);
    const double b = cta_sum(S, xa[v]);
    if (tid == 0) {
      S.loc[v] = a;
      S.loc[kB + v] = b;
    }
  }
  __syncthreads();
  team_reduce(T, S, 2 * kB);
  double lam[kB], nx[kB];
#pragma unroll
  for (int v = 0; v < kB; ++v) {
    nx[v] = S.tot[v];
    lam[v] = nx[v] > 0.0 ? S.tot[kB + v] / nx[v] : 0.0;
  }
  __syncthreads();
  double rr[kB] = {0, 0, 0, 0}, bv[kB] = {-1, -1, -1, -1};
  int br[kB] = {0, 0, 0, 0};
  for (int r = r0 + tid; r < r1; r += kT) {
#pragma unroll
    for (int v = 0; v < kB; ++v) {
      const double x = J.X[(size_t)r * 4 + v];
      const double t = J.AX[(size_t)r * 4 + v] - lam[v] * x;
      rr[v] = fma(t, t, rr[v]);
      if (fabs(x) > bv[v]) {
        bv[v] = fabs(x);
        br[v] = r;
      }
    }
  }
  for (int v = 0; v < kB; ++v) {
    const double s = cta_sum(S, rr[v]);
    if (tid == 0) S.loc[v] = s;
  }
  __syncthreads();
  team_reduce(T, S, kB);
  double worst = 0.0;
  for (int v = 0; v < kB; ++v)
    if (i0 + v < k) worst = fmax(worst, sqrt(S.tot[v] / nx[v]) / sigma);
  // argmax |x| per column: warp shuffles on (value, row), then over warps, then over the team
#pragma unroll
  for (int v = 0; v < kB; ++v) {
    double b = bv[v];
    int rw = br[v];
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, b, o);
      const int orw = __shfl_xor_sync(0xffffffffu, rw, o);
      if (ob > b || (ob == b && orw < rw)) {
        b = ob;
        rw = orw;
      }
    }
    if (lane == 0) {
      S.red[warp * 8 + v] = b;
      S.red[warp * 8 + 4 + v] = (double)rw;
    }
  }
  __syncthreads();
  if (tid < kB) {
    double b = -1.0, rw = 0.0;
    for (int w = 0; w < kW; ++w) {
      const double ob = S.red[w * 8 + tid], orw = S.red[w * 8 + 4 + tid];
      if (ob > b || (ob == b && orw < rw)) {
        b = ob;
        rw = orw;
      }
    }
    S.loc[tid] = b;
    S.loc[kB + tid] = rw;
  }
  __syncthreads();
  team_reduce(T, S, 2 * kB, 2);
  if (tid < kB) {
    const int row = (int)S.tot[kB + tid];
    const double xv = __ldcg(J.X + (size_t)row * 4 + tid);
    S.misc[12 + tid] = (xv < 0.0 ? -1.0 : 1.0) / sqrt(nx[tid]);
    if (T.rank == 0 && i0 + tid < k) J.lam[i0 + tid] = lam[tid];
  }
  __syncthreads();
  if (J.H)
    for (int r = r0 + tid; r < r1; r += kT)
      for (int v = 0; v < kB && i0 + v < k; ++v)
        J.H[(size_t)r * k + i0 + v] = S.misc[12 + v] * J.dinv64[r] * J.X[(size_t)r * 4 + v];
  team_barrier(T, S);
  return worst;
}

// ------------------------------------------------------------------ one graph
__device__ void solve_graph(const Job& J, Stat* st, const Params& prm, Sm& S, Team& T, const Layout& L, long& seq) {
  const int n = J.n, h = J.h, k = J.k, m = J.m, ldh = L.mmax + kB, slot = L.slot;
  const int tid = threadIdx.x;
  double sigma = 0.0;
  const int status = setup_graph(J, prm, S, T, L, sigma);
  const int r0 = S.ints[2], r1 = S.ints[3];
  if (status != SFAIRSC_OK) {
    if (tid == 0 && T.rank == 0) {
      st->status = status;
      st->max_resid = INFINITY;
      st->sigma = sigma;
    }
    return;
  }
  int sweeps = 0;
  random_block(J, r0, r1, prm.seed);
  __syncthreads();
  orth_block(J, S, T, L, seq, r0, r1, 0, -1, false, sweeps);
  for (int i = tid; i < ldh * L.mmax; i += kT) S.Hm[i] = 0.0;
  __syncthreads();
  int j0 = 0, restarts = 0, matvecs = 0, breakdowns = 0, since_break = 1 << 20, checks = 0;
  uint64_t fresh = 0;
  double maxres = INFINITY;
  bool converged = false;
  for (;;) {
    int mv = m;
    bool broke = false;
    for (int j = j0; j < m; j += kB) {
      operator_f32(J, S, T, L, r0, r1, j / 4, sigma);
      matvecs += kB;
      if (!orth_block(J, S, T, L, seq, r0, r1, j + kB, j, true, sweeps)) {
        broke = true;
        mv = j + kB;
        ++breakdowns;
        break;
      }
    }
    since_break = broke ? 0 : since_break + 1;
    // projected matrix from the upper triangle of Hm, then its eigen-decomposition
    for (int i = tid; i < mv * mv; i += kT) {
      const int r = i % mv, c = i / mv;
      S.A[i] = r <= c ? S.Hm[r + (size_t)ldh * c] : S.Hm[c + (size_t)ldh * r];
    }
    __syncthreads();
    jacobi_eig(S, mv);
    // residual estimates ||B y_i[mv-4:mv]|| (B = the last R factor) of the k wanted Ritz pairs
    if (tid < 32) {
      int nconv = 0;
      for (int i = 0; i < min(k, mv); ++i) {
        double acc = 0.0;
        if (tid < kB) {
          double s = 0.0;
          for (int q = 0; q < kB; ++q)
            s += S.Hm[(size_t)(mv + tid) + (size_t)ldh * (mv - kB + q)] * S.A[(mv - kB + q) + i * mv];
          acc = s * s;
        }
        acc = warp_allsum(acc);
        nconv += sqrt(acc) <= prm.tol * sigma;
      }
      if (tid == 0) S.ints[5] = nconv;
    }
    __syncthreads();
    const bool out = restarts >= prm.max_restarts;
    const bool est_ok = mv >= k && S.ints[5] == k && since_break >= 1;
    if (out && mv < k) break;
    if ((est_ok || out) && S.ints[0] == 0) {
      ++checks;
      double worst = 0.0;
      for (int i0 = 0; i0 < k; i0 += kB) worst = fmax(worst, final_check4(J, S, T, L, seq, r0, r1, mv, i0, sigma));
      maxres = worst;
      if (maxres <= prm.tol || out) {
        converged = maxres <= prm.tol;
        break;
      }
      since_break = 0;
    }
    if (out || S.ints[0]) break;
    // ---- thick restart: V[:, 0:K] = V[:, 0:mv] Y[:, 0:K]; carry the newest block or start a fresh one
    int K = k + (m - k) / 2;
    K = max(K / kB * kB, (k + kB - 1) / kB * kB);
    K = min(K, min(m - kB, mv));
    for (int i = tid; i < mv * K; i += kT) {
      const int q = i % mv, c = i / mv;
      S.Yf[q * K + c] = (float)S.A[i];
    }
    __syncthreads();
    const bool carry = !broke;
    {
      // warp per 32/LPR rows, lane po of a row computing output panel po (4 columns)
      const int npo = K / 4;
      const int LPR = lanes_for(npo), RPW = 32 / LPR;
      const int po = (tid & 31) & (LPR - 1), ri = (tid & 31) / LPR;
      const int ps = L.stage_rows * 4 + 4;
      const size_t pan = (size_t)n * 4;
      stream_rows(J, S, L, T.err, seq, r0, r1, mv / 4 + (carry ? 1 : 0), false,
                  [&](int rg, int nr, const float* st) {
                    for (int i0 = (tid >> 5) * RPW; i0 < nr; i0 += kW * RPW) {
                      const int i = i0 + ri;
                      if (i >= nr) continue;
                      if (po < npo) {
                        float o[4] = {0.f, 0.f, 0.f, 0.f};
                        for (int q = 0; q < mv; ++q) {
                          const float x = st[(q >> 2) * ps + i * 4 + (q & 3)];
                          const float4 y = *reinterpret_cast<const float4*>(S.Yf + q * K + 4 * po);
                          o[0] = fmaf(x, y.x, o[0]);
                          o[1] = fmaf(x, y.y, o[1]);
                          o[2] = fmaf(x, y.z, o[2]);
                          o[3] = fmaf(x, y.w, o[3]);
                        }
                        *reinterpret_cast<float4*>(J.V + po * pan + (size_t)(rg + i) * 4) =
                            make_float4(o[0], o[1], o[2], o[3]);
                      }
                      if (carry && po == 0)
                        *reinterpret_cast<float4*>(J.V + (size_t)(K / 4) * pan + (size_t)(rg + i) * 4) =
                            *reinterpret_cast<const float4*>(st + (mv / 4) * ps + i * 4);
                    }
                  });
    }
    for (int i = tid; i < ldh * L.mmax; i += kT) S.Hm[i] = 0.0;
    __syncthreads();
    if (tid < K) S.Hm[(size_t)tid * (ldh + 1)] = S.theta[tid];
    __syncthreads();
    if (carry) {
      // group solve of D^{-1/2} times the carried block, for the next operator
      const float* Qp = J.V + (size_t)(K / 4) * n * 4;
      group_sums_f32(S, slot, r0, r1, h, J.lab, [&](int r, float(&x)[kB]) {
        const float4 t = *reinterpret_cast<const float4*>(Qp + (size_t)r * 4);
        const float d = J.dinv[r];
        x[0] = d * t.x;
        x[1] = d * t.y;
        x[2] = d * t.z;
        x[3] = d * t.w;
      });
      warps_to_loc_pairs(S, slot, h * kB);
      team_reduce(T, S, h * kB);
      if (h > 1) {
        solve_groups(S, S.tot, h, S.av, S.coefA, S.coefAf);
      } else {
        for (int i = tid; i < kMaxH * kB; i += kT) {
          S.coefA[i] = S.av[i] = 0.0;
          S.coefAf[i] = 0.f;
        }
        __syncthreads();
      }
    } else {
      ++fresh;
      random_block(J, r0, r1, prm.seed + fresh * 0x632BE59BD9B4E019ull);
      __syncthreads();
      orth_block(J, S, T, L, seq, r0, r1, K, -1, false, sweeps);
    }
    j0 = K;
    ++restarts;
  }
  if (tid == 0 && T.rank == 0) {
    st->status = converged ? SFAIRSC_OK : SFAIRSC_ERR_NOT_CONVERGED;
    st->restarts = restarts;
    st->matvecs = matvecs;
    st->breakdowns = breakdowns;
    st->max_resid = checks ? maxres : INFINITY;
    st->sigma = sigma;
  }
}

// ------------------------------------------------------------------ kernel
template <int MINB>
__global__ void __launch_bounds__(kT, MINB) batched_kernel(const __grid_constant__ Sched P) {
  extern __shared__ __align__(128) unsigned char smraw[];
  unsigned char* base = smraw + ((128u - (smem_u32(smraw) & 127u)) & 127u);
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages];
  __shared__ int ints[16];
  __shared__ double smallbuf[kMaxH + 4 * kMaxH * kB + 2 * kMaxM + 16 * 5];
  __shared__ int pq[2 * kMaxM];
  __shared__ float smallf[2 * kMaxH * kB + 20];
  const Layout& L = P.L;
  Sm S;
  S.red = reinterpret_cast<double*>(base + L.red);
  S.loc = reinterpret_cast<double*>(base + L.loc);
  S.tot = reinterpret_cast<double*>(base + L.tot);
  S.Hm = reinterpret_cast<double*>(base + L.hm);
  S.A = reinterpret_cast<double*>(base + L.A);
  S.E = reinterpret_cast<double*>(base + L.E);
  S.Yf = reinterpret_cast<float*>(base + L.yf);
  S.cf = reinterpret_cast<float*>(base + L.cf);
  S.Lc = reinterpret_cast<double*>(base + L.lc);
  S.ring = base + L.ring;
  double* sb = smallbuf;
  S.z = sb;
  sb += kMaxH;
  S.coefA = sb;
  sb += kMaxH * kB;
  S.coefD = sb;
  sb += kMaxH * kB;
  S.av = sb;
  sb += kMaxH * kB;
  S.cs = sb;
  sb += kMaxH * kB;
  S.theta = sb;
  sb += 2 * kMaxM;
  S.gram = sb;
  sb += 16;
  S.R1 = sb;
  sb += 16;
  S.R2 = sb;
  sb += 16;
  S.Rd = sb;
  sb += 16;
  S.misc = sb;
  S.pq = pq;
  S.coefAf = smallf;
  S.coefDf = smallf + kMaxH * kB;
  S.Rdf = smallf + 2 * kMaxH * kB;
  S.full = full;
  S.empty = empty;
  S.ints = ints;

  const int cta = blockIdx.x;
  Team T;
  const int t0 = P.cta_team0[cta];
  T.size = P.cta_size[cta];
  T.rank = cta - t0;
  T.bar = P.bar + 2 * t0;
  T.part = P.part + (size_t)t0 * 2 * L.slot;
  T.err = P.err;
  T.slot = L.slot;
  T.parity = 0;
  const int cls = P.cta_class[cta];
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kW);
    }
    mbar_fence_init();
    for (int i = 0; i < 16; ++i) ints[i] = 0;
  }
  __syncthreads();
  long seq = 0;
  const int cb = P.class_begin[cls], ce = P.class_begin[cls + 1];
  for (;;) {
    // the team's first CTA takes the next graph of its class and posts it to the team
    if (threadIdx.x == 0 && T.rank == 0) {
      const unsigned idx = atomicAdd(&P.class_next[cls], 1u);
      if (T.size == 1) ints[1] = (int)idx;
      else st_release_gpu(P.mailbox + t0, idx);
    }
    team_barrier(T, S);
    if (threadIdx.x == 0 && T.size > 1) ints[1] = (int)ld_acquire_gpu(P.mailbox + t0);
    __syncthreads();
    const long t = (long)cb + ints[1];
    team_barrier(T, S);  // every CTA has read the mailbox before it is written again
    if (t >= ce || ints[0]) break;
    const int g = P.order[t];
    solve_graph(P.jobs[g], P.stats + g, P.prm, S, T, L, seq);
    if (ints[0]) break;
  }
}

Layout make_layout(int mmax, int stage_target) {
  Layout L{};
  L.mmax = mmax;
  L.jmax = mmax + kB;
  L.slot = std::max(L.jmax * kB + 32, kBadOff + 8);
  const int bytes_per_row = (L.jmax / 4) * 16 + 16;
  int SR = stage_target / bytes_per_row;
  SR = std::max(16, SR / 16 * 16);
  L.stage_rows = SR;
  L.stage_floats = (L.jmax / 4) * (SR * 4 + 4) + SR * 4;
  int off = 0;
  auto take = [&](int bytes) {
    const int o = off;
    off += (bytes + 127) / 128 * 128;
    return o;
  };
  L.red = take(kW * L.slot * 8);
  L.loc = take(L.slot * 8);
  L.tot = take(L.slot * 8);
  L.hm = take((mmax + kB) * mmax * 8);
  L.A = take(mmax * mmax * 8);
  L.E = take(mmax * mmax * 8);
  L.yf = take(mmax * mmax * 4);
  L.cf = take(L.jmax * kB * 4);
  L.lc = take(kMaxH * kMaxH * 8);
  // the ring also serves as Jacobi scratch: 2 mmax^2 floats (or mmax^2 doubles)
  L.ring = take(std::max(kStages * L.stage_floats, 2 * mmax * mmax) * 4);
  L.total = off + 128;
  return L;
}

}  // namespace bat

// ====================================================================== host plan
struct BatchPlan {
  int count = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  sfairsc_opts opts{};
  std::vector<bat::Job> jobs;
  std::vector<double> cost;
  int mmax = 0;
  void* arena = nullptr;
  void* sched_mem = nullptr;
  bat::Job* djobs = nullptr;
  bat::Stat* dstats = nullptr;
  int* dorder = nullptr;
  int* dclass_begin = nullptr;
  unsigned* dclass_next = nullptr;
  int* dteam0 = nullptr;
  int* dsize = nullptr;
  int* dclass = nullptr;
  unsigned* dbar = nullptr;
  double* dpart = nullptr;
  unsigned* dmailbox = nullptr;
  unsigned* derr = nullptr;
  int maxcta = 0;
  int grid = 0, minb = 1, max_team = 1, nclasses = 0;
  double split = 0.5;
  bat::Layout L{};
  std::vector<bat::Stat> hstats;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaGraphExec_t gexec = nullptr;
  bool graph_tried = false;
  float ms_autotune = 0.f;
  int autotuned = 0;
  std::vector<int> team_sizes;  // teams per class size
};

namespace {

constexpr int kMaxClasses = 5;  // team sizes 1, 2, 4, 8, 16

template <int MINB>
int blocks_per_sm(size_t smem) {
  int per = 0;
  check_cuda(cudaFuncSetAttribute(bat::batched_kernel<MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
             "batched shared memory attribute");
  check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, bat::batched_kernel<MINB>, bat::kT, smem),
             "batched occupancy");
  return per;
}

// Team classes and the CTA partition.  A graph whose estimated cost exceeds
// `split` times the mean per-CTA load times the team size gets the next
// larger team (up to max_team CTAs); CTAs go to the classes greedily by the
// largest remaining cost per CTA; within a class graphs are queued largest first.
void build_schedule(BatchPlan& B, int ctas, int max_team, double split) {
  const int count = B.count;
  double total = 0.0;
  for (double c : B.cost) total += c;
  const double per_cta = total / ctas;
  std::vector<int> sizes;
  for (int s = 1; s <= max_team && (int)sizes.size() < kMaxClasses; s *= 2) sizes.push_back(s);
  const int ncls = (int)sizes.size();
  std::vector<int> cls(count);
  std::vector<double> ccost(ncls, 0.0);
  for (int i = 0; i < count; ++i) {
    int c = 0;
    while (c + 1 < ncls && B.cost[i] > split * per_cta * sizes[c]) ++c;
    cls[i] = c;
    ccost[c] += B.cost[i];
  }
  std::vector<int> nct(ncls, 0);
  int used = 0;
  for (int c = 0; c < ncls; ++c)
    if (ccost[c] > 0.0) {
      nct[c] = sizes[c];
      used += sizes[c];
    }
  if (used > ctas) fail(SFAIRSC_ERR_UNSUPPORTED, "batched schedule: not enough co-resident CTAs for the team sizes");
  for (;;) {
    int best = -1;
    double bl = -1.0;
    for (int c = 0; c < ncls; ++c) {
      if (ccost[c] <= 0.0 || used + sizes[c] > ctas) continue;
      const double load = ccost[c] / nct[c];
      if (load > bl) {
        bl = load;
        best = c;
      }
    }
    if (best < 0) break;
    nct[best] += sizes[best];
    used += sizes[best];
  }
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    if (cls[a] != cls[b]) return cls[a] < cls[b];
    return B.cost[a] > B.cost[b];
  });
  std::vector<int> class_begin(kMaxClasses + 1, 0);
  for (int i = 0; i < count; ++i) class_begin[cls[i] + 1]++;
  for (int c = 0; c < kMaxClasses; ++c) class_begin[c + 1] += class_begin[c];
  std::vector<int> team0, tsize, tclass;
  int cta = 0;
  B.team_sizes.assign(ncls, 0);
  for (int c = ncls - 1; c >= 0; --c)
    for (int t = 0; t < nct[c] / sizes[c]; ++t) {
      for (int r = 0; r < sizes[c]; ++r) {
        team0.push_back(cta);
        tsize.push_back(sizes[c]);
        tclass.push_back(c);
      }
      cta += sizes[c];
      B.team_sizes[c]++;
    }
  if (cta > B.maxcta) fail(SFAIRSC_ERR_UNSUPPORTED, "batched schedule larger than its tables");
  B.grid = cta;
  B.nclasses = ncls;
  B.max_team = max_team;
  B.split = split;
  check_cuda(cudaMemcpyAsync(B.dorder, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice, B.stream), "h2d");
  check_cuda(cudaMemcpyAsync(B.dclass_begin, class_begin.data(), sizeof(int) * (kMaxClasses + 1),
                             cudaMemcpyHostToDevice, B.stream),
             "h2d");
  check_cuda(cudaMemcpyAsync(B.dteam0, team0.data(), sizeof(int) * cta, cudaMemcpyHostToDevice, B.stream), "h2d");
  check_cuda(cudaMemcpyAsync(B.dsize, tsize.data(), sizeof(int) * cta, cudaMemcpyHostToDevice, B.stream), "h2d");
  check_cuda(cudaMemcpyAsync(B.dclass, tclass.data(), sizeof(int) * cta, cudaMemcpyHostToDevice, B.stream), "h2d");
  check_cuda(cudaStreamSynchronize(B.stream), "schedule upload");
}

void launch_batched(BatchPlan& B, cudaStream_t s) {
  check_cuda(cudaMemsetAsync(B.dclass_next, 0, sizeof(unsigned) * kMaxClasses, s), "memset");
  check_cuda(cudaMemsetAsync(B.dstats, 0, sizeof(bat::Stat) * B.count, s), "memset");
  check_cuda(cudaMemsetAsync(B.dbar, 0, sizeof(unsigned) * 2 * B.maxcta, s), "memset");
  check_cuda(cudaMemsetAsync(B.derr, 0, sizeof(unsigned), s), "memset");
  bat::Sched P;
  P.jobs = B.djobs;
  P.stats = B.dstats;
  P.order = B.dorder;
  P.class_begin = B.dclass_begin;
  P.class_next = B.dclass_next;
  P.cta_team0 = B.dteam0;
  P.cta_size = B.dsize;
  P.cta_class = B.dclass;
  P.bar = B.dbar;
  P.part = B.dpart;
  P.mailbox = B.dmailbox;
  P.err = B.derr;
  P.prm.tol = B.opts.tol;
  P.prm.max_restarts = B.opts.max_restarts;
  P.prm.validate = B.opts.validate;
  P.prm.seed = B.opts.seed;
  P.L = B.L;
  void* args[] = {&P};
  const void* fn = B.minb == 2 ? (const void*)bat::batched_kernel<2> : (const void*)bat::batched_kernel<1>;
  check_cuda(cudaLaunchCooperativeKernel(fn, dim3(B.grid), dim3(bat::kT), args, (size_t)B.L.total, s),
             "batched cooperative launch");
}

void check_batch_err(BatchPlan& B) {
  unsigned e = 0;
  check_cuda(cudaMemcpyAsync(&e, B.derr, sizeof(unsigned), cudaMemcpyDeviceToHost, B.stream), "d2h");
  check_cuda(cudaStreamSynchronize(B.stream), "batched solve");
  if (e & kErrBarrierTimeout) fail(SFAIRSC_ERR_DEVICE_TIMEOUT, "a team barrier or a copy wait timed out");
}

float run_timed(BatchPlan& B) {
  check_cuda(cudaEventRecord(B.ev0, B.stream), "event");
  launch_batched(B, B.stream);
  check_cuda(cudaEventRecord(B.ev1, B.stream), "event");
  check_batch_err(B);
  float ms = 0.f;
  check_cuda(cudaEventElapsedTime(&ms, B.ev0, B.ev1), "elapsed");
  return ms;
}

void configure(BatchPlan& B, int minb, int max_team, double split) {
  B.L = bat::make_layout(B.mmax, minb == 2 ? 8192 : 16384);
  const size_t smem = (size_t)B.L.total;
  const int per = minb == 2 ? blocks_per_sm<2>(smem) : blocks_per_sm<1>(smem);
  if (per < 1) fail(SFAIRSC_ERR_UNSUPPORTED, "batched kernel does not fit on an SM");
  if (minb == 2 && per < 2) fail(SFAIRSC_ERR_UNSUPPORTED, "two batched CTAs do not fit on an SM");
  int sms = 0;
  check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, B.device), "sm count");
  B.minb = minb;
  build_schedule(B, sms * minb, max_team, split);
  if (B.gexec) {
    cudaGraphExecDestroy(B.gexec);
    B.gexec = nullptr;
  }
  B.graph_tried = false;
}

// Capture the launch sequence (queue resets + the cooperative launch) once into a CUDA graph.
void capture_graph(BatchPlan& B) {
  B.graph_tried = true;
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  cudaGraph_t g = nullptr;
  bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    try {
      launch_batched(B, cs);
    } catch (const SfError&) {
      ok = false;
    }
    ok = (cudaStreamEndCapture(cs, &g) == cudaSuccess) && ok && g != nullptr;
  }
  if (ok && cudaGraphInstantiate(&B.gexec, g, 0) != cudaSuccess) B.gexec = nullptr;
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
  cudaStreamDestroy(cs);
}

}  // namespace

BatchPlan* batch_create(int count, const sfairsc_batch_graph* graphs, const sfairsc_opts* user_opts,
                        cudaStream_t stream) {
  if (count < 1 || !graphs) fail(SFAIRSC_ERR_INVALID_ARG, "count must be >= 1 and graphs non-null");
  auto B = std::make_unique<BatchPlan>();
  B->count = count;
  B->stream = stream;
  sfairsc_opts_default(&B->opts);
  if (user_opts) B->opts = *user_opts;
  if (!(B->opts.tol > 0.0) || B->opts.max_restarts < 1)
    fail(SFAIRSC_ERR_INVALID_ARG, "tol and max_restarts must be positive");
  check_cuda(cudaGetDevice(&B->device), "device");
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  size_t arena = 0;
  B->jobs.resize(count);
  B->cost.resize(count);
  for (int i = 0; i < count; ++i) {
    const sfairsc_batch_graph& G = graphs[i];
    const std::string who = "batched graph " + std::to_string(i) + ": ";
    if (G.n < 16 || G.n > (1ll << 30) || G.nnz < 1 || G.nnz > 0x7fffffffll || G.h < 1 || G.h > bat::kMaxH ||
        G.k < 1 || !G.row_ptr || !G.col_idx || !G.values || !G.group_labels || !G.eigenvalues)
      fail(SFAIRSC_ERR_INVALID_ARG, who + "argument out of range or null pointer");
    if (G.k > G.n - G.h + 1) fail(SFAIRSC_ERR_K_TOO_LARGE, who + "k > n - h + 1");
    bat::Job& J = B->jobs[i];
    std::memset(&J, 0, sizeof(J));
    J.n = (int)G.n;
    J.nnz = (int)G.nnz;
    J.h = G.h;
    J.k = G.k;
    int m = B->opts.basis > 0 ? B->opts.basis : std::max(2 * G.k + 2 * bat::kB, 20);
    m = (m + bat::kB - 1) / bat::kB * bat::kB;
    m = std::min(m, std::min(bat::kMaxM, (J.n / bat::kB) * bat::kB - bat::kB));
    if (m < G.k + bat::kB) fail(SFAIRSC_ERR_K_TOO_LARGE, who + "k needs a basis above 60 columns");
    J.m = m;
    J.ldv = m + bat::kB;
    const double avg = (double)G.nnz / (double)G.n;
    int lanes = 2;
    while (lanes < 32 && lanes * 8 < avg) lanes *= 2;
    J.lanes = lanes;
    J.row_ptr = G.row_ptr;
    J.col = G.col_idx;
    J.val = G.values;
    J.labels = G.group_labels;
    J.lam = G.eigenvalues;
    J.H = G.H;
    B->mmax = std::max(B->mmax, m);
    const size_t n = (size_t)J.n;
    arena += al(4 * n * J.ldv) + 2 * al(16 * n) + al(4 * n) + al(8 * n) + al(n) + 3 * al(32 * n);
    // bytes per Krylov step: CSR + gathers of the operator, and the Gram-Schmidt sweeps
    B->cost[i] = 24.0 * (double)G.nnz + 12.0 * (double)n * m;
  }
  if (cudaMalloc(&B->arena, arena) != cudaSuccess) {
    cudaGetLastError();
    fail(SFAIRSC_ERR_OOM, "batched workspace allocation failed");
  }
  {
    unsigned char* p = static_cast<unsigned char*>(B->arena);
    auto take = [&](size_t b) {
      void* q = p;
      p += al(b);
      return q;
    };
    for (auto& J : B->jobs) {
      const size_t n = (size_t)J.n;
      J.V = (float*)take(4 * n * J.ldv);
      J.U = (float*)take(16 * n);
      J.ytil = (float*)take(16 * n);
      J.dinv = (float*)take(4 * n);
      J.dinv64 = (double*)take(8 * n);
      J.lab = (uint8_t*)take(n);
      J.X = (double*)take(32 * n);
      J.AX = (double*)take(32 * n);
      J.ytil64 = (double*)take(32 * n);
    }
  }
  int sms = 0;
  check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, B->device), "sm count");
  B->maxcta = 2 * sms;
  const bat::Layout Lmax = bat::make_layout(B->mmax, 16384);
  const size_t slot = (size_t)Lmax.slot;
  size_t off = 0;
  auto sal = [&](size_t b) {
    const size_t o = off;
    off += al(b);
    return o;
  };
  const int mc = B->maxcta;
  const size_t o_jobs = sal(sizeof(bat::Job) * count), o_stats = sal(sizeof(bat::Stat) * count),
               o_order = sal(4 * (size_t)count), o_cb = sal(4 * 16), o_cn = sal(4 * 16), o_t0 = sal(4 * mc),
               o_sz = sal(4 * mc), o_cl = sal(4 * mc), o_bar = sal(8 * mc), o_part = sal(8 * slot * 2 * mc),
               o_mb = sal(4 * mc), o_err = sal(16);
  if (cudaMalloc(&B->sched_mem, off) != cudaSuccess) {
    cudaGetLastError();
    fail(SFAIRSC_ERR_OOM, "batched schedule allocation failed");
  }
  unsigned char* s = static_cast<unsigned char*>(B->sched_mem);
  B->djobs = (bat::Job*)(s + o_jobs);
  B->dstats = (bat::Stat*)(s + o_stats);
  B->dorder = (int*)(s + o_order);
  B->dclass_begin = (int*)(s + o_cb);
  B->dclass_next = (unsigned*)(s + o_cn);
  B->dteam0 = (int*)(s + o_t0);
  B->dsize = (int*)(s + o_sz);
  B->dclass = (int*)(s + o_cl);
  B->dbar = (unsigned*)(s + o_bar);
  B->dpart = (double*)(s + o_part);
  B->dmailbox = (unsigned*)(s + o_mb);
  B->derr = (unsigned*)(s + o_err);
  check_cuda(cudaMemcpyAsync(B->djobs, B->jobs.data(), sizeof(bat::Job) * count, cudaMemcpyHostToDevice, stream),
             "h2d");
  check_cuda(cudaEventCreate(&B->ev0), "event");
  check_cuda(cudaEventCreate(&B->ev1), "event");
  B->hstats.resize(count);
  configure(*B, 1, 16, 0.5);  // cost-model default; sfairsc_batch_autotune measures the alternatives
  return B.release();
}

// Time each candidate schedule once (after one warm-up solve) and keep the fastest.
void batch_autotune(BatchPlan& B) {
  struct Cand {
    int minb, max_team;
    double split;
  };
  const Cand cands[] = {{1, 16, 0.5}, {1, 8, 0.5}, {1, 16, 0.25}, {1, 16, 1.0}, {1, 4, 0.5},
                        {2, 16, 0.5}, {2, 8, 0.5}, {1, 1, 1.0}};
  const auto t0 = std::chrono::steady_clock::now();
  Cand best = cands[0];
  float best_ms = 1e30f;
  bool warmed = false;
  for (const Cand& c : cands) {
    try {
      configure(B, c.minb, c.max_team, c.split);
    } catch (const SfError& e) {
      if (e.code != SFAIRSC_ERR_UNSUPPORTED) throw;
      continue;
    }
    if (!warmed) {
      run_timed(B);
      warmed = true;
    }
    const float ms = run_timed(B);
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  configure(B, best.minb, best.max_team, best.split);
  B.autotuned = 1;
  B.ms_autotune = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

int batch_solve(BatchPlan& B, int32_t* status, sfairsc_batch_info* info) {
  if (!B.graph_tried) capture_graph(B);
  check_cuda(cudaEventRecord(B.ev0, B.stream), "event");
  if (B.gexec) check_cuda(cudaGraphLaunch(B.gexec, B.stream), "graph launch");
  else launch_batched(B, B.stream);
  check_cuda(cudaEventRecord(B.ev1, B.stream), "event");
  check_cuda(cudaMemcpyAsync(B.hstats.data(), B.dstats, sizeof(bat::Stat) * B.count, cudaMemcpyDeviceToHost, B.stream),
             "d2h");
  check_batch_err(B);
  float ms = 0.f;
  check_cuda(cudaEventElapsedTime(&ms, B.ev0, B.ev1), "elapsed");
  int rc = SFAIRSC_OK, nconv = 0;
  double worst = 0.0;
  long long restarts = 0, matvecs = 0, brk = 0;
  for (int i = 0; i < B.count; ++i) {
    const bat::Stat& st = B.hstats[i];
    if (status) status[i] = st.status;
    if (st.status == SFAIRSC_OK) ++nconv;
    else if (rc == SFAIRSC_OK) rc = st.status;
    worst = std::max(worst, st.max_resid);
    restarts += st.restarts;
    matvecs += st.matvecs;
    brk += st.breakdowns;
  }
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->status = rc;
    info->converged = nconv;
    info->breakdowns = (int32_t)brk;
    info->grid = B.grid;
    info->restarts = restarts;
    info->matvecs = matvecs;
    info->max_resid = worst;
    info->split = B.split;
    info->ms_solve = ms;
    info->ms_autotune = B.ms_autotune;
    info->ctas_per_sm = B.minb;
    info->max_team = B.max_team;
    info->autotuned = B.autotuned;
    info->cuda_graph = B.gexec != nullptr;
    info->smem_bytes = B.L.total;
    for (int c = 0; c < (int)B.team_sizes.size() && c < 5; ++c) info->teams[c] = B.team_sizes[c];
  }
  return rc;
}

void batch_destroy(BatchPlan* B) {
  if (!B) return;
  if (B->gexec) cudaGraphExecDestroy(B->gexec);
  if (B->ev0) cudaEventDestroy(B->ev0);
  if (B->ev1) cudaEventDestroy(B->ev1);
  if (B->arena) cudaFree(B->arena);
  if (B->sched_mem) cudaFree(B->sched_mem);
  delete B;
}

namespace {
template <typename F>
int batch_guarded(F&& f) {
  try {
    f();
    set_last_error("");
    return SFAIRSC_OK;
  } catch (const SfError& e) {
    set_last_error(e.msg);
    return e.code;
  } catch (const std::bad_alloc&) {
    set_last_error("host allocation failed");
    return SFAIRSC_ERR_OOM;
  } catch (...) {
    set_last_error("unexpected internal error");
    return SFAIRSC_ERR_CUDA;
  }
}
}  // namespace

}  // namespace sfairsc

extern "C" {

SFAIRSC_API int sfairsc_batch_create(sfairsc_batch** out, int32_t count, const sfairsc_batch_graph* graphs,
                                     const sfairsc_opts* opts, void* cuda_stream) {
  if (!out) return SFAIRSC_ERR_INVALID_ARG;
  *out = nullptr;
  return sfairsc::batch_guarded([&] {
    *out = reinterpret_cast<sfairsc_batch*>(
        sfairsc::batch_create(count, graphs, opts, static_cast<cudaStream_t>(cuda_stream)));
  });
}

SFAIRSC_API int sfairsc_batch_autotune(sfairsc_batch* b) {
  if (!b) return SFAIRSC_ERR_INVALID_ARG;
  return sfairsc::batch_guarded([&] { sfairsc::batch_autotune(*reinterpret_cast<sfairsc::BatchPlan*>(b)); });
}

SFAIRSC_API int sfairsc_batch_schedule(sfairsc_batch* b, int32_t ctas_per_sm, int32_t max_team, double split) {
  if (!b || (ctas_per_sm != 1 && ctas_per_sm != 2) || max_team < 1 || max_team > 16 ||
      (max_team & (max_team - 1)) != 0 || !(split >= 0.0))
    return SFAIRSC_ERR_INVALID_ARG;
  return sfairsc::batch_guarded([&] {
    sfairsc::BatchPlan& B = *reinterpret_cast<sfairsc::BatchPlan*>(b);
    sfairsc::configure(B, ctas_per_sm, max_team, split);
    B.autotuned = 0;
  });
}

SFAIRSC_API int sfairsc_batch_solve(sfairsc_batch* b, int32_t* status, sfairsc_batch_info* info) {
  if (!b) return SFAIRSC_ERR_INVALID_ARG;
  int rc = SFAIRSC_OK;
  const int g = sfairsc::batch_guarded(
      [&] { rc = sfairsc::batch_solve(*reinterpret_cast<sfairsc::BatchPlan*>(b), status, info); });
  return g != SFAIRSC_OK ? g : rc;
}

SFAIRSC_API int sfairsc_batch_stats(const sfairsc_batch* b, int32_t* restarts, int32_t* matvecs, double* resid) {
  if (!b) return SFAIRSC_ERR_INVALID_ARG;
  const sfairsc::BatchPlan& B = *reinterpret_cast<const sfairsc::BatchPlan*>(b);
  for (int i = 0; i < B.count; ++i) {
    if (restarts) restarts[i] = B.hstats[i].restarts;
    if (matvecs) matvecs[i] = B.hstats[i].matvecs;
    if (resid) resid[i] = B.hstats[i].max_resid;
  }
  return SFAIRSC_OK;
}

SFAIRSC_API int sfairsc_batch_destroy(sfairsc_batch* b) {
  sfairsc::batch_destroy(reinterpret_cast<sfairsc::BatchPlan*>(b));
  return SFAIRSC_OK;
}

SFAIRSC_API int sfairsc_solve_batched(int32_t count, const sfairsc_batch_graph* graphs, const sfairsc_opts* opts,
                                      int32_t* status, sfairsc_batch_info* info, void* cuda_stream) {
  sfairsc_batch* b = nullptr;
  int rc = sfairsc_batch_create(&b, count, graphs, opts, cuda_stream);
  if (rc != SFAIRSC_OK) return rc;
  rc = sfairsc_batch_solve(b, status, info);
  sfairsc_batch_destroy(b);
  return rc;
}

}  // extern "C"
