// Shared-memory windows for the SpMV of the fused operator.
//
// The operator gathers ytil_j = d_j^{-1/2} (P w)_j for every stored entry
// (i, j).  Without help those gathers are random 4..32-byte reads from L2,
// and at tens of millions of entries per launch their rate, not HBM, bounds
// the kernel.  Graphs whose vertices are numbered so that neighbours are
// close (the m-SBM numbers vertices cluster by cluster, App. B.2, and most
// edges stay inside a cluster) let each CTA stage a contiguous slice of ytil
// in shared memory and serve most of its gathers from there.
//
// Here, once per context: each 256-row chunk histograms its columns in bins
// of half a window; the window of the chunk is the pair of adjacent bins
// (a window starting at a multiple of half its length) that holds most of
// its entries.  Per CTA, consecutive chunks with the same window merge into
// a segment, and a segment keeps its window only when the gathers it saves
// (one 32-byte L2 sector each) outweigh the sectors of loading the window.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace sfairsc {

namespace {

constexpr int kChunkRows = 256;
constexpr int kMaxBins = 12288;  // 48 KB of shared counters

// chunk c: out[3c] = best window (index of its first bin), out[3c+1] = entries inside it, out[3c+2] = entries
__global__ void window_hist_kernel(int n, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                   int half, int nbins, int32_t* out) {
  extern __shared__ int hist[];
  __shared__ int best_c[32], best_i[32];
  const int ch = blockIdx.x;
  const int r0 = ch * kChunkRows, r1 = min(n, r0 + kChunkRows);
  for (int i = threadIdx.x; i < nbins; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  const int e0 = row_ptr[r0], e1 = row_ptr[r1];
  for (int base = e0; base < e1; base += blockDim.x) {
    const int e = base + threadIdx.x;
    const bool in = e < e1;
    const int bin = in ? __ldg(col + e) / half : -1;
    // one shared atomic per distinct bin in the warp
    const unsigned act = __ballot_sync(0xffffffffu, in);
    if (in) {
      const unsigned same = __match_any_sync(act, bin);
      if ((threadIdx.x & 31) == __ffs(same) - 1) atomicAdd(&hist[bin], __popc(same));
    }
  }
  __syncthreads();
  int bc = -1, bi = 0;
  for (int i = threadIdx.x; i < nbins; i += blockDim.x) {
    const int cnt = hist[i] + (i + 1 < nbins ? hist[i + 1] : 0);
    if (cnt > bc) {
      bc = cnt;
      bi = i;
    }
  }
  // first maximum in bin order
  for (int o = 16; o > 0; o >>= 1) {
    const int oc = __shfl_xor_sync(0xffffffffu, bc, o), oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (oc > bc || (oc == bc && oi < bi)) {
      bc = oc;
      bi = oi;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    best_c[warp] = bc;
    best_i[warp] = bi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (best_c[w] > bc || (best_c[w] == bc && best_i[w] < bi)) {
        bc = best_c[w];
        bi = best_i[w];
      }
    out[3 * ch] = bi;
    out[3 * ch + 1] = max(bc, 0);
    out[3 * ch + 2] = e1 - e0;
  }
}

}  // namespace

int window_rows_for(int b, int vs, size_t base_smem) {
  const long long cap = 232448 - (long long)((base_smem + 15) / 16 * 16) - 1024;  // 227 KB per CTA, less the rest
  const long long budget = std::min<long long>(196608, cap);
  long long rows = budget / ((long long)b * vs);
  rows &= ~7ll;  // a multiple of 8: window starts are multiples of 4 rows (16-byte aligned copies)
  return rows >= 256 ? (int)rows : 0;
}

WindowTable build_window_table(int n, const int32_t* row_ptr, const int32_t* col, const std::vector<int32_t>& cta_rows,
                               int win_rows, int bytes_per_row, void* (*alloc)(void*, size_t), void* alloc_ctx,
                               cudaStream_t s) {
  WindowTable t;
  if (win_rows <= 0 || n < 2 * kChunkRows) return t;
  const int half = win_rows / 2;
  const int nbins = (n + half - 1) / half;
  if (nbins > kMaxBins) return t;
  if (nbins < 3) return t;  // the whole vector nearly fits one window: L2 serves it well
  const int nchunks = (n + kChunkRows - 1) / kChunkRows;
  int32_t* dbuf = static_cast<int32_t*>(alloc(alloc_ctx, sizeof(int32_t) * 3 * (size_t)nchunks));
  window_hist_kernel<<<nchunks, 256, sizeof(int) * nbins, s>>>(n, row_ptr, col, half, nbins, dbuf);
  check_cuda(cudaGetLastError(), "window histogram launch");
  std::vector<int32_t> hb((size_t)3 * nchunks);
  check_cuda(cudaMemcpyAsync(hb.data(), dbuf, sizeof(int32_t) * hb.size(), cudaMemcpyDeviceToHost, s), "d2h");
  check_cuda(cudaStreamSynchronize(s), "window histogram");

  const int grid = (int)cta_rows.size() - 1;
  std::vector<int32_t> seg_row, seg_ws, cta_seg(grid + 1);
  const double load_sectors = (double)win_rows * bytes_per_row / 32.0;
  for (int c = 0; c < grid; ++c) {
    cta_seg[c] = (int32_t)seg_ws.size();
    const int r0 = cta_rows[c], r1 = cta_rows[c + 1];
    if (r1 <= r0) continue;
    int start = r0;
    int cur = hb[3 * (r0 / kChunkRows)];
    double saved = 0.0;
    auto close = [&]() {
      seg_row.push_back(start);
      const bool use = saved > load_sectors;
      seg_ws.push_back(use ? cur * half : -1);
      if (use) {
        ++t.windowed;
        t.in_window += (long long)saved;
      }
    };
    for (int ch = r0 / kChunkRows; ch * kChunkRows < r1; ++ch) {
      const int cr0 = std::max(r0, ch * kChunkRows), cr1 = std::min(r1, (ch + 1) * kChunkRows);
      const double part = (double)(cr1 - cr0) / (double)(std::min(n, (ch + 1) * kChunkRows) - ch * kChunkRows);
      if (hb[3 * ch] != cur) {
        close();
        start = cr0;
        cur = hb[3 * ch];
        saved = 0.0;
      }
      saved += part * hb[3 * ch + 1];
    }
    close();
  }
  cta_seg[grid] = (int32_t)seg_ws.size();
  // segment s covers rows [seg_row[s], seg_row[s + 1]): the CTAs' row ranges tile [0, n), so
  // a CTA's last segment ends where the next non-empty CTA's first one starts, and the last at n
  seg_row.push_back(n);
  t.nseg = (int)seg_ws.size();
  int32_t* d = static_cast<int32_t*>(alloc(alloc_ctx, sizeof(int32_t) * (seg_row.size() + seg_ws.size() + cta_seg.size())));
  check_cuda(cudaMemcpyAsync(d, seg_row.data(), sizeof(int32_t) * seg_row.size(), cudaMemcpyHostToDevice, s), "h2d");
  check_cuda(cudaMemcpyAsync(d + seg_row.size(), seg_ws.data(), sizeof(int32_t) * seg_ws.size(), cudaMemcpyHostToDevice,
                             s), "h2d");
  check_cuda(cudaMemcpyAsync(d + seg_row.size() + seg_ws.size(), cta_seg.data(), sizeof(int32_t) * cta_seg.size(),
                             cudaMemcpyHostToDevice, s), "h2d");
  check_cuda(cudaStreamSynchronize(s), "window table upload");
  t.win_rows = win_rows;
  t.seg_row = d;
  t.seg_ws = d + seg_row.size();
  t.cta_seg = d + seg_row.size() + seg_ws.size();
  return t;
}

}  // namespace sfairsc
