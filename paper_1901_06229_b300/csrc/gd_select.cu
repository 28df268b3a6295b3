// Restart selection of the learned proposer: from the predicted scores of every
// (ligand, restart), the restarts each ligand's pruned search takes, as an item list in
// the work queue's order.  Not part of the search kernel's sources, so the search
// kernel's measurements stay attached when this changes.
#include <cuda_runtime.h>

#include <cstdint>

#include "gd_internal.h"

namespace gd {
namespace {

constexpr unsigned FULL = 0xffffffffu;

// ---- restart selection for the learned proposer ----------------------------------
//
// Per ligand (one warp): the k restarts of highest predicted score (ties to the smaller
// restart id) and the spread pred(1st) - pred(k-th).  The ligand falls back to its kf
// best restarts (every restart when kf >= O) when the spread is below `margin` (rule 0:
// the network cannot separate its top choices) or above it (rule 1: the network expects
// only a few restarts to be good, which is where a wrong top-k loses the best pose).
__global__ void select_kernel(const float* pred, int L, int O, int k, int kf, float margin, int rule, int32_t* cnt,
                              uint16_t* topk, float* spread) {
  const int lane = threadIdx.x & 31;
  const int li = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (li >= L) return;
  const float* p = pred + (size_t)li * O;
  // orderable keys of the lane's restarts o = lane + 32 s (larger prediction first),
  // loaded once; the ranking takes the largest key, ties to the smaller restart id
  unsigned ord[8];
  unsigned avail = 0u;  // bit s: restart lane + 32 s not ranked yet
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int o = s * 32 + lane;
    ord[s] = 0u;
    if (o < O) {
      const unsigned u = __float_as_uint(p[o]);
      ord[s] = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
      avail |= 1u << s;
    }
  }
  // rank the k best; a ligand that falls back and searches only its kf < O best is
  // ranked on to kf (rows of topk are kt = kf < O ? kf : k long)
  const int kt = kf < O ? kf : k;
  float first = 0.f, last = 0.f;
  bool fallback = false;
  for (int r = 0; r < kt; ++r) {
    if (r == k) {  // the k best are ranked: fall back?
      fallback = rule ? first - last > margin : first - last < margin;
      if (!fallback) break;
    }
    unsigned mx = 0u;
#pragma unroll
    for (int s = 0; s < 8; ++s)
      if ((avail >> s) & 1u) mx = ord[s] > mx ? ord[s] : mx;
    mx = __reduce_max_sync(FULL, mx);
    unsigned mine = 0xFFFFu;  // this lane's smallest restart holding the maximum
#pragma unroll
    for (int s = 7; s >= 0; --s)
      if (((avail >> s) & 1u) && ord[s] == mx) mine = (unsigned)(s * 32 + lane);
    const int o = (int)__reduce_min_sync(FULL, mine);
    if ((o & 31) == lane) avail &= ~(1u << (o >> 5));
    if (lane == 0) topk[(size_t)li * kt + r] = (uint16_t)o;
    if (r < k) {  // the prediction itself, back from its key
      const float v = __uint_as_float((mx & 0x80000000u) ? (mx & 0x7FFFFFFFu) : ~mx);
      if (r == 0) first = v;
      last = v;
    }
  }
  if (lane == 0) {
    const float sp = first - last;
    spread[li] = sp;
    cnt[li] = (rule ? sp > margin : sp < margin) ? (kf < O ? kf : O) : k;
  }
}

// Exclusive scan of the counts in queue order (one block of 1024 threads, 1024 positions
// at a time: warp shuffles, then the warps' totals): off[p] for position p.  The counts
// of up to 16 chunks are loaded before any is scanned, so their loads overlap.
__global__ void scan_kernel(const int32_t* order, const int32_t* cnt, int L, int32_t* off, int32_t* total) {
  __shared__ int32_t wsum[32];
  __shared__ int32_t chunk_total;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t carry = 0;
  int32_t pre[16];
  for (int base = 0; base < L; base += 1024) {
    const int c = (base >> 10) & 15;
    if (c == 0) {
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int p = base + 1024 * q + (int)threadIdx.x;
        pre[q] = p < L ? cnt[order[p]] : 0;
      }
    }
    int32_t v = pre[0];
#pragma unroll
    for (int q = 1; q < 16; ++q)
      if (q == c) v = pre[q];
    const int p = base + (int)threadIdx.x;
    int32_t x = v;  // inclusive scan within the warp
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int32_t y = __shfl_up_sync(FULL, x, d);
      if (lane >= d) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      const int32_t t = wsum[lane];
      int32_t y = t;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int32_t z = __shfl_up_sync(FULL, y, d);
        if (lane >= d) y += z;
      }
      wsum[lane] = y - t;  // exclusive: the warps before this one
      if (lane == 31) chunk_total = y;
    }
    __syncthreads();
    if (p < L) off[p] = carry + wsum[warp] + x - v;
    carry += chunk_total;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

// Items (rows li * O + o) of every ligand at its queue offset: its ranked restarts
// (rows of topk are kt long), or all of them in order when it searches every restart.
__global__ void items_kernel(const int32_t* order, const int32_t* cnt, const int32_t* off, const uint16_t* topk, int L,
                             int O, int kt, uint32_t* items) {
  const int lane = threadIdx.x & 31;
  const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (p >= L) return;
  const int li = order[p];
  const int c = cnt[li];
  uint32_t* dst = items + off[p];
  for (int s = lane; s < c; s += 32) {
    const int o = c == O && kt < O ? s : (int)topk[(size_t)li * kt + s];
    dst[s] = (uint32_t)li * (uint32_t)O + (uint32_t)o;
  }
}

}  // namespace

cudaError_t launch_selection(const SearchArgs& a, const float* pred, int k, int kf, float margin, int rule,
                             int32_t* cnt, uint16_t* topk, float* spread, int32_t* off, uint32_t* items,
                             int32_t* n_items, cudaStream_t st) {
  if (a.L == 0) return cudaSuccess;
  const int blocks = (a.L * 32 + 255) / 256;
  select_kernel<<<blocks, 256, 0, st>>>(pred, a.L, a.O, k, kf, margin, rule, cnt, topk, spread);
  scan_kernel<<<1, 1024, 0, st>>>(a.order, cnt, a.L, off, n_items);
  items_kernel<<<blocks, 256, 0, st>>>(a.order, cnt, off, topk, a.L, a.O, kf < a.O ? kf : k, items);
  return cudaGetLastError();
}

}  // namespace gd
