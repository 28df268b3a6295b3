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
  // orderable keys: larger prediction first, then smaller restart id
  // rank the k best; a ligand that falls back and searches only its kf < O best is
  // ranked on to kf (rows of topk are kt = kf < O ? kf : k long)
  const int kt = kf < O ? kf : k;
  float first = 0.f, last = 0.f;
  bool fallback = false;
  unsigned taken[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // bit per (lane, slot): restarts o = lane + 32 s
  for (int r = 0; r < kt; ++r) {
    if (r == k) {  // the k best are ranked: fall back?
      fallback = rule ? first - last > margin : first - last < margin;
      if (!fallback) break;
    }
    unsigned long long best = 0;
    for (int sidx = 0; sidx * 32 + lane < O && sidx < 8; ++sidx) {
      if (taken[sidx]) continue;
      const int o = sidx * 32 + lane;
      const unsigned u = __float_as_uint(p[o]);
      const unsigned ord = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
      const unsigned long long key = ((unsigned long long)ord << 32) | (0xFFFFFFFFu - (unsigned)o);
      best = key > best ? key : best;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long q = __shfl_xor_sync(FULL, best, off);
      best = q > best ? q : best;
    }
    const int o = (int)(0xFFFFFFFFu - (unsigned)(best & 0xFFFFFFFFu));
    if ((o & 31) == lane) taken[o >> 5] = 1;
    if (lane == 0) topk[(size_t)li * kt + r] = (uint16_t)o;
    if (r < k) {
      const float v = p[o];
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

// Exclusive scan of the counts in queue order (one block): off[p] for position p.
__global__ void scan_kernel(const int32_t* order, const int32_t* cnt, int L, int32_t* off, int32_t* total) {
  __shared__ int32_t part[1024];
  const int per = (L + blockDim.x - 1) / blockDim.x;
  const int p0 = threadIdx.x * per, p1 = min(L, p0 + per);
  int32_t s = 0;
  for (int p = p0; p < p1; ++p) s += cnt[order[p]];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t run = 0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      const int32_t v = part[t];
      part[t] = run;
      run += v;
    }
    *total = run;
  }
  __syncthreads();
  s = part[threadIdx.x];
  for (int p = p0; p < p1; ++p) {
    off[p] = s;
    s += cnt[order[p]];
  }
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
