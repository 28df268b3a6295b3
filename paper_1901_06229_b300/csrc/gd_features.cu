// Features of the learned orientation proposer (one row of 48 per ligand and restart).
// Not part of the search kernel's sources, so the search kernel's measurements stay
// attached when this changes.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>

#include "gd_internal.h"

namespace gd {
namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ float warp_sum_f(float v) {
  // xor butterfly: every lane ends with the same bits
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = __fadd_rn(v, __shfl_xor_sync(FULL, v, off));
  return v;
}

// Pocket value under a point in grid units (g = x_rel inv_h + shift): the cell floor(g)
// per axis of the crop, 0 outside it.  Through the texture when the pocket has one
// (point sampling of unnormalised coordinates selects texel floor(g), and the border
// returns 0), else from the crop through L1.
__device__ __forceinline__ int grid_value(const PocketDev& pk, bool tex, float gx, float gy, float gz) {
  if (tex) return (int)tex3D<unsigned char>((cudaTextureObject_t)pk.tex, gx, gy, gz);
  const int ix = __float2int_rd(gx), iy = __float2int_rd(gy), iz = __float2int_rd(gz);
  if ((unsigned)ix >= (unsigned)pk.cx || (unsigned)iy >= (unsigned)pk.cy || (unsigned)iz >= (unsigned)pk.cz) return 0;
  return __ldg(pk.grid + (iz * pk.cy + iy) * pk.cx + ix);
}

// ---- features of the learned orientation proposer -----------------------------------
//
// For every (ligand, restart) 48 numbers: the restart's unit quaternion (w >= 0); atoms /
// 250 and rotamers / 60; radius of gyration / 10 A; the fraction of atoms in each of 16
// bins of width 0.75 A of distance to the centroid over [0, 12) A; and the pocket value /
// 255 under 25 atoms of the placed restart pose, chosen by farthest-point sampling
// (first the atom farthest from the centroid, then repeatedly the atom farthest from
// those chosen, ties to the smaller preorder id; cyclic when the ligand has < 25 atoms).
// One warp per ligand: the restart-independent part once, then a row per restart.
constexpr int NFEAT = 48, NFPS = 25, NHIST = 16;

// The restart-independent part of a ligand's features, for ligands of at most 32 NT
// atoms (NT atom slots per lane, all of them in use or empty): the centroid, each atom's
// squared distance to it, lane b's count of histogram bin b (b < 16), the sum of the
// squared distances, and the farthest-point samples in fps[].  The ligand's atoms are
// left in xs (preorder).
template <int NT>
__device__ __forceinline__ void ligand_features(const SearchArgs& a, int a0, int n, float4* xs, int* fps, int lane,
                                                float& cx, float& cy, float& cz, int& hist, float& r2sum) {
  const float4* x0 = a.xyz + a0;
  // the lane's atoms i = lane + 32 t (into shared memory), their input-order ids, and
  // their centroid sum
  unsigned id[NT];
  float sx = 0.f, sy = 0.f, sz = 0.f;
  __syncwarp();
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const int i = lane + 32 * t;
    id[t] = 0u;
    if (i < n) {
      const float4 v = x0[i];
      xs[i] = v;
      id[t] = a.perm[a0 + i];
      sx = __fadd_rn(sx, v.x);
      sy = __fadd_rn(sy, v.y);
      sz = __fadd_rn(sz, v.z);
    }
  }
  __syncwarp();
  sx = warp_sum_f(sx);
  sy = warp_sum_f(sy);
  sz = warp_sum_f(sz);
  cx = __fdiv_rn(sx, (float)n);
  cy = __fdiv_rn(sy, (float)n);
  cz = __fdiv_rn(sz, (float)n);
  // squared distance of each atom to the centroid, and the 16-bin histogram of the
  // distances: one ballot per bin and slot, lane b keeps bin b's count
  float mind[NT];
  hist = 0;
  r2sum = 0.f;
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const int i = lane + 32 * t;
    mind[t] = -1.f;
    int b = -1;
    if (i < n) {
      const float4 v = xs[i];
      const float dx = v.x - cx, dy = v.y - cy, dz = v.z - cz;
      const float d2 = dx * dx + dy * dy + dz * dz;
      mind[t] = d2;
      r2sum += d2;
      b = (int)floorf(sqrtf(d2) / 0.75f);
    }
#pragma unroll
    for (int bin = 0; bin < NHIST; ++bin) {
      const unsigned m = __ballot_sync(FULL, b == bin);
      if (lane == bin) hist += __popc(m);
    }
  }
  r2sum = warp_sum_f(r2sum);
  // farthest-point sampling
  const int nsel = n < NFPS ? n : NFPS;
  for (int k = 0; k < nsel; ++k) {
    // candidates within a relative 1e-4 of the farthest (in distance) count as tied;
    // the smallest input-order atom id among them wins
    float dmax2 = -1.f;
#pragma unroll
    for (int t = 0; t < NT; ++t) dmax2 = fmaxf(dmax2, mind[t]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) dmax2 = fmaxf(dmax2, __shfl_xor_sync(FULL, dmax2, off));
    const float thr2 = dmax2 * ((1.0f - 1e-4f) * (1.0f - 1e-4f));
    unsigned best = 0xFFFFFFFFu;  // (input id << 8) | preorder id
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int i = lane + 32 * t;
      if (i < n && mind[t] >= 0.f && mind[t] >= thr2) {
        const unsigned key = (id[t] << 8) | (unsigned)i;
        best = key < best ? key : best;
      }
    }
    best = __reduce_min_sync(FULL, best);
    const int sel = (int)(best & 0xFFu);  // preorder id (< 256)
    if (lane == 0) fps[k] = sel;
    const float4 vs = xs[sel];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int i = lane + 32 * t;
      if (i == sel) mind[t] = -1.f;
      else if (i < n && mind[t] >= 0.f) {
        const float4 v = xs[i];
        const float dx = v.x - vs.x, dy = v.y - vs.y, dz = v.z - vs.z;
        const float d2 = dx * dx + dy * dy + dz * dz;
        mind[t] = k == 0 ? d2 : fminf(mind[t], d2);
      }
    }
  }
}

__global__ void __launch_bounds__(256, 3) feature_kernel(const __grid_constant__ SearchArgs a, __nv_bfloat16* Xb,
                                                       float* Xf) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  __shared__ int fps_s[8][NFPS];
  __shared__ float inv_s[8][19];
  __shared__ float4 fx_s[8][NFPS];
  // per warp: the ligand's atoms (preorder, at most 256), later its 32 BF16 rows at a time
  // (written out contiguously)
  __shared__ float4 xs_s[8][256];
  __shared__ float v255[256];  // c / 255 (correctly rounded) for every grid value c
  static_assert(32 * NFEAT * 2 <= 256 * 16, "a warp's rows fit in its atom buffer");
  int* fps = fps_s[threadIdx.x >> 5];
  float* inv = inv_s[threadIdx.x >> 5];
  float4* fx = fx_s[threadIdx.x >> 5];
  float4* xs = xs_s[threadIdx.x >> 5];
  uint4* rows = reinterpret_cast<uint4*>(xs);
  const bool tex = a.pk.tex != 0;
  v255[threadIdx.x] = __fdiv_rn((float)threadIdx.x, 255.f);  // blockDim.x == 256
  __syncthreads();
  for (int li = gw; li < a.L; li += nw) {
    const int a0 = a.atom_off[li], n = a.atom_off[li + 1] - a0;
    const int R = a.rot_off[li + 1] - a.rot_off[li];
    const int nt = (n + 31) >> 5;  // atom slots in use per lane (<= 8)
    float cx, cy, cz, r2sum;
    int hist;
    if (nt <= 1) ligand_features<1>(a, a0, n, xs, fps, lane, cx, cy, cz, hist, r2sum);
    else if (nt <= 2) ligand_features<2>(a, a0, n, xs, fps, lane, cx, cy, cz, hist, r2sum);
    else if (nt <= 4) ligand_features<4>(a, a0, n, xs, fps, lane, cx, cy, cz, hist, r2sum);
    else ligand_features<8>(a, a0, n, xs, fps, lane, cx, cy, cz, hist, r2sum);
    const int nsel = n < NFPS ? n : NFPS;
    __syncwarp();
    // restart-independent features 4..22 and the sampled atoms (centred), per warp
    const int hb = __shfl_sync(FULL, hist, (lane - 3) & 31);  // lane 3 + b gets bin b
    if (lane < 19) {
      float v;
      if (lane == 0) v = (float)n / 250.f;
      else if (lane == 1) v = (float)R / 60.f;
      else if (lane == 2) v = sqrtf(r2sum / (float)n) / 10.f;
      else v = (float)hb / (float)n;
      inv[lane] = v;
    }
    if (lane < NFPS) {
      const float4 p = xs[fps[lane % nsel]];
      fx[lane] = make_float4(p.x - cx, p.y - cy, p.z - cz, 0.f);
    }
    __syncwarp();
    // one restart per lane: quaternion, the shared part, the 25 grid samples (through the
    // texture when the pocket has one: the same cell lookup in one instruction)
    for (int o0 = 0; o0 < a.O; o0 += 32) {
      const int o = o0 + lane;
      if (o < a.O) {
        const float* r = a.rmat + 9 * (size_t)o;
        const float r0 = __ldg(r + 0), r1 = __ldg(r + 1), r2 = __ldg(r + 2), r3 = __ldg(r + 3), r4 = __ldg(r + 4);
        const float r5 = __ldg(r + 5), r6 = __ldg(r + 6), r7 = __ldg(r + 7), r8 = __ldg(r + 8);
        float f[NFEAT];
        const float4 q = a.quat[o];
        f[0] = q.x;
        f[1] = q.y;
        f[2] = q.z;
        f[3] = q.w;
#pragma unroll
        for (int e = 0; e < 19; ++e) f[4 + e] = inv[e];
#pragma unroll
        for (int t = 0; t < NFPS; ++t) {
          const float4 d = fx[t];
          const float X = __fmaf_rn(r0, d.x, __fmaf_rn(r1, d.y, __fmul_rn(r2, d.z)));
          const float Y = __fmaf_rn(r3, d.x, __fmaf_rn(r4, d.y, __fmul_rn(r5, d.z)));
          const float Z = __fmaf_rn(r6, d.x, __fmaf_rn(r7, d.y, __fmul_rn(r8, d.z)));
          const float gx = __fmaf_rn(X, a.pk.inv_h, a.pk.shift[0]), gy = __fmaf_rn(Y, a.pk.inv_h, a.pk.shift[1]),
                      gz = __fmaf_rn(Z, a.pk.inv_h, a.pk.shift[2]);
          const int c = grid_value(a.pk, tex, gx, gy, gz);
          f[23 + t] = v255[c];
        }
        const size_t row = (size_t)li * a.O + o;
        if (Xb) {
#pragma unroll
          for (int g = 0; g < NFEAT / 8; ++g) {
            __align__(16) __nv_bfloat16 h[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) h[e] = __float2bfloat16(f[8 * g + e]);
            rows[lane * (NFEAT / 8) + g] = *reinterpret_cast<const uint4*>(h);
          }
        }
        if (Xf) {
          float4* dst = reinterpret_cast<float4*>(Xf + row * NFEAT);
#pragma unroll
          for (int g = 0; g < NFEAT / 4; ++g) dst[g] = make_float4(f[4 * g], f[4 * g + 1], f[4 * g + 2], f[4 * g + 3]);
        }
      }
      __syncwarp();
      if (Xb) {
        // rows li O + o0 .. are consecutive: 16-byte words of the group, lane-contiguous
        const int words = (a.O - o0 < 32 ? a.O - o0 : 32) * (NFEAT / 8);
        uint4* dst = reinterpret_cast<uint4*>(Xb + ((size_t)li * a.O + o0) * NFEAT);
        for (int q = lane; q < words; q += 32) dst[q] = rows[q];
      }
      __syncwarp();
    }
  }
}

// Resident feature-kernel blocks per SM on the current device (queried once per device).
cudaError_t feature_blocks_per_sm(int* per_sm) {
  static std::mutex mu;
  static std::map<int, int> known;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> g(mu);
  auto it = known.find(dev);
  if (it != known.end()) {
    *per_sm = it->second;
    return cudaSuccess;
  }
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, feature_kernel, 256, 0);
  if (e == cudaSuccess) known[dev] = *per_sm;
  return e;
}

}  // namespace

cudaError_t launch_features(const SearchArgs& a, __nv_bfloat16* Xb, float* Xf, int num_sms, cudaStream_t st) {
  if (a.L == 0) return cudaSuccess;
  // the restart rotations and quaternions (the pose-setup kernel's tables)
  cudaError_t e = launch_restart_tables(a, st);
  if (e != cudaSuccess) return e;
  // one wave of resident blocks (8 warps each, a ligand per warp at a time)
  int per_sm = 0;
  e = feature_blocks_per_sm(&per_sm);
  if (e != cudaSuccess) return e;
  int blocks = (a.L + 7) / 8;
  if (blocks > num_sms * std::max(per_sm, 1)) blocks = num_sms * std::max(per_sm, 1);
  feature_kernel<<<blocks, 256, 0, st>>>(a, Xb, Xf);
  return cudaGetLastError();
}

}  // namespace gd
