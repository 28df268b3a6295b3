// Tensor-core (tcgen05) kernels of the learned orientation proposer: a BF16 MLP
// 48 -> 256 -> 256 -> 1 with FP32 accumulation, trained and evaluated on the GPU.
//
// gemm_kernel computes D[m][n] = sum_k A[m][k] * B[n][k] for one 128-row block of A
// and up to 256 columns of B per CTA:
//   * operands are staged from global memory into shared memory in the K-major
//     "core matrix" layout the tensor core reads without swizzling (8 rows x 16 bytes
//     per core matrix; LBO = distance between core matrices along K, SBO = along M/N),
//     optionally transposing on the way in (operands stored [K][M] in memory);
//   * one thread issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32) into a TMEM
//     accumulator of 128 lanes x N columns and commits to an mbarrier;
//   * the epilogue reads TMEM with tcgen05.ld (each warp its 32 lanes) and applies
//     bias / ReLU / BF16 rounding / a fused dot product with the last layer.
// Every wait is bounded (clock64); on a timeout the kernel records an error, frees its
// TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <vector>

#include "gd_mlp.h"
#include "geodock_mlp.h"

namespace gd {
namespace {

constexpr int KC = 64;  // K elements staged per chunk (4 MMAs of K = 16)

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle (layout type 0), descriptor version 1.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor: D = F32, A = B = BF16, both K-major, M x N.
__host__ __device__ __forceinline__ uint32_t make_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* m, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(m)), "r"(count));
}

// Bounded wait for phase `parity`; false after ~2 s at the maximum clock.  Each try_wait
// may suspend the thread for up to 20 us (a hint) until the phase completes, so waiting
// warps poll the barrier's shared-memory word less often.
__device__ __forceinline__ bool mbar_wait(uint64_t* m, uint32_t parity) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(m)), "r"(parity), "r"(20000u)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > 4000000000LL) return false;
  }
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, bool acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"((uint32_t)acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* m) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(m))
               : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Stage rows [r0, r0 + rows) x K chunk [k0, k0 + kc) of an operand into the core-matrix
// layout at `dst` (row group g, K chunk c at g * (kc/8) * 128 + c * 128, row r % 8 at
// 16 bytes each).  trans: the operand is stored [K][rows] (element (r, k) at src[k * ld + r]).
// Rows or K beyond the matrix are zero-filled.  Consecutive threads take consecutive K
// chunks of a row (one 16-byte load each), or with trans consecutive rows of a K chunk
// (so that each of the eight element loads is coalesced across the warp).
__device__ void stage(uint8_t* dst, const __nv_bfloat16* src, int ld, int nrows_total, int ktotal, int r0, int rows,
                      int k0, int kc, bool trans) {
  const int chunks = kc / 8;
  for (int idx = threadIdx.x; idx < rows * chunks; idx += blockDim.x) {
    const int r = trans ? idx % rows : idx / chunks, c = trans ? idx / rows : idx % chunks;
    const int gr = r0 + r, gk = k0 + c * 8;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (gr < nrows_total) {
      if (!trans) {
        if (gk + 8 <= ktotal) v = *reinterpret_cast<const uint4*>(src + (size_t)gr * ld + gk);
        else {
          __nv_bfloat16 t[8];
          for (int e = 0; e < 8; ++e) t[e] = gk + e < ktotal ? src[(size_t)gr * ld + gk + e] : __float2bfloat16(0.f);
          v = *reinterpret_cast<uint4*>(t);
        }
      } else {
        __nv_bfloat16 t[8];
        for (int e = 0; e < 8; ++e) t[e] = gk + e < ktotal ? src[(size_t)(gk + e) * ld + gr] : __float2bfloat16(0.f);
        v = *reinterpret_cast<uint4*>(t);
      }
    }
    *reinterpret_cast<uint4*>(dst + (size_t)(r >> 3) * chunks * 128 + c * 128 + (r & 7) * 16) = v;
  }
}

__global__ void __launch_bounds__(128) gemm_kernel(const __grid_constant__ GemmArgs g) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sa = smem;                       // 128 x KC bf16 = 16 KB
  uint8_t* sb = smem + 128 * KC * 2;        // 256 x KC bf16 = 32 KB
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + 128 * KC * 2 + 256 * KC * 2);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * 128, n0 = blockIdx.y * 256;
  const int nt = g.N - n0 < 256 ? g.N - n0 : 256;  // multiple of 16 by contract
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_addr(tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    mbar_init(mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = make_idesc(128, nt);
  bool ok = true;
  uint32_t phase = 0;
  // this CTA's K range (all of K unless split)
  const int kb = g.partial ? (int)blockIdx.z * g.kslice : 0;
  const int ke = g.partial ? min(g.K, kb + g.kslice) : g.K;
  for (int k0 = kb; k0 < ke && ok; k0 += KC) {
    const int kc = ke - k0 < KC ? ke - k0 : KC;  // multiple of 16 by contract
    stage(sa, g.A, g.lda, g.M, ke, m0, 128, k0, kc, g.transA);
    stage(sb, g.B, g.ldb, g.N, ke, n0, nt, k0, kc, g.transB);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      tc_fence_after();
      const uint32_t sbo = (uint32_t)(kc / 8) * 128;
      for (int kk = 0; kk < kc / 16; ++kk) {
        const uint64_t da = make_desc(smem_addr(sa) + kk * 256, 128, sbo);
        const uint64_t db = make_desc(smem_addr(sb) + kk * 256, 128, sbo);
        mma_bf16(tmem, da, db, idesc, k0 > kb || kk > 0);
      }
      if (!(g.hold && k0 == kb)) mma_commit(mbar);
    }
    // one outcome for the whole block: every thread takes the same branch and barriers
    ok = __syncthreads_and(mbar_wait(mbar, phase)) != 0;
    if (!ok) break;  // phase stays that of the commit that did not arrive
    phase ^= 1;
    tc_fence_after();
  }
  if (!ok) {
    if (threadIdx.x == 0) {
      if (g.err) atomicExch(g.err, 1);
      // before TMEM is freed: one more commit, which arrives once every MMA queued so far
      // is complete (or the late one does), and a bounded wait for it
      mma_commit(mbar);
      mbar_wait(mbar, phase);
    }
  } else if (g.partial) {
    // this K range's raw sums (zeros if the range is empty) for reduce_splits
    const int row = m0 + warp * 32 + lane;
    float* out = g.partial + ((size_t)blockIdx.z * g.M + row) * g.N;
    for (int c0 = 0; c0 < nt; c0 += 32) {
      float v[32];
      if (kb < ke) {
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = 0.f;
      }
      if (row < g.M) {
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          if (c0 + i >= nt) break;
          out[n0 + c0 + i] = v[i];
        }
      }
    }
  } else {
    // epilogue: warp w owns rows 32w .. 32w + 31 (TMEM lanes)
    const int row = m0 + warp * 32 + lane;
    float dot = 0.f;
    for (int c0 = 0; c0 < nt; c0 += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (row < g.M) {
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int col = n0 + c0 + i;
          if (c0 + i >= nt) break;
          float x = v[i];
          if (g.bias) x += g.bias[col];
          if (g.relu) x = fmaxf(x, 0.f);
          if (g.C) g.C[(size_t)row * g.ldc + col] = x;
          if (g.Cb) g.Cb[(size_t)row * g.ldc + col] = __float2bfloat16(x);
          if (g.dotw) dot = fmaf(__bfloat162float(__float2bfloat16(x)), g.dotw[col], dot);
        }
      }
    }
    if (g.dotw && row < g.M) g.dot_out[row] = dot + g.dot_bias + (g.dot_bias_dev ? *g.dot_bias_dev : 0.f);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
}

// Fused inference: y = relu(relu(X W1^T + b1) W2^T + b2) . w3 + b3 for 128-row tiles.
// One persistent CTA per SM keeps W1 (28 KB, b1 folded in), W2 (128 KB), b2's MMA
// operands and w3 in shared memory and owns all 512 TMEM columns: layer 1 accumulates in
// columns [0, 256), layer 2 in [256, 512).  Warp 8 only issues MMAs: layer 1 of a tile
// once the eight epilogue warps have stored its X rows, then layer 2 four K = 16 slices
// at a time as epilogue 1 completes 32-column chunks of H1.  Epilogue warp w reads TMEM
// lanes 32 (w % 4) and columns 128 (w / 4) .. + 128.
//
// Both biases are added by MMAs, so that neither epilogue loads them from shared memory,
// where those loads waited behind the tensor core's operand reads:
//   * layer 1 runs over K = 64: X's 48 features, three columns of ones and 13 of zeros,
//     against W1's rows extended by b1 = hi + mid + lo (the BF16 rounding of b1, of
//     what it leaves, and of the rest: the three sum to the FP32 b1 exactly) and zeros;
//   * layer 2 starts with one more MMA, ones against b2 split the same way, which
//     writes b2 into the accumulator before the 16 slices of H1 W2^T add to it.
//
// The tensor pipe is kept fed across tiles:
//   * a tile's X rows live in the H1 slots of epilogue 1's first chunk (K columns
//     0-31 and 128-159 of H1), which layer 2 has finished reading after its first four
//     MMAs: the next tile's X, loaded into registers during epilogue 1, is stored then,
//     so its layer 1 queues right behind this tile's layer 2;
//   * when layer 2 completes, the warps copy their accumulator rows into registers and
//     release the accumulator at once, so the next tile's layer 2 can start as soon as
//     the first chunk of its epilogue 1 is written; ReLU and BF16 rounding of those rows
//     run while the next layer 1 does, and their dot with w3 once all of the next tile's
//     layer 2 is queued.
constexpr int INF_EPI = 256;                // epilogue threads (8 warps)
constexpr int INF_THREADS = INF_EPI + 32;   // + the issuing warp
// W1 holds 7 K chunks per row (X's 6 and b1's), 896 bytes per 8-row group: the last
// layer-1 MMA reads K chunks 6 and 7, and "chunk 7" of a row group is the first chunk of
// the next one (of W2 for the last group), finite weights that meet the zeros of H1's
// chunk 19 and so add exactly nothing.
constexpr size_t INF_W1 = 256 * 56 * 2, INF_W2 = 256 * 256 * 2, INF_H1 = 128 * 256 * 2;
// b2's operands for the first layer-2 MMA: B2 (b2 = hi + mid + lo per row, one K chunk
// per 8-row group, 128 bytes apart, "chunk 1" again the next group's and zeros after the
// last) and ONE (8 rows of ones in K columns 0-2 and zeros, read by every 8-row group
// of the tile: stride 0)
constexpr size_t INF_B2 = 256 * 16 + 128, INF_ONE = 256, INF_VEC = 256 * 4;  // + w3
constexpr size_t INF_BAR = 128;  // 12 mbarriers + the TMEM address
constexpr size_t INF_SMEM = INF_W1 + INF_W2 + INF_H1 + INF_B2 + INF_ONE + INF_VEC + INF_BAR;
constexpr int INF_XCH = 128 * 6 / INF_EPI;  // 16-byte X chunks per epilogue thread and tile (128 rows x 6)

// This thread's share of a tile's X rows, loaded into registers ahead of time (rows
// past M read as zero): chunk j is X row idx / 6, K chunk idx % 6 with idx = t + 256 j.
struct XRegs {
  uint4 v[INF_XCH];
};
__device__ __forceinline__ void x_load(XRegs& xr, const __nv_bfloat16* X, int M, int r0) {
#pragma unroll
  for (int j = 0; j < INF_XCH; ++j) {
    const int idx = threadIdx.x + INF_EPI * j, r = idx / 6, c = idx % 6;
    xr.v[j] = r0 + r < M ? __ldg(reinterpret_cast<const uint4*>(X + (size_t)(r0 + r) * 48 + c * 8))
                         : make_uint4(0u, 0u, 0u, 0u);
  }
}

// Store them into layer 1's A operand (K = 64) in H1's core-matrix layout (8-row groups
// 4096 bytes apart, 8-column K chunks 128 bytes apart) and make the stores visible to the
// tensor core: X's K chunks 0-3 go to H1 chunks 0-3 and X's K chunks 4-5 to H1 chunks
// 16-17, all of them slots of epilogue 1's first 32-column chunk; H1 chunks 18 (ones in
// K columns 48-50, which multiply b1's three parts) and 19 (zeros) complete K = 64.
__device__ __forceinline__ void x_store(uint8_t* h1s, const XRegs& xr) {
  {
    const int r = threadIdx.x & 127, kc = 18 + (threadIdx.x >> 7);
    const uint32_t one = 0x3F80u;  // BF16 1.0
    const uint4 v = kc == 18 ? make_uint4(one | (one << 16), one, 0u, 0u) : make_uint4(0u, 0u, 0u, 0u);
    *reinterpret_cast<uint4*>(h1s + (size_t)(r >> 3) * 4096 + kc * 128 + (r & 7) * 16) = v;
  }
#pragma unroll
  for (int j = 0; j < INF_XCH; ++j) {
    const int idx = threadIdx.x + INF_EPI * j, r = idx / 6, c = idx % 6;
    const int kc = c < 4 ? c : c + 12;
    *reinterpret_cast<uint4*>(h1s + (size_t)(r >> 3) * 4096 + kc * 128 + (r & 7) * 16) = xr.v[j];
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* m) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(m)) : "memory");
}

// bf16x2 of max(round(a), 0), max(round(b), 0): a in the low half.  ReLU after rounding
// equals rounding after ReLU (rounding keeps signs).
__device__ __forceinline__ uint32_t relu_bf16x2(float a, float b) {
  uint32_t r;
  asm("{\n .reg .b32 t, z;\n cvt.rn.bf16x2.f32 t, %2, %1;\n mov.b32 z, 0;\n max.bf16x2 %0, t, z;\n}"
      : "=r"(r)
      : "f"(a), "f"(b));
  return r;
}

// ReLU and BF16 rounding of 32 layer-2 accumulator columns (b2 already in them), packed
// in pairs.
__device__ __forceinline__ void e2_pack(const float (&v)[32], uint32_t* hp) {
#pragma unroll
  for (int e2 = 0; e2 < 16; ++e2) hp[e2] = relu_bf16x2(v[2 * e2], v[2 * e2 + 1]);
}

// Epilogue 1 of one 32-column chunk of this thread's row (b1 already in the
// accumulator): ReLU and BF16 rounding into H1.
__device__ __forceinline__ void e1_chunk(uint32_t taddr, int col0, uint8_t* h1s, int row) {
  float v[32];
  tmem_ld32(taddr, v);
#pragma unroll
  for (int c8 = 0; c8 < 4; ++c8) {
    const float* w = v + c8 * 8;
    const uint4 h = make_uint4(relu_bf16x2(w[0], w[1]), relu_bf16x2(w[2], w[3]), relu_bf16x2(w[4], w[5]),
                               relu_bf16x2(w[6], w[7]));
    const int kc = (col0 >> 3) + c8;
    *reinterpret_cast<uint4*>(h1s + (size_t)(row >> 3) * 4096 + kc * 128 + (row & 7) * 16) = h;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // H1 for the tensor core
  tc_fence_before();
}

// Epilogue 2 of the tile at row r0 from this thread's 128 packed layer-2 activations:
// the dot with w3 in column order; the second half's warps hand their partial dots to
// the first half's (through red and mbarriers 9 / 10; `handed` counts the hand-overs,
// pr / pf are the wait parities), which write y.  Returns ok && every wait completed; a
// lane that comes in with ok false skips the waits, and the warp still runs every other
// step together, so that it stays converged.
__device__ __forceinline__ bool e2_finish(const uint32_t (&hp)[64], const float* w3s, int col0, int half, int row,
                                          int lane, int r0, int M, float bias3, float* red, uint64_t* mbar,
                                          int& handed, uint32_t& pr, uint32_t& pf, float* y, bool ok) {
  const float4* ww = reinterpret_cast<const float4*>(w3s + col0);
  float dot = 0.f;
#pragma unroll
  for (int e4 = 0; e4 < 32; ++e4) {
    const float4 w = ww[e4];
    const uint32_t f = hp[2 * e4], g = hp[2 * e4 + 1];
    dot = fmaf(__uint_as_float(f << 16), w.x, dot);
    dot = fmaf(__uint_as_float(f & 0xFFFF0000u), w.y, dot);
    dot = fmaf(__uint_as_float(g << 16), w.z, dot);
    dot = fmaf(__uint_as_float(g & 0xFFFF0000u), w.w, dot);
  }
  if (half == 1) {
    if (handed > 0) {  // the previous partials have been read
      if (ok) ok = mbar_wait(mbar + 10, pf);
      pf ^= 1;
    }
    ++handed;
    red[row] = dot;
    __syncwarp();
    if (lane == 0) mbar_arrive(mbar + 9);
  } else {
    if (ok) ok = mbar_wait(mbar + 9, pr);
    pr ^= 1;
    __syncwarp();
    const float other = red[row];
    __syncwarp();
    if (lane == 0) mbar_arrive(mbar + 10);
    if (r0 + row < M) y[r0 + row] = dot + other + bias3;
  }
  return ok;
}

// A bias as one 16-byte K chunk of BF16: (hi, mid, lo, 0, 0, 0, 0, 0) with hi + mid + lo
// equal to b exactly (each remainder is exact in FP32 and the last has at most 8
// significant bits), for an MMA against ones.
__device__ __forceinline__ void split_bias(float b, uint8_t* dst) {
  const __nv_bfloat16 hi = __float2bfloat16_rn(b);
  const float r1 = b - __bfloat162float(hi);
  const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
  const __nv_bfloat16 lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
  __nv_bfloat16* k = reinterpret_cast<__nv_bfloat16*>(dst);
  k[0] = hi;
  k[1] = mid;
  k[2] = lo;
  for (int e = 3; e < 8; ++e) k[e] = __float2bfloat16_rn(0.f);
}

__global__ void __launch_bounds__(INF_THREADS, 1)
    mlp_infer_kernel(const __nv_bfloat16* X, int M, const __nv_bfloat16* W1b, const __nv_bfloat16* W2b,
                     const float* b1, const float* b2, const float* w3r, const float* b3, float* y, int* err,
                     int hold) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* w1s = smem;
  uint8_t* w2s = smem + INF_W1;
  uint8_t* h1s = smem + INF_W1 + INF_W2;
  uint8_t* b2o = smem + INF_W1 + INF_W2 + INF_H1;
  uint8_t* one = b2o + INF_B2;
  float* w3s = reinterpret_cast<float*>(one + INF_ONE);
  // mbar[0] layer 1 done, [1] layer 2 done, [7] layer 2's first four MMAs done (MMA
  // commits); [2] X rows copied in, [3 + c] chunk c of epilogue 1 written, [8] layer 2's
  // accumulator copied out (one arrival per epilogue warp); [9] the second half's
  // partial dots written, [10] read (four arrivals each); [11] the final commit after a
  // wait ran out (see the end of the kernel).  Every barrier completes one
  // phase per tile, and no warp can arrive twice on one before its phase completes:
  // each next arrival waits, directly or through the issuing warp, for every warp's
  // current one.
  uint64_t* mbar = reinterpret_cast<uint64_t*>(reinterpret_cast<uint8_t*>(w3s) + INF_VEC);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 12);
  __shared__ float red[128];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = (M + 127) / 128;
  if ((int)blockIdx.x >= ntiles) return;
  stage(w1s, W1b, 48, 256, 48, 0, 256, 0, 56, false);  // K columns 48-55 zero
  stage(w2s, W2b, 256, 256, 256, 0, 256, 0, 256, false);
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += INF_THREADS) {
    w3s[i] = w3r[i];
    split_bias(b2[i], b2o + (size_t)(i >> 3) * 128 + (i & 7) * 16);
    split_bias(b1[i], w1s + (size_t)(i >> 3) * 896 + 6 * 128 + (i & 7) * 16);  // W1 row i, K columns 48-55
  }
  if (threadIdx.x < 24) {  // ONE: 8 rows of (1, 1, 1, 0, 0, 0, 0, 0), then 8 of zeros; B2's trailing zeros
    const uint32_t o = 0x3F80u;  // BF16 1.0
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    if (threadIdx.x < 16) reinterpret_cast<uint4*>(one)[threadIdx.x] = threadIdx.x < 8 ? make_uint4(o | (o << 16), o, 0u, 0u) : z;
    else reinterpret_cast<uint4*>(b2o + 4096)[threadIdx.x - 16] = z;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_addr(tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    mbar_init(mbar, 1);
    mbar_init(mbar + 1, 1);
    for (int b = 2; b < 7; ++b) mbar_init(mbar + b, INF_EPI / 32);
    mbar_init(mbar + 7, 1);
    mbar_init(mbar + 8, INF_EPI / 32);
    mbar_init(mbar + 9, INF_EPI / 64);
    mbar_init(mbar + 10, INF_EPI / 64);
    mbar_init(mbar + 11, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // W1 / W2 for the tensor core
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot, acc1 = tmem, acc2 = tmem + 256;
  bool ok = true;
  if (warp == INF_EPI / 32) {
    // ---- issuing warp
    if (lane == 0) {
      const uint32_t idesc = make_idesc(128, 256);
      // Every operand sits at a fixed shared-memory address, so each MMA's descriptors are
      // these bases with the start-address field (the low 14 bits, in 16-byte units)
      // advanced by a compile-time offset: a few integer adds per MMA, which keeps the
      // single issuing thread ahead of the tensor pipe.
      const uint64_t dh = make_desc(smem_addr(h1s), 128, 4096), dw1 = make_desc(smem_addr(w1s), 128, 896),
                     dw2 = make_desc(smem_addr(w2s), 128, 4096), db2 = make_desc(smem_addr(b2o), 128, 128),
                     done = make_desc(smem_addr(one), 128, 0);
      uint32_t px = 0, pc = 0, pd = 0;  // parities: X stored, epilogue-1 chunks, accumulator copied
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        ok = mbar_wait(mbar + 2, px);
        px ^= 1;
        if (!ok) break;
        tc_fence_after();
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)  // X's K chunks 0-3 and 16-17, then the ones (18-19), of H1's slots
          mma_bf16(acc1, dh + (uint64_t)((kk < 2 ? kk * 256 : (16 + 2 * (kk - 2)) * 128) >> 4),
                   dw1 + (uint64_t)((kk * 256) >> 4), idesc, kk > 0);
        if (!(hold && tile == (int)blockIdx.x)) mma_commit(mbar);  // hold (a test): the wait on it runs out
        if (tile != (int)blockIdx.x) {  // the previous layer 2 copied out
          ok = mbar_wait(mbar + 8, pd);
          pd ^= 1;
          if (!ok) break;
          tc_fence_after();
        }
        mma_bf16(acc2, done, db2, idesc, false);  // layer 2 starts from b2
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          ok = mbar_wait(mbar + 3 + c, pc);
          if (!ok) break;
          tc_fence_after();
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int k = t < 2 ? 2 * c + t : 8 + 2 * c + (t - 2);  // K slices of chunk c
            mma_bf16(acc2, dh + (uint64_t)((k * 256) >> 4), dw2 + (uint64_t)((k * 256) >> 4), idesc, true);
          }
          if (c == 0) mma_commit(mbar + 7);
        }
        pc ^= 1;
        if (ok) mma_commit(mbar + 1);
      }
    }
    __syncwarp();
  } else {
    // ---- epilogue warps
    const int quad = warp & 3, half = warp >> 2;
    const uint32_t lanebase = ((uint32_t)(quad * 32) << 16) + (uint32_t)(half * 128);
    const int row = quad * 32 + lane, col0 = half * 128;
    const float bias3 = *b3;
    uint32_t ph1 = 0, ph2 = 0, ph7 = 0, pr = 0, pf = 0;
    int prev_r0 = -1;   // first row of the tile whose layer-2 rows sit in acc
    int handed = 0;     // partial dots the second half has handed over so far
    uint32_t hp[64];    // this thread's 128 layer-2 activations of tile prev_r0 (BF16 pairs)
    XRegs xr;           // the next tile's X rows, in flight during epilogue 1
    x_load(xr, X, M, (int)blockIdx.x * 128);
    x_store(h1s, xr);
    __syncwarp();
    if (lane == 0) mbar_arrive(mbar + 2);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      const int r0 = tile * 128, next = tile + (int)gridDim.x;
      if (next < ntiles) x_load(xr, X, M, next * 128);
      // Waits inside a tile: each lane records its outcome and the warp goes on together
      // (no branch on it before the vote after the layer-2 wait), so the warp reaches
      // every .sync.aligned instruction converged; a timed-out lane skips the tile's
      // later waits.
      ok = mbar_wait(mbar, ph1);  // layer 1 of this tile
      ph1 ^= 1;
      __syncwarp();
      tc_fence_after();
      for (int c = 0; c < 4; ++c) {
        e1_chunk(acc1 + lanebase + (uint32_t)(32 * c), col0 + 32 * c, h1s, row);
        __syncwarp();
        if (lane == 0) mbar_arrive(mbar + 3 + c);
      }
      // all of this tile's layer 2 is queued.  Once its first MMAs are done, their H1
      // slots take the next tile's X rows (loaded during epilogue 1), so the next layer 1
      // queues behind this layer 2 before the previous tile is finished
      if (next < ntiles) {
        if (ok) ok = mbar_wait(mbar + 7, ph7);
        ph7 ^= 1;
        __syncwarp();
        tc_fence_after();
        x_store(h1s, xr);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(mbar + 2);
      }
      if (prev_r0 >= 0) ok = e2_finish(hp, w3s, col0, half, row, lane, prev_r0, M, bias3, red, mbar, handed, pr, pf, y, ok);
      if (ok) ok = mbar_wait(mbar + 1, ph2);  // layer 2 done: copy its rows out, release it
      ph2 ^= 1;
      if (!__all_sync(0xffffffffu, ok)) {  // the warp's one outcome for this tile
        ok = false;
        break;
      }
      tc_fence_after();
      {
        float v[2][32];
#pragma unroll
        for (int k = 0; k < 2; ++k) tmem_ld32(acc2 + lanebase + (uint32_t)(32 * k), v[k]);
#pragma unroll
        for (int k = 0; k < 2; ++k) e2_pack(v[k], hp + 16 * k);
#pragma unroll
        for (int k = 0; k < 2; ++k) tmem_ld32(acc2 + lanebase + (uint32_t)(64 + 32 * k), v[k]);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(mbar + 8);
#pragma unroll
        for (int k = 0; k < 2; ++k) e2_pack(v[k], hp + 32 + 16 * k);  // during the next layer 1
      }
      prev_r0 = r0;
    }
    if (ok && prev_r0 >= 0)
      ok = e2_finish(hp, w3s, col0, half, row, lane, prev_r0, M, bias3, red, mbar, handed, pr, pf, y, ok);
  }
  // A wait that ran out anywhere in the block: before the tensor memory is freed, the
  // issuing thread commits once more and waits (bounded) for that commit, which arrives
  // when every MMA it has queued is complete.
  if (__syncthreads_or(!ok)) {
    if (warp == INF_EPI / 32 && lane == 0) {
      mma_commit(mbar + 11);
      mbar_wait(mbar + 11, 0);
    }
    if (threadIdx.x == 0 && err) atomicExch(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

}  // namespace

// Operand staging (48 KB) plus 32 KB of headroom: at most two CTAs share an SM, so the
// two 256-column TMEM allocations always fit the SM's 512 columns.  (The inference
// kernel takes all 512 columns, but its 226 KB of shared memory keeps any other
// tensor-core CTA off its SM.)
size_t gemm_smem_bytes() { return 128 * KC * 2 + 256 * KC * 2 + 16 + 32 * 1024; }

// Dynamic shared-memory limit of a kernel, raised once per device (any host thread).
cudaError_t smem_attr_once(const void* fn, size_t bytes, std::atomic<bool>* done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (done[dev].load(std::memory_order_acquire)) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done[dev].store(true, std::memory_order_release);
  return e;
}

cudaError_t infer_launch(const __nv_bfloat16* X, int M, const __nv_bfloat16* W1b, const __nv_bfloat16* W2b,
                         const float* b1, const float* b2, const float* w3r, const float* b3, float* y, int* err,
                         int hold, int num_sms, cudaStream_t st) {
  static std::atomic<bool> attr[64];
  const size_t smem = INF_SMEM;
  cudaError_t e = smem_attr_once((const void*)mlp_infer_kernel, smem, attr);
  if (e != cudaSuccess) return e;
  if (M <= 0) return cudaSuccess;
  const int tiles = (M + 127) / 128;
  mlp_infer_kernel<<<tiles < num_sms ? tiles : num_sms, INF_THREADS, smem, st>>>(X, M, W1b, W2b, b1, b2, w3r, b3, y,
                                                                                 err, hold);
  return cudaGetLastError();
}

cudaError_t gemm_launch(const GemmArgs& g, cudaStream_t st) {
  static std::atomic<bool> attr[64];
  cudaError_t e = smem_attr_once((const void*)gemm_kernel, gemm_smem_bytes(), attr);
  if (e != cudaSuccess) return e;
  dim3 grid((g.M + 127) / 128, (g.N + 255) / 256, g.partial ? g.ksplit : 1);
  gemm_kernel<<<grid, 128, gemm_smem_bytes(), st>>>(g);
  return cudaGetLastError();
}

__global__ void k_reduce_splits(const float* partial, int S, int M, int N, float* C, int ldc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M * N) return;
  float s = 0.f;
  for (int z = 0; z < S; ++z) s += partial[(size_t)z * M * N + i];
  C[(size_t)(i / N) * ldc + i % N] = s;
}

cudaError_t reduce_splits(const float* partial, int S, int M, int N, float* C, int ldc, cudaStream_t st) {
  k_reduce_splits<<<(M * N + 255) / 256, 256, 0, st>>>(partial, S, M, N, C, ldc);
  return cudaGetLastError();
}

}  // namespace gd

extern "C" gd_status gd_mlp_gemm(const void* A, int lda, int transA, const void* B, int ldb, int transB, float* C,
                                 void* Cb, int ldc, int M, int N, int K, const float* bias, int relu,
                                 const float* dotw, float dot_bias, float* dot_out, int* dev_err, void* stream) {
  if (!A || !B || M < 1 || N < 16 || K < 16 || N % 16 || K % 16) return GD_EINVAL;
  if (dotw && (N > 256 || !dot_out)) return GD_EINVAL;
  if ((!transA && (lda < K || lda % 8)) || (transA && lda < M) || (!transB && (ldb < K || ldb % 8)) ||
      (transB && ldb < N))
    return GD_EINVAL;
  gd::GemmArgs g{};
  g.A = (const __nv_bfloat16*)A;
  g.B = (const __nv_bfloat16*)B;
  g.lda = lda;
  g.ldb = ldb;
  g.ldc = ldc;
  g.M = M;
  g.N = N;
  g.K = K;
  g.transA = transA != 0;
  g.transB = transB != 0;
  g.bias = bias;
  g.relu = relu != 0;
  g.C = C;
  g.Cb = (__nv_bfloat16*)Cb;
  g.dotw = dotw;
  g.dot_bias = dot_bias;
  g.dot_out = dot_out;
  g.err = dev_err;
  return gd::gemm_launch(g, (cudaStream_t)stream) == cudaSuccess ? GD_OK : GD_ECUDA;
}

// ============================================================================ the model
//
// Parameters (FP32 masters, public layout): W1[256][48] | b1[256] | W2[256][256] | b2[256]
// | w3[256] | b3.  The forward pass uses their BF16 roundings; activations are stored as
// BF16 (the next product's operand), accumulation is FP32 throughout:
//   H1 = bf16(relu(X W1^T + b1)), H2 = bf16(relu(H1 W2^T + b2)), y = H2 . w3 + b3.
// Loss: mean squared error.  Backward (B rows):
//   dy = 2 (y - t) / B;  dw3 = H2^T dy;  db3 = sum dy
//   G2 = dy w3^T * [H2 > 0] (FP32; BF16 copy for the products);  db2 = column sums of G2
//   dW2 = bf16(G2)^T H1;  dH1 = bf16(G2) W2;  G1 = dH1 * [H1 > 0];  db1 = column sums
//   dW1 = bf16(G1)^T X;  then Adam on the FP32 masters.
namespace gd {
namespace {

constexpr int F_IN = 48, HID = 256;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + HID * F_IN, OFF_W2 = OFF_B1 + HID, OFF_B2 = OFF_W2 + HID * HID,
              OFF_W3 = OFF_B2 + HID, OFF_B3 = OFF_W3 + HID, NPARAM = OFF_B3 + 1;
constexpr int COLSUM_ROWS = 32;  // rows per block of the column-sum kernels
constexpr int MAX_SPLITS = 64;    // K splits of the weight-gradient GEMMs (K = batch rows)
constexpr int PREDICT_CHUNK = 1 << 18;

__global__ void k_gather(const __nv_bfloat16* X, const float* t, const int32_t* idx, int B, __nv_bfloat16* Xg,
                         float* tg) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * F_IN) return;
  const int r = i / F_IN, c = i % F_IN;
  const int src = idx ? idx[r] : r;
  Xg[i] = X[(size_t)src * F_IN + c];
  if (c == 0) tg[r] = t[src];
}

__global__ void k_loss(const float* y, const float* t, int B, float* dy, float* loss) {
  __shared__ float red[256];
  float acc = 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B; i += gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    dy[i] = 2.f * d / (float)B;
    acc += d * d;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0 && loss) atomicAdd(loss, red[0] / (float)B);
}

// Per block of COLSUM_ROWS rows, one thread per column j (blockDim = HID):
//   mode 0: v = dy[m] * w3[j] * [H[m][j] > 0]  -> Gb[m][j] = bf16(v), partial[blk][j] += v,
//           partial2[blk][j] += dy[m] * H[m][j]   (dw3), partial2[blk][HID] += dy (db3)
//   mode 1: v = D[m][j] * [H[m][j] > 0]        -> Gb[m][j] = bf16(v), partial[blk][j] += v
__global__ void k_grad_rows(int mode, const float* dy, const float* w3, const float* D, const __nv_bfloat16* H,
                            int B, __nv_bfloat16* Gb, float* partial, float* partial2) {
  const int j = threadIdx.x, r0 = blockIdx.x * COLSUM_ROWS;
  float acc = 0.f, acc2 = 0.f, acc3 = 0.f;
  for (int m = r0; m < r0 + COLSUM_ROWS && m < B; ++m) {
    const float h = __bfloat162float(H[(size_t)m * HID + j]);
    const float mask = h > 0.f ? 1.f : 0.f;
    float v;
    if (mode == 0) {
      v = dy[m] * w3[j] * mask;
      acc2 += dy[m] * h;
      acc3 += dy[m];
    } else {
      v = D[(size_t)m * HID + j] * mask;
    }
    Gb[(size_t)m * HID + j] = __float2bfloat16(v);
    acc += v;
  }
  partial[blockIdx.x * (HID + 1) + j] = acc;
  if (mode == 0) {
    partial2[blockIdx.x * (HID + 1) + j] = acc2;
    if (j == 0) partial2[blockIdx.x * (HID + 1) + HID] = acc3;
  }
}

// out[j] = sum over blocks of partial[blk][j] (fixed order), j < n
__global__ void k_sum_partials(const float* partial, int nblk, int n, float* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  float s = 0.f;
  for (int b = 0; b < nblk; ++b) s += partial[b * (HID + 1) + j];
  out[j] = s;
}

__global__ void k_adam(float* P, float* Mo, float* Vo, const float* G, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = G[i];
  const float m = b1 * Mo[i] + (1.f - b1) * g;
  const float v = b2 * Vo[i] + (1.f - b2) * g * g;
  Mo[i] = m;
  Vo[i] = v;
  P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

__global__ void k_refresh(const float* P, __nv_bfloat16* W1b, __nv_bfloat16* W2b, float* w3r) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < HID * F_IN) W1b[i] = __float2bfloat16(P[OFF_W1 + i]);
  if (i < HID * HID) W2b[i] = __float2bfloat16(P[OFF_W2 + i]);
  if (i < HID) w3r[i] = __bfloat162float(__float2bfloat16(P[OFF_W3 + i]));
}

}  // namespace
}  // namespace gd

struct gd_mlp {
  int device = 0, max_batch = 0, step = 0;
  float *P = nullptr, *Mo = nullptr, *Vo = nullptr, *G = nullptr, *w3r = nullptr;
  __nv_bfloat16 *W1b = nullptr, *W2b = nullptr;
  __nv_bfloat16 *Xg = nullptr, *H1 = nullptr, *H2 = nullptr, *G2b = nullptr, *G1b = nullptr;
  float *tg = nullptr, *y = nullptr, *dy = nullptr, *dH1 = nullptr, *partial = nullptr, *partial2 = nullptr,
        *loss = nullptr;
  int* err = nullptr;
  __nv_bfloat16* H1p = nullptr;  // prediction chunk activations
  int hold = 0;                  // test: the next tensor-core launch withholds its first commit
  float* ws = nullptr;           // split-K partial sums (MAX_SPLITS x 256 x 256)
};

namespace {

using gd::HID;
using gd::F_IN;

// The weight gradients' GEMMs sum over the batch (K = B rows): split K into ranges of a
// multiple of 64 rows, at most MAX_SPLITS of them, one CTA each (so that a 4,096-row batch
// takes 64 x 2 CTAs instead of 2), and add the partial sums in order.
gd_status gemm_split_k(gd_mlp* m, gd::GemmArgs g, cudaStream_t s) {
  const int per = (g.K + gd::MAX_SPLITS - 1) / gd::MAX_SPLITS;
  g.kslice = (per + 63) / 64 * 64;
  g.ksplit = (g.K + g.kslice - 1) / g.kslice;
  float* C = g.C;
  const int ldc = g.ldc;
  g.C = nullptr;
  g.partial = m->ws;
  if (gd::gemm_launch(g, s) != cudaSuccess) return GD_ECUDA;
  return gd::reduce_splits(m->ws, g.ksplit, g.M, g.N, C, ldc, s) == cudaSuccess ? GD_OK : GD_ECUDA;
}

// The test hold, for the one launch that takes it.
int take_hold(gd_mlp* m) {
  const int h = m->hold;
  m->hold = 0;
  return h;
}

gd_status mlp_forward(gd_mlp* m, const __nv_bfloat16* X, int M, __nv_bfloat16* H1, __nv_bfloat16* H2, float* y,
                      cudaStream_t s) {
  gd::GemmArgs g{};
  g.A = X;
  g.B = m->W1b;
  g.lda = F_IN;
  g.ldb = F_IN;
  g.ldc = HID;
  g.M = M;
  g.N = HID;
  g.K = F_IN;
  g.bias = m->P + gd::OFF_B1;
  g.relu = true;
  g.Cb = H1;
  g.err = m->err;
  g.hold = take_hold(m);
  if (gd::gemm_launch(g, s) != cudaSuccess) return GD_ECUDA;
  g = gd::GemmArgs{};
  g.A = H1;
  g.B = m->W2b;
  g.lda = HID;
  g.ldb = HID;
  g.ldc = HID;
  g.M = M;
  g.N = HID;
  g.K = HID;
  g.bias = m->P + gd::OFF_B2;
  g.relu = true;
  g.Cb = H2;
  g.dotw = m->w3r;
  g.dot_bias_dev = m->P + gd::OFF_B3;
  g.dot_out = y;
  g.err = m->err;
  g.hold = take_hold(m);
  return gd::gemm_launch(g, s) == cudaSuccess ? GD_OK : GD_ECUDA;
}

// Forward + backward of the batch MSE into m->G (and the loss into m->loss).
gd_status mlp_backward(gd_mlp* m, const void* X, const float* t, const int32_t* idx, int B, cudaStream_t s) {
  if (B < 16 || B % 16 || B > m->max_batch) return GD_EINVAL;
  gd::k_gather<<<(B * F_IN + 255) / 256, 256, 0, s>>>((const __nv_bfloat16*)X, t, idx, B, m->Xg, m->tg);
  gd_status st = mlp_forward(m, m->Xg, B, m->H1, m->H2, m->y, s);
  if (st) return st;
  cudaMemsetAsync(m->loss, 0, sizeof(float), s);
  gd::k_loss<<<32, 256, 0, s>>>(m->y, m->tg, B, m->dy, m->loss);
  const int nblk = (B + gd::COLSUM_ROWS - 1) / gd::COLSUM_ROWS;
  gd::k_grad_rows<<<nblk, HID, 0, s>>>(0, m->dy, m->w3r, nullptr, m->H2, B, m->G2b, m->partial, m->partial2);
  gd::k_sum_partials<<<1, HID, 0, s>>>(m->partial, nblk, HID, m->G + gd::OFF_B2);
  gd::k_sum_partials<<<2, HID, 0, s>>>(m->partial2, nblk, HID + 1, m->G + gd::OFF_W3);  // dw3 | db3
  // dW2 = G2^T H1
  gd::GemmArgs g{};
  g.A = m->G2b;
  g.transA = true;
  g.lda = HID;
  g.B = m->H1;
  g.transB = true;
  g.ldb = HID;
  g.M = HID;
  g.N = HID;
  g.K = B;
  g.C = m->G + gd::OFF_W2;
  g.ldc = HID;
  g.err = m->err;
  g.hold = take_hold(m);
  if (gemm_split_k(m, g, s) != GD_OK) return GD_ECUDA;
  // dH1 = G2 W2
  g = gd::GemmArgs{};
  g.A = m->G2b;
  g.lda = HID;
  g.B = m->W2b;
  g.transB = true;
  g.ldb = HID;
  g.M = B;
  g.N = HID;
  g.K = HID;
  g.C = m->dH1;
  g.ldc = HID;
  g.err = m->err;
  g.hold = take_hold(m);
  if (gd::gemm_launch(g, s) != cudaSuccess) return GD_ECUDA;
  gd::k_grad_rows<<<nblk, HID, 0, s>>>(1, nullptr, nullptr, m->dH1, m->H1, B, m->G1b, m->partial, nullptr);
  gd::k_sum_partials<<<1, HID, 0, s>>>(m->partial, nblk, HID, m->G + gd::OFF_B1);
  // dW1 = G1^T X
  g = gd::GemmArgs{};
  g.A = m->G1b;
  g.transA = true;
  g.lda = HID;
  g.B = m->Xg;
  g.transB = true;
  g.ldb = F_IN;
  g.M = HID;
  g.N = F_IN;
  g.K = B;
  g.C = m->G + gd::OFF_W1;
  g.ldc = F_IN;
  g.err = m->err;
  g.hold = take_hold(m);
  if (gemm_split_k(m, g, s) != GD_OK) return GD_ECUDA;
  return cudaGetLastError() == cudaSuccess ? GD_OK : GD_ECUDA;
}

void mlp_refresh(gd_mlp* m, cudaStream_t s) {
  gd::k_refresh<<<(HID * HID + 255) / 256, 256, 0, s>>>(m->P, m->W1b, m->W2b, m->w3r);
}

}  // namespace

extern "C" {

int gd_mlp_param_count(void) { return gd::NPARAM; }

gd_status gd_mlp_create(int device, uint64_t seed, int max_batch, gd_mlp** out) {
  if (!out || max_batch < 16 || max_batch % 16) return GD_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return GD_ECUDA;
  gd_mlp* m = new gd_mlp();
  m->device = device;
  m->max_batch = max_batch;
  const size_t B = (size_t)max_batch, nblk = (B + gd::COLSUM_ROWS - 1) / gd::COLSUM_ROWS;
  bool ok = cudaMalloc(&m->P, 4 * gd::NPARAM) == cudaSuccess && cudaMalloc(&m->Mo, 4 * gd::NPARAM) == cudaSuccess &&
            cudaMalloc(&m->Vo, 4 * gd::NPARAM) == cudaSuccess && cudaMalloc(&m->G, 4 * gd::NPARAM) == cudaSuccess &&
            cudaMalloc(&m->w3r, 4 * HID) == cudaSuccess && cudaMalloc(&m->W1b, 2 * HID * F_IN) == cudaSuccess &&
            cudaMalloc(&m->W2b, 2 * HID * HID) == cudaSuccess && cudaMalloc(&m->Xg, 2 * B * F_IN) == cudaSuccess &&
            cudaMalloc(&m->H1, 2 * B * HID) == cudaSuccess && cudaMalloc(&m->H2, 2 * B * HID) == cudaSuccess &&
            cudaMalloc(&m->G2b, 2 * B * HID) == cudaSuccess && cudaMalloc(&m->G1b, 2 * B * HID) == cudaSuccess &&
            cudaMalloc(&m->tg, 4 * B) == cudaSuccess && cudaMalloc(&m->y, 4 * B) == cudaSuccess &&
            cudaMalloc(&m->dy, 4 * B) == cudaSuccess && cudaMalloc(&m->dH1, 4 * B * HID) == cudaSuccess &&
            cudaMalloc(&m->partial, 4 * nblk * (HID + 1)) == cudaSuccess &&
            cudaMalloc(&m->partial2, 4 * nblk * (HID + 1)) == cudaSuccess &&
            cudaMalloc(&m->loss, 4) == cudaSuccess && cudaMalloc(&m->err, 4) == cudaSuccess &&
            cudaMalloc(&m->H1p, 2 * (size_t)gd::PREDICT_CHUNK * HID) == cudaSuccess &&
            cudaMalloc(&m->ws, 4 * (size_t)gd::MAX_SPLITS * HID * HID) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    gd_mlp_destroy(m);
    return GD_ENOMEM;
  }
  // He-uniform initialisation from a SplitMix64 stream; biases 0, output bias 0.5
  std::vector<float> h(gd::NPARAM, 0.f);
  uint64_t st = seed;
  auto u01 = [&]() {
    st += 0x9E3779B97F4A7C15ull;
    uint64_t z = st;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
  };
  const double a1 = std::sqrt(6.0 / F_IN), a2 = std::sqrt(6.0 / HID), a3 = std::sqrt(3.0 / HID);
  for (int i = 0; i < HID * F_IN; ++i) h[gd::OFF_W1 + i] = (float)((2 * u01() - 1) * a1);
  for (int i = 0; i < HID * HID; ++i) h[gd::OFF_W2 + i] = (float)((2 * u01() - 1) * a2);
  for (int i = 0; i < HID; ++i) h[gd::OFF_W3 + i] = (float)((2 * u01() - 1) * a3);
  h[gd::OFF_B3] = 0.5f;
  return gd_mlp_set_params(m, h.data()) ? GD_ECUDA : ((*out = m), GD_OK);
}

gd_status gd_mlp_destroy(gd_mlp* m) {
  if (!m) return GD_OK;
  cudaSetDevice(m->device);
  cudaDeviceSynchronize();
  for (void* p : {(void*)m->P, (void*)m->Mo, (void*)m->Vo, (void*)m->G, (void*)m->w3r, (void*)m->W1b,
                  (void*)m->W2b, (void*)m->Xg, (void*)m->H1, (void*)m->H2, (void*)m->G2b, (void*)m->G1b,
                  (void*)m->tg, (void*)m->y, (void*)m->dy, (void*)m->dH1, (void*)m->partial, (void*)m->partial2,
                  (void*)m->loss, (void*)m->err, (void*)m->H1p, (void*)m->ws})
    if (p) cudaFree(p);
  delete m;
  return GD_OK;
}

gd_status gd_mlp_set_params(gd_mlp* m, const float* host) {
  if (!m || !host) return GD_EINVAL;
  cudaSetDevice(m->device);
  if (cudaMemcpy(m->P, host, 4 * gd::NPARAM, cudaMemcpyHostToDevice) != cudaSuccess) return GD_ECUDA;
  cudaMemset(m->Mo, 0, 4 * gd::NPARAM);
  cudaMemset(m->Vo, 0, 4 * gd::NPARAM);
  cudaMemset(m->err, 0, 4);
  m->step = 0;
  mlp_refresh(m, 0);
  return cudaDeviceSynchronize() == cudaSuccess ? GD_OK : GD_ECUDA;
}

gd_status gd_mlp_get_params(gd_mlp* m, float* host) {
  if (!m || !host) return GD_EINVAL;
  cudaSetDevice(m->device);
  return cudaMemcpy(host, m->P, 4 * gd::NPARAM, cudaMemcpyDeviceToHost) == cudaSuccess ? GD_OK : GD_ECUDA;
}

gd_status gd_mlp_predict(gd_mlp* m, const void* X, long long M, float* y, void* stream) {
  if (!m || !X || !y || M < 0 || M > 0x7FFFFFFFll) return GD_EINVAL;
  cudaSetDevice(m->device);
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device);
  const int hold = M > 0 ? take_hold(m) : 0;
  return gd::infer_launch((const __nv_bfloat16*)X, (int)M, m->W1b, m->W2b, m->P + gd::OFF_B1, m->P + gd::OFF_B2,
                          m->w3r, m->P + gd::OFF_B3, y, m->err, hold, sms, (cudaStream_t)stream) == cudaSuccess
             ? GD_OK
             : GD_ECUDA;
}

gd_status gd_mlp_gradients(gd_mlp* m, const void* X, const float* t, const int32_t* idx, int B, float* grad,
                           float* loss, void* stream) {
  if (!m || !X || !t) return GD_EINVAL;
  cudaSetDevice(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  gd_status st = mlp_backward(m, X, t, idx, B, s);
  if (st) return st;
  if (grad && cudaMemcpyAsync(grad, m->G, 4 * gd::NPARAM, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return GD_ECUDA;
  if (loss && cudaMemcpyAsync(loss, m->loss, 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return GD_ECUDA;
  return GD_OK;
}

gd_status gd_mlp_train_step(gd_mlp* m, const void* X, const float* t, const int32_t* idx, int B, float lr,
                            float* loss, void* stream) {
  if (!m || !X || !t) return GD_EINVAL;
  cudaSetDevice(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  gd_status st = mlp_backward(m, X, t, idx, B, s);
  if (st) return st;
  m->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)m->step), c2 = 1.f - std::pow(b2, (float)m->step);
  gd::k_adam<<<(gd::NPARAM + 255) / 256, 256, 0, s>>>(m->P, m->Mo, m->Vo, m->G, gd::NPARAM, lr, b1, b2, 1e-8f, c1, c2);
  mlp_refresh(m, s);
  if (loss && cudaMemcpyAsync(loss, m->loss, 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return GD_ECUDA;
  return cudaGetLastError() == cudaSuccess ? GD_OK : GD_ECUDA;
}

gd_status gd_mlp_error(gd_mlp* m, int* host_err) {
  if (!m || !host_err) return GD_EINVAL;
  cudaSetDevice(m->device);
  return cudaMemcpy(host_err, m->err, 4, cudaMemcpyDeviceToHost) == cudaSuccess ? GD_OK : GD_ECUDA;
}

gd_status gd_mlp_test_hold(gd_mlp* m, int on) {
  if (!m) return GD_EINVAL;
  cudaSetDevice(m->device);
  m->hold = on ? 1 : 0;
  if (on) return GD_OK;
  if (cudaMemset(m->err, 0, 4) != cudaSuccess) return GD_ECUDA;
  return cudaDeviceSynchronize() == cudaSuccess ? GD_OK : GD_ECUDA;
}

}  // extern "C"
