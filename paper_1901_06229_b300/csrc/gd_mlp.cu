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

#include <cstdint>

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

// Bounded wait for phase `parity`; false after ~2 s at the maximum clock.
__device__ __forceinline__ bool mbar_wait(uint64_t* m, uint32_t parity) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(m)), "r"(parity)
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
// Rows or K beyond the matrix are zero-filled.
__device__ void stage(uint8_t* dst, const __nv_bfloat16* src, int ld, int nrows_total, int ktotal, int r0, int rows,
                      int k0, int kc, bool trans) {
  const int chunks = kc / 8;
  for (int idx = threadIdx.x; idx < rows * chunks; idx += blockDim.x) {
    const int r = idx / chunks, c = idx % chunks;
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
  for (int k0 = 0; k0 < g.K && ok; k0 += KC) {
    const int kc = g.K - k0 < KC ? g.K - k0 : KC;  // multiple of 16 by contract
    stage(sa, g.A, g.lda, g.M, g.K, m0, 128, k0, kc, g.transA);
    stage(sb, g.B, g.ldb, g.N, g.K, n0, nt, k0, kc, g.transB);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      tc_fence_after();
      const uint32_t sbo = (uint32_t)(kc / 8) * 128;
      for (int kk = 0; kk < kc / 16; ++kk) {
        const uint64_t da = make_desc(smem_addr(sa) + kk * 256, 128, sbo);
        const uint64_t db = make_desc(smem_addr(sb) + kk * 256, 128, sbo);
        mma_bf16(tmem, da, db, idesc, k0 > 0 || kk > 0);
      }
      mma_commit(mbar);
    }
    ok = mbar_wait(mbar, phase);
    phase ^= 1;
    tc_fence_after();
  }
  if (!ok) {
    if (threadIdx.x == 0 && g.err) atomicExch(g.err, 1);
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
    if (g.dotw && row < g.M) g.dot_out[row] = dot + g.dot_bias;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
}

}  // namespace

// Operand staging (48 KB) plus 32 KB of headroom: at most two CTAs share an SM, so the
// two 256-column TMEM allocations always fit the SM's 512 columns.
size_t gemm_smem_bytes() { return 128 * KC * 2 + 256 * KC * 2 + 16 + 32 * 1024; }

cudaError_t gemm_launch(const GemmArgs& g, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)gemm_smem_bytes());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid((g.M + 127) / 128, (g.N + 255) / 256);
  gemm_kernel<<<grid, 128, gemm_smem_bytes(), st>>>(g);
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
