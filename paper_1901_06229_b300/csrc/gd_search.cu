// Fused GeoDock pose-search kernel for sm_103a.
//
// One warp owns one pose (ligand, restart orientation) from placement to its final
// score; the CTA is persistent and its warps pull poses from a global counter, a few
// restarts of one ligand at a time.
//   a1  the pocket grid is staged once per CTA into shared memory with bulk async
//       copies completing on an mbarrier (when the cropped grid fits, 128-register
//       builds), else read through a 3D texture (point sampling, border 0) or L1/L2;
//   a2  the ligand (preorder-packed float4) and its rotamer descriptors and excluded
//       pairs are read into per-warp shared buffers;
//   a3  generate_starting_pose: ZYZ Euler restart about the centroid, moved to the
//       pocket centre (Listing 1 / Sec. 3.1); a small kernel writes every restart's
//       rotation and the centred ligands once per launch, and pose coordinates are
//       kept in grid units (a point's cell is the floor of its coordinates);
//   a4  rigid score: sum of grid cells under the atoms (scoring function, Sec. 3.2),
//       each atom's cell cached beside its coordinates;
//   a5-a8 optimize_pose (Sec. 3.1, Sec. 4.1): for each rotamer in order, every lane
//       evaluates its own angles k = lane + 32 j.  An exact reach filter keeps only
//       the moving x static pairs (not excluded by bond separation) whose closest
//       approach over the whole turn is below bump_dist + 0.01 A; each kept pair's
//       squared distance at angle theta is |x_a - x_b|^2 + (cos - 1) P + sin Q, two
//       FMAs per angle (BumpCheck, Sec. 3.2; the unfiltered sweep tests every pair).
//       The moving fragment is turned about the current bond axis (Rodrigues split
//       into the axis frame) and its cells gathered; a warp max-reduction over a
//       packed (score, -k) key is the per-fragment reduction, and the winning
//       rotation is committed;
//   a9  the rotamer loop repeats `reps` times (num_repetitions, Listing 1);
//   a10 the last warp to finish a ligand reduces over its restarts (ties: smallest
//       o), replays the winning pose to recover its coordinates and writes results.
// All geometry uses explicitly rounded FP32 intrinsics, so the search and the replay
// produce bitwise-identical coordinates, and neither the launch tile nor the filter
// path (near list, masks, none) can change a result.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>

#include "gd_internal.h"

namespace gd {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr float PARK = 1.0e18f;  // far-away position for excluded static atoms

struct Rot3 {
  float m[9];
  float p[3];  // rotation centre: x' = p + M (x - p)
};

// Rodrigues: M = c I + s [u]x + (1 - c) u u^T for the unit axis u.
__device__ __forceinline__ Rot3 rodrigues(float ux, float uy, float uz, float c, float s, float4 p) {
  Rot3 R;
  const float omc = __fsub_rn(1.0f, c);
  const float ox = __fmul_rn(omc, ux), oy = __fmul_rn(omc, uy), oz = __fmul_rn(omc, uz);
  const float sx = __fmul_rn(s, ux), sy = __fmul_rn(s, uy), sz = __fmul_rn(s, uz);
  R.m[0] = __fmaf_rn(ox, ux, c);
  R.m[1] = __fsub_rn(__fmul_rn(ox, uy), sz);
  R.m[2] = __fadd_rn(__fmul_rn(ox, uz), sy);
  R.m[3] = __fadd_rn(__fmul_rn(oy, ux), sz);
  R.m[4] = __fmaf_rn(oy, uy, c);
  R.m[5] = __fsub_rn(__fmul_rn(oy, uz), sx);
  R.m[6] = __fsub_rn(__fmul_rn(oz, ux), sy);
  R.m[7] = __fadd_rn(__fmul_rn(oz, uy), sx);
  R.m[8] = __fmaf_rn(oz, uz, c);
  R.p[0] = p.x;
  R.p[1] = p.y;
  R.p[2] = p.z;
  return R;
}

__device__ __forceinline__ void rot_apply(const Rot3& R, float x, float y, float z, float& ox,
                                          float& oy, float& oz) {
  const float dx = __fsub_rn(x, R.p[0]), dy = __fsub_rn(y, R.p[1]), dz = __fsub_rn(z, R.p[2]);
  ox = __fadd_rn(R.p[0], __fmaf_rn(R.m[0], dx, __fmaf_rn(R.m[1], dy, __fmul_rn(R.m[2], dz))));
  oy = __fadd_rn(R.p[1], __fmaf_rn(R.m[3], dx, __fmaf_rn(R.m[4], dy, __fmul_rn(R.m[5], dz))));
  oz = __fadd_rn(R.p[2], __fmaf_rn(R.m[6], dx, __fmaf_rn(R.m[7], dy, __fmul_rn(R.m[8], dz))));
}

// Angle theta_k = 2 pi k / A as (cos theta - 1, sin theta), computed once per block into
// a table; cos - 1 = -2 sin^2(theta / 2) keeps its relative precision at small angles.
__device__ __forceinline__ float2 angle_entry(int k, int A) {
  float sh, ch, s, c;
  sincospif(__fdiv_rn((float)k, (float)A), &sh, &ch);
  sincospif(__fdiv_rn(2.0f * (float)k, (float)A), &s, &c);
  return make_float2(__fmul_rn(-2.0f, __fmul_rn(sh, sh)), s);
}

// Rotation about the axis through p along the unit vector u (Rodrigues' formula split
// about the axis): with d = x - p, h = d.u, d_perp = d - h u and w = u x d, the point
// turned by theta is x + (cos theta - 1) d_perp + sin theta w.  axis_frame gives
// (d_perp, w.x) in dp and (w.y, w.z) in w2, once per atom and rotamer step; turn is then
// six FMAs per angle.  frame_w2 is (w.y, w.z) alone, with the same roundings, for the
// compact builds that keep dp but not w2.  The search and the commit of a step share
// these functions.
__device__ __forceinline__ float2 frame_w2(float4 x, float4 p, float ux, float uy, float uz) {
  const float dx = __fsub_rn(x.x, p.x), dy = __fsub_rn(x.y, p.y), dz = __fsub_rn(x.z, p.z);
  return make_float2(__fmaf_rn(uz, dx, -__fmul_rn(ux, dz)), __fmaf_rn(ux, dy, -__fmul_rn(uy, dx)));
}

__device__ __forceinline__ void axis_frame(float x, float y, float z, float4 p, float ux, float uy, float uz,
                                           float4& dp, float2& w2, float& h) {
  const float dx = __fsub_rn(x, p.x), dy = __fsub_rn(y, p.y), dz = __fsub_rn(z, p.z);
  h = __fmaf_rn(dx, ux, __fmaf_rn(dy, uy, __fmul_rn(dz, uz)));
  dp.x = __fmaf_rn(-h, ux, dx);
  dp.y = __fmaf_rn(-h, uy, dy);
  dp.z = __fmaf_rn(-h, uz, dz);
  dp.w = __fmaf_rn(uy, dz, -__fmul_rn(uz, dy));
  w2.x = __fmaf_rn(uz, dx, -__fmul_rn(ux, dz));
  w2.y = __fmaf_rn(ux, dy, -__fmul_rn(uy, dx));
}

__device__ __forceinline__ void turn(float4 x, float4 dp, float2 w2, float2 cs, float& ox, float& oy, float& oz) {
  ox = __fmaf_rn(cs.y, dp.w, __fmaf_rn(cs.x, dp.x, x.x));
  oy = __fmaf_rn(cs.y, w2.x, __fmaf_rn(cs.x, dp.y, x.y));
  oz = __fmaf_rn(cs.y, w2.y, __fmaf_rn(cs.x, dp.z, x.z));
}

// Bump test of a moving atom a against a static atom b.  Both decomposed about the
// axis, the squared distance with a turned by theta is
//   |x_a - x_b|^2 + (cos theta - 1) P + sin theta Q,
//   P = -2 d_perp,a . d_perp,b,  Q = -2 (u x d_a) . d_perp,b,
// so pair_coef (once per pair and step) leaves two FMAs per angle (pair_d2).  Every
// bump test of the search goes through these two functions.
__device__ __forceinline__ float4 pair_coef(float4 xa, float4 dpa, float2 w2a, float4 xb, float4 p, float ux,
                                            float uy, float uz) {
  float4 dpb;
  float2 w2b;
  float hb;
  axis_frame(xb.x, xb.y, xb.z, p, ux, uy, uz, dpb, w2b, hb);
  const float dx = __fsub_rn(xa.x, xb.x), dy = __fsub_rn(xa.y, xb.y), dz = __fsub_rn(xa.z, xb.z);
  const float c0 = __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz)));
  const float P = __fmul_rn(-2.0f, __fmaf_rn(dpa.x, dpb.x, __fmaf_rn(dpa.y, dpb.y, __fmul_rn(dpa.z, dpb.z))));
  const float Q = __fmul_rn(-2.0f, __fmaf_rn(dpa.w, dpb.x, __fmaf_rn(w2a.x, dpb.y, __fmul_rn(w2a.y, dpb.z))));
  return make_float4(c0, P, Q, 0.f);
}

__device__ __forceinline__ float pair_d2(float c0, float P, float Q, float2 cs) {
  return __fmaf_rn(cs.x, P, __fmaf_rn(cs.y, Q, c0));
}

// Grid access modes of the search: the cropped grid read through L1 (GRID_LDG), staged
// in shared memory (GRID_SMEM), or fetched by the texture unit (GRID_TEX: point
// sampling of unnormalised coordinates selects texel floor(f) exactly, and the border
// mode returns 0 outside the crop, so the fetch is the same lookup in one instruction).
constexpr int GRID_LDG = 0, GRID_SMEM = 1, GRID_TEX = 2;

// Grid cell under a point in grid units (cell = floor per axis); 0 outside the crop.
template <int G>
__device__ __forceinline__ int cell(const PocketDev& pk, const uint8_t* sg, float fx, float fy, float fz) {
  if (G == GRID_TEX) return (int)tex3D<unsigned char>((cudaTextureObject_t)pk.tex, fx, fy, fz);
  const int ix = __float2int_rd(fx), iy = __float2int_rd(fy), iz = __float2int_rd(fz);
  if ((unsigned)ix >= (unsigned)pk.cx || (unsigned)iy >= (unsigned)pk.cy || (unsigned)iz >= (unsigned)pk.cz)
    return 0;
  const int idx = (iz * pk.cy + iy) * pk.cx + ix;
  if (G == GRID_SMEM) return sg[idx];
  return __ldg(pk.grid + idx);
}

__device__ __forceinline__ float warp_sum_f(float v) {
  // xor butterfly: every lane adds the same two partial sums in either order, so all
  // lanes end with the same bits
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = __fadd_rn(v, __shfl_xor_sync(FULL, v, off));
  return v;
}

// a3: x <- R_o (x0 - c_lig), coordinates relative to the pocket centre, kept in grid
// units (x inv_h + shift).  The centred coordinates x0 - c_lig and the restart
// rotations R_o come from pose_setup_kernel.
template <bool SRV>
__device__ void place(const SearchArgs& a, float4* X, int a0, int n, int o, int lane) {
  const float* r = a.rmat + 9 * (size_t)o;
  const float r00 = __ldg(r + 0), r01 = __ldg(r + 1), r02 = __ldg(r + 2);
  const float r10 = __ldg(r + 3), r11 = __ldg(r + 4), r12 = __ldg(r + 5);
  const float r20 = __ldg(r + 6), r21 = __ldg(r + 7), r22 = __ldg(r + 8);
#pragma unroll 2
  for (int i = lane; i < n; i += 32) {
    // the server's slots are rewritten while it runs: read them coherently (L2), not
    // through the read-only path
    const float4 d = SRV ? __ldcg(a.xc + a0 + i) : __ldg(a.xc + a0 + i);
    const float x = __fmaf_rn(r00, d.x, __fmaf_rn(r01, d.y, __fmul_rn(r02, d.z)));
    const float y = __fmaf_rn(r10, d.x, __fmaf_rn(r11, d.y, __fmul_rn(r12, d.z)));
    const float z = __fmaf_rn(r20, d.x, __fmaf_rn(r21, d.y, __fmul_rn(r22, d.z)));
    X[i] = make_float4(__fmaf_rn(x, a.pk.inv_h, a.pk.shift[0]), __fmaf_rn(y, a.pk.inv_h, a.pk.shift[1]),
                       __fmaf_rn(z, a.pk.inv_h, a.pk.shift[2]), 0.f);
  }
  __syncwarp();
}

// Per launch, before the search: R_o of every restart (ZYZ Euler angles, Listing 1:
// R = Rz(alpha) Ry(beta) Rz(gamma)) and every ligand's coordinates minus its centroid;
// the work counter and the per-ligand completion counters of the search that follows on
// the same stream are cleared here too.
__global__ void __launch_bounds__(256) pose_setup_kernel(const __grid_constant__ SearchArgs a) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  if (tid == 0) *a.work = 0ull;
  for (int i = tid; i < a.L; i += nth) a.done[i] = 0;
  for (int o = tid; o < a.O; o += nth) {
    const int ia = o / (a.nb * a.ng), jb = (o / a.ng) % a.nb, kg = o % a.ng;
    float sa, ca, sb, cb, sg, cg;
    sincospif(__fdiv_rn(2.0f * (float)ia, (float)a.na), &sa, &ca);
    sincospif(__fdiv_rn(__fadd_rn((float)jb, 0.5f), (float)a.nb), &sb, &cb);
    sincospif(__fdiv_rn(2.0f * (float)kg, (float)a.ng), &sg, &cg);
    const float cacb = __fmul_rn(ca, cb), sacb = __fmul_rn(sa, cb);
    float* r = a.rmat + 9 * (size_t)o;
    r[0] = __fsub_rn(__fmul_rn(cacb, cg), __fmul_rn(sa, sg));
    r[1] = __fsub_rn(__fmul_rn(-cacb, sg), __fmul_rn(sa, cg));
    r[2] = __fmul_rn(ca, sb);
    r[3] = __fadd_rn(__fmul_rn(sacb, cg), __fmul_rn(ca, sg));
    r[4] = __fadd_rn(__fmul_rn(-sacb, sg), __fmul_rn(ca, cg));
    r[5] = __fmul_rn(sa, sb);
    r[6] = __fmul_rn(-sb, cg);
    r[7] = __fmul_rn(sb, sg);
    r[8] = cb;
    // half-angle quaternion of Rz(alpha) Ry(beta) Rz(gamma):
    // (cos(b/2) cos((a+g)/2), sin(b/2) sin((g-a)/2), sin(b/2) cos((g-a)/2), cos(b/2) sin((a+g)/2))
    float hb_s, hb_c, hp_s, hp_c, hm_s, hm_c;
    sincospif(__fdiv_rn((float)jb + 0.5f, 2.0f * (float)a.nb), &hb_s, &hb_c);
    const float apg = (float)ia / (float)a.na + (float)kg / (float)a.ng;  // (alpha + gamma) / 2 in units of pi
    const float gma = (float)kg / (float)a.ng - (float)ia / (float)a.na;  // (gamma - alpha) / 2
    sincospif(apg, &hp_s, &hp_c);
    sincospif(gma, &hm_s, &hm_c);
    float4 q = make_float4(hb_c * hp_c, hb_s * hm_s, hb_s * hm_c, hb_c * hp_s);
    if (q.x < 0.f) q = make_float4(-q.x, -q.y, -q.z, -q.w);
    a.quat[o] = q;
  }
  const int lane = threadIdx.x & 31;
  for (int li = tid >> 5; li < a.L; li += nth >> 5) {
    const int a0 = a.atom_off[li], n = a.atom_off[li + 1] - a0;
    const float4* x0 = a.xyz + a0;
    float sx = 0.f, sy = 0.f, sz = 0.f;
    for (int i = lane; i < n; i += 32) {
      const float4 v = x0[i];
      sx = __fadd_rn(sx, v.x);
      sy = __fadd_rn(sy, v.y);
      sz = __fadd_rn(sz, v.z);
    }
    sx = warp_sum_f(sx);
    sy = warp_sum_f(sy);
    sz = warp_sum_f(sz);
    const float cx = __fdiv_rn(sx, (float)n), cy = __fdiv_rn(sy, (float)n), cz = __fdiv_rn(sz, (float)n);
    for (int i = lane; i < n; i += 32) {
      const float4 v = x0[i];
      a.xc[a0 + i] = make_float4(__fsub_rn(v.x, cx), __fsub_rn(v.y, cy), __fsub_rn(v.z, cz), 0.f);
    }
  }
}

// Ligand li's first atom a0 / atom count n and first rotamer r0 / rotamer count R: from the
// CSR offsets of a batch, or (SRV, the streaming server) from its slot.
template <bool SRV>
__device__ __forceinline__ void lig_span(const SearchArgs& a, int li, int& a0, int& n, int& r0, int& R) {
  if (SRV) {
    a0 = li * a.slot_amax;
    n = __ldcg(a.slot_n + li);
    r0 = li * a.slot_rmax;
    R = __ldcg(a.slot_r + li);
  } else {
    a0 = a.atom_off[li];
    n = a.atom_off[li + 1] - a0;
    r0 = a.rot_off[li];
    R = a.rot_off[li + 1] - r0;
  }
}

// Unit bond axis from the static end p to the moving end q (current coordinates).
__device__ __forceinline__ void bond_axis(const float4* X, const RotDesc& rd, float& ux, float& uy, float& uz) {
  const float4 xp = X[rd.p], xq = X[rd.q];
  const float dx = __fsub_rn(xq.x, xp.x), dy = __fsub_rn(xq.y, xp.y), dz = __fsub_rn(xq.z, xp.z);
  // hardware reciprocal square root: deterministic, so the search and its replay agree,
  // and within 1e-7 relative of the rounded one
  const float inv = rsqrtf(__fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz))));
  ux = __fmul_rn(dx, inv);
  uy = __fmul_rn(dy, inv);
  uz = __fmul_rn(dz, inv);
}

// i-th atom of the rotating fragment (preorder id), i in [0, f).
__device__ __forceinline__ int frag_atom(const RotDesc& rd, int i) {
  return rd.comp ? (i < rd.lo ? i : rd.hi + (i - rd.lo)) : rd.lo + i;
}

__device__ __forceinline__ int frag_size(const RotDesc& rd, int n) {
  return rd.comp ? n - (rd.hi - rd.lo) : rd.hi - rd.lo;
}

// Commit the winning rotation to the fragment (same arithmetic as the candidate); the
// w component of each moved atom caches its new grid cell.  DP / W2: the step's axis
// frames in sweep order when the search has them (W2 NULL in the compact builds: rebuilt
// from the atom and p), else (replay) NULL and recomputed.
template <int G>
__device__ void commit(const PocketDev& pk, const uint8_t* sg, float4* X, int n, const RotDesc& rd, float ux,
                       float uy, float uz, float2 cs, int lane, const float4* DP, const float2* W2) {
  const float4 xp = X[rd.p];
  __syncwarp();
  const int f = frag_size(rd, n);
#pragma unroll 2
  for (int i = lane; i < f; i += 32) {
    const int t = frag_atom(rd, i);
    const float4 v = X[t];
    float4 dp;
    float2 w2;
    float h, x, y, z;
    if (DP) {
      dp = DP[i];
      w2 = W2 ? W2[i] : frame_w2(v, xp, ux, uy, uz);
    } else {
      axis_frame(v.x, v.y, v.z, xp, ux, uy, uz, dp, w2, h);
    }
    turn(v, dp, w2, cs, x, y, z);
    X[t] = make_float4(x, y, z, __int_as_float(cell<G>(pk, sg, x, y, z)));
  }
  __syncwarp();
}

// Rigid score of the pose (sum of the grid cells under its atoms); each atom's cell is
// cached in the w component of its coordinates.
template <int G>
__device__ __forceinline__ int score_atoms(const PocketDev& pk, const uint8_t* sg, float4* X, int n, int lane) {
  int s = 0;
  for (int i = lane; i < n; i += 32) {
    const float4 v = X[i];
    const int c = cell<G>(pk, sg, v.x, v.y, v.z);
    X[i].w = __int_as_float(c);
    s += c;
  }
  __syncwarp();
  return __reduce_add_sync(FULL, s);
}

// Smallest squared distance from moving atom a, turned by each of the S angles, to the
// static atoms [b0, b1).
template <int S>
__device__ __forceinline__ void min_d2_range(const float4* X, int b0, int b1, float4 xa, float4 dpa, float2 w2a,
                                             float4 xp, float ux, float uy, float uz, const float2 (&cs)[S],
                                             float (&mind)[S]) {
  for (int b = b0; b < b1; ++b) {
    const float4 k = pair_coef(xa, dpa, w2a, X[b], xp, ux, uy, uz);
#pragma unroll
    for (int j = 0; j < S; ++j) mind[j] = fminf(mind[j], pair_d2(k.x, k.y, k.z, cs[j]));
  }
}

struct WarpMem {
  float4* X;       // current pose, preorder
  float2* HR;      // (height along the bond axis, distance from it) per atom
  float4* DP;      // per moving atom (sweep order): d_perp and (u x d).x of axis_frame
  float2* W2;      // per moving atom: (u x d).y, (u x d).z
  uint16_t* NEAR;  // the step's near pairs (ia << 8 | b), at most 4 nmax (overwrites HR once dead)
  float4* PC;      // pair_coef of the 32 near pairs being swept (lane t writes entry t)
  uint8_t* SL;     // the reach filter's columns: static atom of column k (aliases PC[0, 16))
  uint8_t* POS;    // the reach filter's column of atom b, 0xFF if none (aliases PC[16, 32))
  uint32_t* MASK;  // near-pair masks: word ia * nch + c, bit t <-> static atom 32 c + t
  RotDesc* RDs;    // per-warp copies of the ligand's rotamer descriptors / excluded pairs
  uint16_t* EXLs;  //   (NULL in the compact builds)
  const RotDesc* RD;    // the current ligand's rotamer descriptors: RDs, or global memory
  const uint16_t* EXL;  // its excluded pairs (all rotamers), from the first one's offset on
  const float2* CS;  // (cos, sin) of every angle, shared by the block
};

// Per-warp buffers (see warp_smem_bytes).  compact: no W2 (rebuilt from DP) and no copies
// of the descriptors and excluded pairs (read through L1 instead).
__device__ __forceinline__ WarpMem warp_mem(unsigned char* base, int nmax, int fmax, int mask_words, int rmax,
                                            int emax, bool compact) {
  auto a16 = [](int v) { return (v + 15) / 16 * 16; };
  WarpMem w;
  w.X = reinterpret_cast<float4*>(base);
  base += a16(16 * nmax);
  w.HR = reinterpret_cast<float2*>(base);
  w.NEAR = reinterpret_cast<uint16_t*>(base);
  base += a16(8 * nmax);
  w.DP = reinterpret_cast<float4*>(base);
  base += a16(16 * fmax);
  w.W2 = nullptr;
  if (!compact) {
    w.W2 = reinterpret_cast<float2*>(base);
    base += a16(8 * fmax);
  }
  w.MASK = reinterpret_cast<uint32_t*>(base);
  base += a16(4 * mask_words);
  w.EXLs = nullptr;
  w.RDs = nullptr;
  if (!compact) {
    w.EXLs = reinterpret_cast<uint16_t*>(base);
    base += a16(2 * emax);
    w.RDs = reinterpret_cast<RotDesc*>(base);
    base += 16 * rmax;
  }
  w.RD = w.RDs;
  w.EXL = w.EXLs;
  w.PC = reinterpret_cast<float4*>(base);
  w.SL = reinterpret_cast<uint8_t*>(base);  // GD_MAX_ATOMS = 256: 255 columns at most
  w.POS = reinterpret_cast<uint8_t*>(base) + 256;
  w.CS = nullptr;
  return w;
}

// (u x d).y, (u x d).z of moving atom ia (sweep order) at x (its coordinates this step):
// stored, or rebuilt from x and p in the compact builds (bitwise the same values).
template <bool COMPACT>
__device__ __forceinline__ float2 w2_at(const WarpMem& w, int ia, float4 x, float4 p, float ux, float uy, float uz) {
  if (COMPACT) return frame_w2(x, p, ux, uy, uz);
  return w.W2[ia];
}

// Per rotamer step: (h, rho) of every atom about the bond axis for the reach filter, and
// the axis frame of every moving atom (sweep order) for the candidate rotations.
template <bool COMPACT>
__device__ void prep_step(const WarpMem& w, int n, const RotDesc& rd, float4 xp, float ux, float uy, float uz,
                          int lane) {
  for (int i = lane; i < n; i += 32) {
    const float4 v = w.X[i];
    float4 dp;
    float2 w2;
    float h;
    axis_frame(v.x, v.y, v.z, xp, ux, uy, uz, dp, w2, h);
    // rho from the hardware reciprocal square root (error ~1e-6 A, far inside the
    // filter's 0.01 A margin; rho only feeds the filter)
    const float r2 = fmaxf(__fmaf_rn(dp.x, dp.x, __fmaf_rn(dp.y, dp.y, __fmul_rn(dp.z, dp.z))), 1e-30f);
    w.HR[i] = make_float2(h, __fmul_rn(r2, rsqrtf(r2)));
    const bool in = i >= rd.lo && i < rd.hi;
    if (in != (rd.comp != 0)) {
      const int ia = rd.comp ? (i < rd.lo ? i : i - (rd.hi - rd.lo)) : i - rd.lo;
      w.DP[ia] = dp;
      if (!COMPACT) w.W2[ia] = w2;
    }
  }
  __syncwarp();
}

// Evaluate every angle of one rotamer step; returns the warp-wide best key
// ((score + 1) << 16 | (0xFFFF - k)), 0 if every candidate is bumped.
template <int S, int G, bool COMPACT>
__device__ unsigned eval_step(const SearchArgs& a, const uint8_t* sg, const WarpMem& w, const uint16_t* excl,
                              int n, const RotDesc& rd, float4 xp, float ux, float uy, float uz, int cur,
                              int lane, unsigned long long& pairs, uint8_t* dbg) {
  float4* X = w.X;
  int m0a, m0b, m1a, m1b, s0a, s0b, s1a, s1b;
  if (rd.comp) {
    m0a = 0; m0b = rd.lo; m1a = rd.hi; m1b = n;
    s0a = rd.lo; s0b = rd.hi; s1a = 0; s1b = 0;
  } else {
    m0a = rd.lo; m0b = rd.hi; m1a = 0; m1b = 0;
    s0a = 0; s0b = rd.lo; s1a = rd.hi; s1b = n;
  }
  const unsigned n_static = (unsigned)((s0b - s0a) + (s1b - s1a));
  const int passes = (a.A + 32 * S - 1) / (32 * S);
  unsigned best = 0;
  for (int pass = 0; pass < passes; ++pass) {
    float2 cs[S];
    int kk[S], sc[S];
    bool bump[S];
#pragma unroll
    for (int j = 0; j < S; ++j) {
      kk[j] = lane + 32 * (pass * S + j);
      cs[j] = w.CS[kk[j] < a.A ? kk[j] : 0];
      sc[j] = 0;
      bump[j] = kk[j] >= a.A;  // idle slots count as rejected
    }
    const int n_excl = rd.n_excl;
    int ex = 0;
    int next_a = n_excl ? (int)(excl[0] & 0xFF) : -1;  // moving atom of the next excluded pair
    bool stop = false;
    int stat = cur;  // running score minus the fragment's cached cells
    int ia = 0;
    for (int seg = 0; seg < 2 && !stop; ++seg) {
      const int ma = seg ? m1a : m0a, mb = seg ? m1b : m0b;
      for (int ai = ma; ai < mb; ++ai, ++ia) {
        const float4 xa = X[ai];
        stat -= __float_as_int(xa.w);
        const float4 dp = w.DP[ia];
        const float2 w2 = w2_at<COMPACT>(w, ia, xa, xp, ux, uy, uz);
        // park the static atoms this moving atom must not be tested against
        int ex_end = ex;
        float4 saved = make_float4(0.f, 0.f, 0.f, 0.f);
        int my_b = -1;
        if (ai == next_a) {
          while (ex_end < n_excl && (int)(excl[ex_end] & 0xFF) == ai) ++ex_end;
          next_a = ex_end < n_excl ? (int)(excl[ex_end] & 0xFF) : -1;
          __syncwarp();
          if (lane < ex_end - ex) {
            my_b = (int)(excl[ex + lane] >> 8);
            saved = X[my_b];
            X[my_b] = make_float4(PARK, PARK, PARK, 0.f);
          }
          __syncwarp();
        }
        float xr[S][3], mind[S];
#pragma unroll
        for (int j = 0; j < S; ++j) {
          turn(xa, dp, w2, cs[j], xr[j][0], xr[j][1], xr[j][2]);
          sc[j] += cell<G>(a.pk, sg, xr[j][0], xr[j][1], xr[j][2]);
          mind[j] = 3.0e38f;
        }
        min_d2_range<S>(X, s0a, s0b, xa, dp, w2, xp, ux, uy, uz, cs, mind);
        min_d2_range<S>(X, s1a, s1b, xa, dp, w2, xp, ux, uy, uz, cs, mind);
        bool done = true;
        const unsigned tested = n_static - (unsigned)(ex_end - ex);  // parked pairs are not tests
#pragma unroll
        for (int j = 0; j < S; ++j) {
          if (!bump[j]) pairs += tested;
          bump[j] = bump[j] || (mind[j] < a.thr2);
          done = done && bump[j];
        }
        if (ex_end > ex) {
          __syncwarp();
          if (my_b >= 0) X[my_b] = saved;
          __syncwarp();
          ex = ex_end;
        }
        if (__all_sync(FULL, done)) {
          stop = true;
          break;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < S; ++j)
      if (kk[j] < a.A) {
        const unsigned key = bump[j] ? 0u : (((unsigned)(stat + sc[j] + 1) << 16) | (0xFFFFu - (unsigned)kk[j]));
        best = key > best ? key : best;
        if (dbg) dbg[kk[j]] = bump[j] ? 1 : 0;
      }
  }
  return __reduce_max_sync(FULL, best);
}

// Columns of a step's reach filter: the static atoms it tests, in ascending preorder.
// Column k is static atom k (static order: [s0a, s0a + ns0) then from s1a) unless the
// filter pruned, in which case it is SL[k].
struct Cols {
  int prune, ns0, s0a, s1a;
};

template <bool PRUNE>
__device__ __forceinline__ Cols step_cols(const RotDesc& rd) {
  return rd.comp ? Cols{PRUNE, rd.hi - rd.lo, rd.lo, 0} : Cols{PRUNE, rd.lo, 0, rd.hi};
}

__device__ __forceinline__ int col_atom(const WarpMem& w, const Cols& c, int k) {
  return c.prune ? (int)w.SL[k] : (k < c.ns0 ? c.s0a + k : c.s1a + (k - c.ns0));
}

// Reach filter of one rotamer step.  A moving atom a sweeps a circle about the bond
// axis: height h_a along it, radius rho_a.  For a static atom b the distance over the
// whole turn is at least sqrt((h_a - h_b)^2 + (rho_a - rho_b)^2), so only pairs below
// bump_dist + margin (and not excluded by graph distance) need per-angle tests.
// With PRUNE (the 128-register kernels: on the 80-register ones the extra code costs
// more than it saves), the static atoms farther than that from the box
// [min h_a, max h_a] x [min rho_a, max rho_a] of the moving atoms are dropped first:
// the box distance is computed with the same roundings as the pair distance, and every
// rounding step is monotone, so no dropped atom could pass the pair test with any
// moving atom.  The remaining static atoms, in ascending preorder, are the filter's
// columns (SL[k] is column k's atom, POS[b] atom b's column, 0xFF if dropped); without
// pruning every static atom is a column.  Moving atoms are numbered ia in sweep order;
// lane t of chunk c tests column 32 c + t against every moving atom and the warp's
// ballot is the mask word MASK[ia * nch + c], nch = *n_chunks.  The rotamer's excluded
// pairs are then cleared from the masks, and the masks are compacted into the step's
// list of near pairs (NEAR, at most 4 nmax entries: the bytes of HR).  Returns the
// number of near pairs; above 4 nmax only the masks are usable.  HOIST (the compact
// builds, which read the excluded pairs through L1): ex0 is excluded pair `lane`, read by
// the caller at the start of the step so that the load is in flight during the axis
// frames and the ballots.
template <bool PRUNE, bool HOIST>
__device__ int build_near(const SearchArgs& a, const WarpMem& w, const uint16_t* excl, uint32_t ex0, int n,
                          const RotDesc& rd, int lane, unsigned long long& reach, int& nch_out) {
  int m0a, m0b, m1a, m1b, s0a, s0b, s1a;
  if (rd.comp) {
    m0a = 0; m0b = rd.lo; m1a = rd.hi; m1b = n;
    s0a = rd.lo; s0b = rd.hi; s1a = 0;
  } else {
    m0a = rd.lo; m0b = rd.hi; m1a = 0; m1b = 0;
    s0a = 0; s0b = rd.lo; s1a = rd.hi;
  }
  const int ns0 = s0b - s0a;
  const int n_moving = (m0b - m0a) + (m1b - m1a), n_static = n - n_moving;
  const Cols cl{PRUNE, ns0, s0a, s1a};
  int ncol = n_static;
  if (PRUNE) {
    // the moving atoms' (h, rho) box
    float hlo = 3.0e38f, hhi = -3.0e38f, rlo = 3.0e38f, rhi = -3.0e38f;
    for (int ia = lane; ia < n_moving; ia += 32) {
      const float2 ha = w.HR[frag_atom(rd, ia)];
      hlo = fminf(hlo, ha.x);
      hhi = fmaxf(hhi, ha.x);
      rlo = fminf(rlo, ha.y);
      rhi = fmaxf(rhi, ha.y);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      hlo = fminf(hlo, __shfl_xor_sync(FULL, hlo, off));
      hhi = fmaxf(hhi, __shfl_xor_sync(FULL, hhi, off));
      rlo = fminf(rlo, __shfl_xor_sync(FULL, rlo, off));
      rhi = fmaxf(rhi, __shfl_xor_sync(FULL, rhi, off));
    }
    // columns: the static atoms within reach of the box
    ncol = 0;
    for (int k0 = 0; k0 < n_static; k0 += 32) {
      const int k = k0 + lane;
      const bool real = k < n_static;
      const int b = k < ns0 ? s0a + k : s1a + (k - ns0);
      bool keep = false;
      if (real) {
        const float2 hb = w.HR[b];
        const float dh = fmaxf(fmaxf(__fsub_rn(hlo, hb.x), __fsub_rn(hb.x, hhi)), 0.f);
        const float dr = fmaxf(fmaxf(__fsub_rn(rlo, hb.y), __fsub_rn(hb.y, rhi)), 0.f);
        keep = __fmaf_rn(dh, dh, __fmul_rn(dr, dr)) < a.reach2;
      }
      const unsigned km = __ballot_sync(FULL, keep);
      const int col = ncol + __popc(km & ((1u << lane) - 1u));
      if (keep) w.SL[col] = (uint8_t)b;
      if (real) w.POS[b] = keep ? (uint8_t)col : (uint8_t)0xFF;
      ncol += __popc(km);
    }
    __syncwarp();
  }
  const int nch = (ncol + 31) >> 5;
  nch_out = nch;
  for (int c = 0; c < nch; ++c) {
    const int k = (c << 5) + lane;
    float2 hb = make_float2(3.0e18f, 0.f);  // lanes past the last column never pass
    if (k < ncol) hb = w.HR[col_atom(w, cl, k)];
    uint32_t* col = w.MASK + c;
    for (int seg = 0; seg < 2; ++seg) {
      const int ma = seg ? m1a : m0a, mb = seg ? m1b : m0b;
#pragma unroll 2
      for (int ai = ma; ai < mb; ++ai, col += nch) {
        const float2 ha = w.HR[ai];
        const float dh = __fsub_rn(ha.x, hb.x), dr = __fsub_rn(ha.y, hb.y);
        const unsigned mk = __ballot_sync(FULL, __fmaf_rn(dh, dh, __fmul_rn(dr, dr)) < a.reach2);
        if (lane == 0) *col = mk;
      }
    }
  }
  __syncwarp();
  for (int e = lane; e < rd.n_excl; e += 32) {
    const uint32_t x = HOIST && e == lane ? ex0 : excl[e];
    const int av = x & 0xFF, bv = x >> 8;
    int ia, k;
    if (rd.comp) {
      ia = av < rd.lo ? av : av - (rd.hi - rd.lo);
      k = bv - rd.lo;
    } else {
      ia = av - rd.lo;
      k = bv < rd.lo ? bv : bv - (rd.hi - rd.lo);
    }
    if (PRUNE) k = w.POS[bv];
    if (!PRUNE || k != 0xFF) atomicAnd(w.MASK + ia * nch + (k >> 5), ~(1u << (k & 31)));
  }
  __syncwarp();
  // compaction: lane t takes mask word w0 + t (row ia = word / nch, chunk c); an
  // exclusive scan of the words' bit counts gives each word's first NEAR slot
  const int words = n_moving * nch, cap = 4 * a.nmax;
  // (wi + 1/2) / nch is >= 1/16 from an integer; nch >= 1 without pruning (static atoms exist)
  const float inv_nch = __frcp_rn((float)(PRUNE && nch == 0 ? 1 : nch));
  int base = 0;
  for (int w0 = 0; w0 < words; w0 += 32) {
    const int wi = w0 + lane;
    unsigned mk = wi < words ? w.MASK[wi] : 0u;
    const int cnt = __popc(mk);
    int incl = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int v = __shfl_up_sync(FULL, incl, off);
      if (lane >= off) incl += v;
    }
    int pos = base + incl - cnt;
    const int ia = __float2int_rz(__fmul_rn(__fadd_rn((float)wi, 0.5f), inv_nch));
    const int c = wi - ia * nch;
    while (mk) {
      const int k = (c << 5) + __ffs(mk) - 1;
      mk &= mk - 1;
      if (pos < cap) w.NEAR[pos] = (uint16_t)((ia << 8) | col_atom(w, cl, k));
      ++pos;
    }
    base += __shfl_sync(FULL, incl, 31);
  }
  reach += (unsigned long long)n_moving * (unsigned long long)n_static;
  __syncwarp();
  return base;
}

// Every angle of one rotamer step: bump tests over the step's near pairs (chunks of 32:
// lane t computes pair t's coefficients, shuffles hand them to every lane), then the grid
// gathers of the moving atoms.
template <int S, int G, bool COMPACT>
__device__ unsigned eval_step_near(const SearchArgs& a, const uint8_t* sg, const WarpMem& w, int n,
                                   const RotDesc& rd, float4 xp, float ux, float uy, float uz, int cur,
                                   int n_near, int lane, unsigned long long& pairs, uint8_t* dbg) {
  const float4* X = w.X;
  int m0a, m0b, m1a, m1b;
  if (rd.comp) {
    m0a = 0; m0b = rd.lo; m1a = rd.hi; m1b = n;
  } else {
    m0a = rd.lo; m0b = rd.hi; m1a = 0; m1b = 0;
  }
  const int passes = (a.A + 32 * S - 1) / (32 * S);
  unsigned best = 0;
  for (int pass = 0; pass < passes; ++pass) {
    float2 cs[S];
    int kk[S], sc[S];
    float mind[S];
#pragma unroll
    for (int j = 0; j < S; ++j) {
      kk[j] = lane + 32 * (pass * S + j);
      cs[j] = w.CS[kk[j] < a.A ? kk[j] : 0];
      sc[j] = 0;
      mind[j] = 3.0e38f;
      if (kk[j] < a.A) pairs += (unsigned)n_near;
    }
    for (int e0 = 0; e0 < n_near; e0 += 32) {
      __syncwarp();
      if (e0 + lane < n_near) {
        const int ent = w.NEAR[e0 + lane], ia = ent >> 8;
        const float4 xa = X[frag_atom(rd, ia)], dpa = w.DP[ia];
        w.PC[lane] = pair_coef(xa, dpa, w2_at<COMPACT>(w, ia, xa, xp, ux, uy, uz), X[ent & 0xFF], xp, ux, uy, uz);
      }
      __syncwarp();
      const int cnt = n_near - e0 < 32 ? n_near - e0 : 32;
      // unrolled by 8 with four angles per lane, by 4 with fewer (measured best for each)
#pragma unroll(S >= 4 ? 8 : 4)
      for (int t = 0; t < cnt; ++t) {
        const float4 k = w.PC[t];
#pragma unroll
        for (int j = 0; j < S; ++j) mind[j] = fminf(mind[j], pair_d2(k.x, k.y, k.z, cs[j]));
      }
    }
    int stat = cur;  // running score minus the fragment's cached cells
    int ia = 0;
    for (int seg = 0; seg < 2; ++seg) {
      const int ma = seg ? m1a : m0a, mb = seg ? m1b : m0b;
      for (int ai = ma; ai < mb; ++ai, ++ia) {
        const float4 xa = X[ai];
        stat -= __float_as_int(xa.w);
        const float4 dp = w.DP[ia];
        const float2 w2 = w2_at<COMPACT>(w, ia, xa, xp, ux, uy, uz);
#pragma unroll
        for (int j = 0; j < S; ++j) {
          float x, y, z;
          turn(xa, dp, w2, cs[j], x, y, z);
          sc[j] += cell<G>(a.pk, sg, x, y, z);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < S; ++j)
      if (kk[j] < a.A) {
        const bool bump = mind[j] < a.thr2;
        const unsigned key = bump ? 0u : (((unsigned)(stat + sc[j] + 1) << 16) | (0xFFFFu - (unsigned)kk[j]));
        best = key > best ? key : best;
        if (dbg) dbg[kk[j]] = bump ? 1 : 0;
      }
  }
  return __reduce_max_sync(FULL, best);
}

// Every angle of one rotamer step, bump tests restricted to the near pairs of the
// step's masks (n_near of them); used when the near list overflowed.
template <int S, int G, bool PRUNE, bool COMPACT>
__device__ unsigned eval_step_masks(const SearchArgs& a, const uint8_t* sg, const WarpMem& w, int n,
                                   const RotDesc& rd, float4 xp, float ux, float uy, float uz, int cur,
                                   int n_near, int nch_pruned, int lane, unsigned long long& pairs, uint8_t* dbg) {
  const float4* X = w.X;
  int m0a, m0b, m1a, m1b;
  if (rd.comp) {
    m0a = 0; m0b = rd.lo; m1a = rd.hi; m1b = n;
  } else {
    m0a = rd.lo; m0b = rd.hi; m1a = 0; m1b = 0;
  }
  const Cols cl = step_cols<PRUNE>(rd);
  const int nch = PRUNE ? nch_pruned : (n - (m0b - m0a) - (m1b - m1a) + 31) >> 5;
  const int passes = (a.A + 32 * S - 1) / (32 * S);
  unsigned best = 0;
  for (int pass = 0; pass < passes; ++pass) {
    float2 cs[S];
    int kk[S], sc[S];
    float mind[S];
#pragma unroll
    for (int j = 0; j < S; ++j) {
      kk[j] = lane + 32 * (pass * S + j);
      cs[j] = w.CS[kk[j] < a.A ? kk[j] : 0];
      sc[j] = 0;
      mind[j] = 3.0e38f;
      if (kk[j] < a.A) pairs += (unsigned)n_near;
    }
    int stat = cur;  // running score minus the fragment's cached cells
    const uint32_t* row = w.MASK;
    int ia = 0;
    for (int seg = 0; seg < 2; ++seg) {
      const int ma = seg ? m1a : m0a, mb = seg ? m1b : m0b;
      for (int ai = ma; ai < mb; ++ai, ++ia, row += nch) {
        const float4 xa = X[ai];
        stat -= __float_as_int(xa.w);
        const float4 dp = w.DP[ia];
        const float2 w2 = w2_at<COMPACT>(w, ia, xa, xp, ux, uy, uz);
        float xr[S][3];
#pragma unroll
        for (int j = 0; j < S; ++j) {
          turn(xa, dp, w2, cs[j], xr[j][0], xr[j][1], xr[j][2]);
          sc[j] += cell<G>(a.pk, sg, xr[j][0], xr[j][1], xr[j][2]);
        }
        for (int c = 0; c < nch; ++c) {
          unsigned mk = row[c];
          while (mk) {
            const int k = (c << 5) + __ffs(mk) - 1;
            mk &= mk - 1;
            const float4 kc = pair_coef(xa, dp, w2, X[col_atom(w, cl, k)], xp, ux, uy, uz);
#pragma unroll
            for (int j = 0; j < S; ++j) mind[j] = fminf(mind[j], pair_d2(kc.x, kc.y, kc.z, cs[j]));
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < S; ++j)
      if (kk[j] < a.A) {
        const bool bump = mind[j] < a.thr2;
        const unsigned key = bump ? 0u : (((unsigned)(stat + sc[j] + 1) << 16) | (0xFFFFu - (unsigned)kk[j]));
        best = key > best ? key : best;
        if (dbg) dbg[kk[j]] = bump ? 1 : 0;
      }
  }
  return __reduce_max_sync(FULL, best);
}

// Rigid alignment sweep (align_ligand, Sec. 3.1 / 4.1): candidate m of a local grid of
// rotation vectors step * (i - s, j - s, k - s), i, j, k in [0, 2s], about the pocket
// centre (the origin of the pose's coordinates); m = 0 is the identity and the others
// follow in lexicographic (i, j, k) order without it.
__device__ __forceinline__ Rot3 rigid_rotation(const SearchArgs& a, int m) {
  const int W = 2 * a.rigid_span + 1, centre = (a.rigid_span * W + a.rigid_span) * W + a.rigid_span;
  const int g = m - 1, idx = g < centre ? g : g + 1;
  const float vx = __fmul_rn(a.rigid_step, (float)(idx / (W * W) - a.rigid_span));
  const float vy = __fmul_rn(a.rigid_step, (float)((idx / W) % W - a.rigid_span));
  const float vz = __fmul_rn(a.rigid_step, (float)(idx % W - a.rigid_span));
  const float th = __fsqrt_rn(__fmaf_rn(vx, vx, __fmaf_rn(vy, vy, __fmul_rn(vz, vz))));
  float sn, cs;
  sincosf(th, &sn, &cs);
  const float inv = __frcp_rn(th);
  // about the pocket centre, which sits at `shift` in grid units
  return rodrigues(__fmul_rn(vx, inv), __fmul_rn(vy, inv), __fmul_rn(vz, inv), cs, sn,
                   make_float4(a.pk.shift[0], a.pk.shift[1], a.pk.shift[2], 0.f));
}

__device__ void rigid_apply(const SearchArgs& a, float4* X, int n, int m, int lane) {
  if (m <= 0) return;
  const Rot3 R = rigid_rotation(a, m);
  __syncwarp();
  for (int i = lane; i < n; i += 32) {
    const float4 v = X[i];
    float x, y, z;
    rot_apply(R, v.x, v.y, v.z, x, y, z);
    X[i] = make_float4(x, y, z, 0.f);
  }
  __syncwarp();
}

// Best rigid candidate by score (ties to the smaller m); applies it and returns m.
template <int G>
__device__ int rigid_align(const SearchArgs& a, const uint8_t* sg, float4* X, int n, int lane) {
  unsigned best = 0;
  for (int m = lane; m < a.rigid_n; m += 32) {
    int sc = 0;
    if (m == 0) {
      for (int i = 0; i < n; ++i) {
        const float4 v = X[i];
        sc += cell<G>(a.pk, sg, v.x, v.y, v.z);
      }
    } else {
      const Rot3 R = rigid_rotation(a, m);
      for (int i = 0; i < n; ++i) {
        const float4 v = X[i];
        float x, y, z;
        rot_apply(R, v.x, v.y, v.z, x, y, z);
        sc += cell<G>(a.pk, sg, x, y, z);
      }
    }
    const unsigned key = ((unsigned)(sc + 1) << 16) | (0xFFFFu - (unsigned)m);
    best = key > best ? key : best;
  }
  best = __reduce_max_sync(FULL, best);
  const int m = (int)(0xFFFFu - (best & 0xFFFFu));
  rigid_apply(a, X, n, m, lane);
  return m;
}

// a10: reduce over the ligand's restarts, replay the winner, write the results.  SRV (the
// streaming server): the results go to the slot's row of the mapped result arrays, then
// the slot's completion counter is cleared and result_seq raised (system scope) so the
// host sees them.
template <int G, bool SRV>
__device__ void finalize(const SearchArgs& a, const uint8_t* sg, const WarpMem& w, int li, int lane,
                         const ServeArgs* sv) {
  float4* X = w.X;
  const int O = a.O;
  unsigned best = 0;
  unsigned long long pairs = 0, reach = 0;
  for (int o = lane; o < O; o += 32) {
    const unsigned s = __ldcg(a.pose_score + (size_t)li * O + o);
    if (s == NOT_SEARCHED) continue;  // restarts left out of a chosen subset
    const unsigned key = ((s + 1u) << 16) | (0xFFFFu - (unsigned)o);
    best = key > best ? key : best;
    pairs += __ldcg(a.pose_pairs + (size_t)li * O + o);
    reach += __ldcg(a.pose_reach + (size_t)li * O + o);
  }
  best = __reduce_max_sync(FULL, best);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    pairs += __shfl_xor_sync(FULL, pairs, off);
    reach += __shfl_xor_sync(FULL, reach, off);
  }
  const int ob = (int)(0xFFFFu - (best & 0xFFFFu));
  const unsigned sb = (best >> 16) - 1u;
  int a0, n, r0, R;
  lig_span<SRV>(a, li, a0, n, r0, R);
  const size_t pick_base = (size_t)r0 * a.reps * O + (size_t)ob * a.reps * R;
  unsigned long long fsum = 0;  // sum of fragment sizes over the rotamers
  for (int r = lane; r < R; r += 32) {
    const RotDesc d = w.RD[r];  // the ligand's descriptors (this warp's copy, or global memory)
    const int sub = (int)d.hi - (int)d.lo;
    fsum += (unsigned long long)(d.comp ? n - sub : sub);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) fsum += __shfl_xor_sync(FULL, fsum, off);
  const unsigned long long nres = SRV ? (unsigned long long)__ldcg(sv->slot_nres + li)
                                       : (a.item_cnt ? (unsigned long long)a.item_cnt[li] : (unsigned long long)O);
  if (lane == 0) {
    a.best_score[li] = sb;
    a.best_orient[li] = ob;
    a.evals[li] = nres * a.reps * R * a.A;
    a.pair_tests[li] = pairs;
    a.reach_tests[li] = reach;
    a.atom_moves[li] = nres * a.reps * a.A * fsum;
  }
  for (int s = lane; s < a.reps * R; s += 32)
    a.best_angle[(size_t)r0 * a.reps + s] = __ldcg(a.pose_pick + pick_base + s);
  place<SRV>(a, X, a0, n, ob, lane);
  int rig = 0;
  if (a.rigid_n > 1) {
    rig = __ldcg(a.pose_rigid + (size_t)li * O + ob);
    rigid_apply(a, X, n, rig, lane);
  }
  if (lane == 0 && a.best_rigid) a.best_rigid[li] = (int16_t)rig;
  for (int rep = 0; rep < a.reps; ++rep)
    for (int r = 0; r < R; ++r) {
      const int k = __ldcg(a.pose_pick + pick_base + rep * R + r);
      if (k < 0) continue;
      const RotDesc rd = w.RD[r];  // registers: the loops below also write shared memory
      float ux, uy, uz;
      bond_axis(X, rd, ux, uy, uz);
      commit<G>(a.pk, sg, X, n, rd, ux, uy, uz, w.CS[k], lane, nullptr, nullptr);
    }
  for (int i = lane; i < n; i += 32) {
    const float4 v = X[i];
    float* dst = a.best_xyz + 3 * ((size_t)a0 + (SRV ? __ldcg(a.perm + a0 + i) : a.perm[a0 + i]));
    dst[0] = __fadd_rn(__fmul_rn(__fsub_rn(v.x, a.pk.shift[0]), a.pk.h), a.pk.centre[0]);
    dst[1] = __fadd_rn(__fmul_rn(__fsub_rn(v.y, a.pk.shift[1]), a.pk.h), a.pk.centre[1]);
    dst[2] = __fadd_rn(__fmul_rn(__fsub_rn(v.z, a.pk.shift[2]), a.pk.h), a.pk.centre[2]);
  }
  __syncwarp();
  if (SRV) {
    // every lane's result stores before the flag the host polls
    __threadfence_system();
    __syncwarp();
    if (lane == 0) {
      a.done[li] = 0;  // the slot's next ligand starts its count from zero
      const unsigned long long seq1 = __ldcg(sv->slot_ready + li);  // seq + 1
      __threadfence_system();
      asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(sv->result_seq + li), "l"(seq1) : "memory");
    }
    __syncwarp();
  }
}

template <int S, int G, bool PRUNE, bool COMPACT, bool SRV>
__device__ void search_pose(const SearchArgs& a, const uint8_t* sg, const WarpMem& w, int li, int o, int e0,
                            int lane) {
  float4* X = w.X;
  int a0, n, r0, R;
  lig_span<SRV>(a, li, a0, n, r0, R);
  place<SRV>(a, X, a0, n, o, lane);
  {
    const int m = a.rigid_n > 1 ? rigid_align<G>(a, sg, X, n, lane) : 0;
    if (lane == 0 && a.pose_rigid) a.pose_rigid[(size_t)li * a.O + o] = (int16_t)m;
  }
  int cur = score_atoms<G>(a.pk, sg, X, n, lane);
  unsigned long long pairs = 0, reach = 0;
  const size_t pick_base = (size_t)r0 * a.reps * a.O + (size_t)o * a.reps * R;
  for (int rep = 0; rep < a.reps; ++rep)
    for (int r = 0; r < R; ++r) {
      const RotDesc rd = w.RD[r];  // registers: the loops below also write shared memory
      const uint16_t* excl = w.EXL + ((int)rd.excl_off - e0);
      const uint32_t ex0 = COMPACT && a.use_filter && lane < rd.n_excl ? excl[lane] : 0u;
      float ux, uy, uz;
      bond_axis(X, rd, ux, uy, uz);
      uint8_t* dbg = nullptr;
      if (a.bump_bits)
        dbg = a.bump_bits + (size_t)r0 * a.reps * a.O * a.A + ((size_t)o * a.reps * R + rep * R + r) * a.A;
      unsigned key;
      const float4 xp = X[rd.p];
      prep_step<COMPACT>(w, n, rd, xp, ux, uy, uz, lane);
      if (a.use_filter) {
        int nch;
        const int n_near = build_near<PRUNE, COMPACT>(a, w, excl, ex0, n, rd, lane, reach, nch);
        if (n_near <= 4 * a.nmax && !a.mask_sweep)
          key = eval_step_near<S, G, COMPACT>(a, sg, w, n, rd, xp, ux, uy, uz, cur, n_near, lane, pairs, dbg);
        else
          key = eval_step_masks<S, G, PRUNE, COMPACT>(a, sg, w, n, rd, xp, ux, uy, uz, cur, n_near, nch, lane, pairs,
                                                      dbg);
      } else
        key = eval_step<S, G, COMPACT>(a, sg, w, excl, n, rd, xp, ux, uy, uz, cur, lane, pairs, dbg);
      const int k = key ? (int)(0xFFFFu - (key & 0xFFFFu)) : -1;
      if (k >= 0) {
        commit<G>(a.pk, sg, X, n, rd, ux, uy, uz, w.CS[k], lane, w.DP, COMPACT ? nullptr : w.W2);
        cur = (int)(key >> 16) - 1;
      }
      if (lane == 0) a.pose_pick[pick_base + rep * R + r] = (int16_t)k;
      __syncwarp();
    }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) pairs += __shfl_xor_sync(FULL, pairs, off);
  if (lane == 0) {
    a.pose_score[(size_t)li * a.O + o] = (uint32_t)cur;
    a.pose_pairs[(size_t)li * a.O + o] = pairs;
    a.pose_reach[(size_t)li * a.O + o] = reach;
  }
  __syncwarp();
}

// A ligand's rotamer descriptors and excluded pairs into the warp's buffers (compact
// builds: pointed at in global memory, read through L1); returns the offset of its first
// excluded pair.
template <bool COMPACT, bool SRV>
__device__ int load_ligand(const SearchArgs& a, WarpMem& w, int li, int lane) {
  static_assert(!(COMPACT && SRV), "the server's slots are copied into each warp's buffers");
  int a0, n, r0, R;
  lig_span<SRV>(a, li, a0, n, r0, R);
  int e0 = 0;
  if (COMPACT) {
    w.RD = a.rots + r0;
    if (R > 0) e0 = (int)__ldg(&a.rots[r0].excl_off);
    w.EXL = a.excl + e0;
    return e0;
  }
  __syncwarp();
  if (R > 0) {
    for (int i = lane; i < 4 * R; i += 32)
      reinterpret_cast<uint32_t*>(w.RDs)[i] = SRV ? __ldcg(reinterpret_cast<const uint32_t*>(a.rots + r0) + i)
                                                  : __ldg(reinterpret_cast<const uint32_t*>(a.rots + r0) + i);
    __syncwarp();
    e0 = (int)w.RDs[0].excl_off;
    const int ne = (int)w.RDs[R - 1].excl_off + w.RDs[R - 1].n_excl - e0;
    for (int i = lane; i < ne; i += 32) w.EXLs[i] = SRV ? __ldcg(a.excl + e0 + i) : __ldg(a.excl + e0 + i);
  }
  __syncwarp();
  return e0;
}

// Completion of `done` poses of ligand li by this warp: the warp that completes the
// ligand's count reduces its restarts (a10); the fence orders the poses' results first.
template <int G, bool SRV>
__device__ void complete(const SearchArgs& a, const uint8_t* sg, const WarpMem& w, int li, int done, int lane,
                         const ServeArgs* sv = nullptr) {
  __threadfence();
  int prev = 0;
  if (lane == 0) prev = atomicAdd(a.done + li, done);
  prev = __shfl_sync(FULL, prev, 0);
  const int target = SRV ? __ldcg(sv->slot_nres + li) : (a.item_cnt ? a.item_cnt[li] : a.O);
  if (prev + done == target) {
    __threadfence();
    finalize<G, SRV>(a, sg, w, li, lane, sv);
  }
}

// ---- bulk async copy of the grid into shared memory --------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ bool stage_grid(const SearchArgs& a, uint8_t* sg, uint64_t* mbar) {
  const int bytes = a.pk.bytes_pad;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)),
                 "r"(bytes + a.stage_extra_bytes)
                 : "memory");
    constexpr int CHUNK = 32768;
    for (int off = 0; off < bytes; off += CHUNK) {
      const int len = bytes - off < CHUNK ? bytes - off : CHUNK;
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              smem_u32(sg + off)),
          "l"(a.pk.grid + off), "r"(len), "r"(smem_u32(mbar))
          : "memory");
    }
  }
  // bounded wait on phase 0 (about two seconds at the maximum clock).  The outcome is
  // decided once for the block, so every thread returns or goes on together.  A timeout
  // whose copies never land leaves them in flight into this block's shared memory when it
  // exits; the test hook (stage_extra_bytes) only makes the barrier expect more bytes
  // than are copied, so there every copy has landed.
  const long long t0 = clock64();
  uint32_t ok = 0;
  while (!ok) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(mbar))
        : "memory");
    if (!ok && clock64() - t0 > 4000000000LL) break;
  }
  return __syncthreads_and((int)ok) != 0;
}

template <int S, int G, int B>
__global__ void __launch_bounds__(B == BUILD_LEAN ? 256 : (B == BUILD_COMPACT ? 640 : 512), B == BUILD_LEAN ? 3 : 1)
    search_kernel(const __grid_constant__ SearchArgs a) {
  constexpr bool PRUNE = B != BUILD_LEAN, COMPACT = B == BUILD_COMPACT;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint8_t* sg = nullptr;
  size_t off = 0;
  if (G == GRID_SMEM) {
    sg = smem;
    off = (size_t)a.pk.bytes_pad;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + off);
    off += 16;
    if (!stage_grid(a, sg, mbar)) {
      if (threadIdx.x == 0) atomicExch(a.err, ERR_STAGE_TIMEOUT);
      return;
    }
  }
  // (cos, sin) of every angle, once per block
  float2* cs = reinterpret_cast<float2*>(smem + off);
  for (int k = threadIdx.x; k < a.A; k += blockDim.x) cs[k] = angle_entry(k, a.A);
  off += ((size_t)a.A * 8 + 15) / 16 * 16;
  __syncthreads();
  const int warp_bytes = warp_smem_bytes(a.nmax, a.fmax, a.mask_words, a.rmax, a.emax, COMPACT);
  WarpMem w = warp_mem(smem + off + (size_t)warp * warp_bytes, a.nmax, a.fmax, a.mask_words, a.rmax, a.emax, COMPACT);
  w.CS = cs;
  // items: every (ligand, restart) in queue order, or an explicit list of rows li*O + o;
  // a warp takes a.chunk consecutive items at a time (mostly restarts of one ligand), loads
  // a ligand's descriptors once per run of its restarts and reports the run's completion
  // with one atomic
  const unsigned long long CHUNK = (unsigned long long)a.chunk;
  const unsigned long long n_items = a.items ? (unsigned long long)*a.n_items_dev : (unsigned long long)a.n_items;
  const unsigned long long n_chunks = (n_items + CHUNK - 1) / CHUNK;
  int cur = -1, e0 = 0, pending = 0;
  for (;;) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(a.work, 1ull);
    t = __shfl_sync(FULL, t, 0);
    if (t >= n_chunks) break;
    const unsigned long long q1 = (t + 1) * CHUNK < n_items ? (t + 1) * CHUNK : n_items;
    for (unsigned long long q = t * CHUNK; q < q1; ++q) {
      int li, o;
      if (a.items) {
        const unsigned row = __ldg(a.items + q);
        li = (int)(row / (unsigned)a.O);
        o = (int)(row % (unsigned)a.O);
      } else {
        li = a.order[q / (unsigned long long)a.O];
        o = (int)(q % (unsigned long long)a.O);
      }
      if (li != cur) {
        if (pending) complete<G, false>(a, sg, w, cur, pending, lane);
        cur = li;
        pending = 0;
        e0 = load_ligand<COMPACT, false>(a, w, li, lane);
      }
      search_pose<S, G, PRUNE, COMPACT, false>(a, sg, w, li, o, e0, lane);
      ++pending;
    }
  }
  if (pending) complete<G, false>(a, sg, w, cur, pending, lane);
}

// ---- the streaming server's persistent launch ---------------------------------------
//
// Continuous batching into one running launch: the host writes each arriving ligand's
// record into its slot of mapped host memory and raises a published count; each warp
// takes a ticket for the next work item (4 restarts of one ligand) and starts on it once
// it is published; a ticket still unpublished when the launch ends idle is parked for the
// same warp of the next launch, which goes on from the same device-side counter.  The
// first warp to start on any of a ligand's items (an atomic per slot decides) copies its
// record into the slot's device arrays (centred coordinates computed as the pose-setup
// kernel does) and releases the slot; warps with the ligand's other items wait for that
// (bounded).
// The warp that completes a ligand's restarts writes its results into the slot's row of
// the mapped result arrays and raises the slot's result sequence.  Every wait is bounded
// by the SM clock: a launch closes once every warp has waited idle_cycles without work
// (or is gone), a slot wait that runs out sets ERR_SLOT_TIMEOUT in the mapped status word
// and ends the warp.

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// A word of mapped host memory: fetched again over the bus (cached copies of system
// memory count as stale), then a system-scope fence orders the reads after it.
__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long* p) {
  const unsigned long long v = __ldcv(p);
  asm volatile("fence.acq_rel.sys;" ::: "memory");
  return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed_gpu(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// The launch's warp counts -- warps started (bits 31..61), warps idle or gone (bits
// 0..30) -- and its closing flag, changed together by compare-and-swap.  step +1: this
// warp is idle or gone (the warp that makes every started warp idle or gone sets
// SERVE_CLOSING); -1: it has work again; 0: it starts (a warp scheduled late, after the
// others, joins the count).  Each returns false, changing nothing, once the launch is
// closing.
__device__ bool serve_idle_step(const ServeArgs& s, int step) {
  unsigned long long v = ld_relaxed_gpu(s.idle_state);
  for (;;) {
    if (v & SERVE_CLOSING) return false;
    unsigned long long nv = step > 0 ? v + 1ull : (step < 0 ? v - 1ull : v + SERVE_STARTED_ONE);
    if (step > 0 && (nv & (SERVE_STARTED_ONE - 1ull)) == (nv >> 31)) nv |= SERVE_CLOSING;
    const unsigned long long w = atomicCAS(s.idle_state, v, nv);
    if (w == v) return true;
    v = w;
  }
}

// Lane 0 of warp gw (its position in the grid, the same in every launch): take the next
// work item and wait until it is published (0, *t set); 1 when the host asked the launch
// to stop (the ticket is dropped: nothing more is published); 2 when the launch closes
// idle -- the ticket is then parked in parked[gw] and taken up again by the same grid
// position of the next launch, so no item is lost.  A warp whose item is not published
// within idle_cycles SM cycles counts itself idle; the launch closes when every started
// warp is idle or gone (one compare-and-swap decides it), so no warp leaves while others
// run: a parked item is never one that a running launch's warps wait for, and a warp that
// starts after the launch closed leaves without a ticket.  (Past 64 idle_cycles a warp
// leaves regardless, which only bounds the wait.)  Tickets come from one atomicAdd each,
// so warps never retry against each other.  The mapped control words are read by one
// warp at a time, at most every 2 us of the global timer, and in any case by a warp whose
// own last read is about 0.5 ms of its SM clock old (so no timer can keep the launch from
// seeing new work); between checks a waiting warp sleeps 64 ns doubling up to 32 us.
__device__ int serve_claim(const ServeArgs& s, int gw, unsigned long long* t, long long& my_poll) {
  unsigned long long tk = s.parked[gw];
  if (tk) {
    s.parked[gw] = 0ull;
    tk -= 1ull;
  } else {
    tk = atomicAdd(s.work, 1ull);
  }
  const long long c0 = clock64();
  unsigned sleep_ns = 64;
  bool idle = false;
  for (;;) {
    if (tk < ld_acquire_gpu(s.pub_dev) * (unsigned long long)s.chunks) {
      if (idle && !serve_idle_step(s, -1)) break;  // published as the launch closed
      *t = tk;
      return 0;
    }
    const long long c = clock64();
    const unsigned long long now = globaltimer_ns();
    const unsigned long long last = ld_relaxed_gpu(s.last_poll);
    const bool due = now - last > 2000ull && now >= last && atomicCAS(s.last_poll, last, now) == last;
    if (due || c - my_poll > 1000000LL) {
      my_poll = c;
      const unsigned long long ph = ld_acquire_sys(s.published);
      const int stop = __ldcv(s.stop);
      asm volatile("red.release.gpu.global.max.u64 [%0], %1;" ::"l"(s.pub_dev), "l"(ph) : "memory");
      if (stop) atomicExch(s.stop_dev, 1ull);
      atomicAdd(s.polls, 1ull);
      if (tk < ph * (unsigned long long)s.chunks) continue;
    }
    if (ld_relaxed_gpu(s.stop_dev)) return 1;
    if (!idle && c - c0 > s.idle_cycles) {
      idle = true;
      serve_idle_step(s, +1);
    }
    if (idle && (ld_relaxed_gpu(s.idle_state) & SERVE_CLOSING)) break;
    if (c - c0 > 64 * s.idle_cycles) break;
    // backoff to 32 us: with every warp of the GPU idle here, shorter sleeps put ~1e9
    // loads/s of these words on one L2 slice and starved the warps still searching
    // (their items ran 200x slower at the end of a stream)
    __nanosleep(sleep_ns);
    sleep_ns = sleep_ns < 32768u ? 2u * sleep_ns : 32768u;
  }
  s.parked[gw] = tk + 1ull;
  return 2;
}

// The warp that claimed ligand seq's first item: its record (mapped host memory, read
// with cache-bypassing loads) into slot `slot`, then the slot released to the other items.
__device__ void serve_stage(const SearchArgs& a, const ServeArgs& s, int slot, unsigned long long seq, int lane) {
  const unsigned char* rec = s.rec + (size_t)slot * (size_t)s.rec_stride;
  const int4 h = __ldcv(reinterpret_cast<const int4*>(rec));
  const int amax = a.slot_amax, rmax = a.slot_rmax;
  // the host validated these against the slot sizes; clamped again so that no record can
  // make this warp write outside its slot
  const int n = min(max(h.x, 1), amax), R = min(max(h.y, 0), rmax), ne = min(max(h.z, 0), s.emax);
  // the restarts to search: a list of n_res of them (validated on the host), else all;
  // a listed ligand's other restarts are marked unsearched for the reduction over them
  const int nres = h.w > 0 && h.w < a.O ? h.w : a.O;
  if (nres < a.O) {
    const unsigned short* res = reinterpret_cast<const unsigned short*>(rec + serve_rec_res_dev(amax, rmax, s.emax));
    for (int i = lane; i < nres; i += 32) s.slot_res[(size_t)slot * a.O + i] = (uint16_t)min((int)__ldcv(res + i), a.O - 1);
    for (int o = lane; o < a.O; o += 32) a.pose_score[(size_t)slot * a.O + o] = NOT_SEARCHED;
  }
  if (lane == 0) s.slot_nres[slot] = nres;
  const float4* x0 = reinterpret_cast<const float4*>(rec + 16);
  // centroid and centred coordinates with the pose-setup kernel's arithmetic and order
  float sx = 0.f, sy = 0.f, sz = 0.f;
  for (int i = lane; i < n; i += 32) {
    const float4 v = __ldcv(x0 + i);
    sx = __fadd_rn(sx, v.x);
    sy = __fadd_rn(sy, v.y);
    sz = __fadd_rn(sz, v.z);
  }
  sx = warp_sum_f(sx);
  sy = warp_sum_f(sy);
  sz = warp_sum_f(sz);
  const float cx = __fdiv_rn(sx, (float)n), cy = __fdiv_rn(sy, (float)n), cz = __fdiv_rn(sz, (float)n);
  float4* xc = a.xc + (size_t)slot * amax;
  for (int i = lane; i < n; i += 32) {
    const float4 v = __ldcv(x0 + i);
    xc[i] = make_float4(__fsub_rn(v.x, cx), __fsub_rn(v.y, cy), __fsub_rn(v.z, cz), 0.f);
  }
  const unsigned char* perm = rec + serve_rec_perm_dev(amax);
  uint8_t* dperm = const_cast<uint8_t*>(a.perm) + (size_t)slot * amax;
  for (int i = lane; i < n; i += 32) dperm[i] = __ldcv(perm + i);
  const uint4* rots = reinterpret_cast<const uint4*>(rec + serve_rec_rots_dev(amax));
  uint4* drots = reinterpret_cast<uint4*>(const_cast<RotDesc*>(a.rots) + (size_t)slot * rmax);
  for (int r = lane; r < R; r += 32) {
    uint4 d = __ldcv(rots + r);
    d.w += (unsigned)(slot * s.emax);  // excl_off: into the slot's excluded pairs
    drots[r] = d;
  }
  const unsigned short* ex = reinterpret_cast<const unsigned short*>(rec + serve_rec_excl_dev(amax, rmax));
  uint16_t* dex = const_cast<uint16_t*>(a.excl) + (size_t)slot * s.emax;
  for (int i = lane; i < ne; i += 32) dex[i] = __ldcv(ex + i);
  if (lane == 0) {
    const_cast<int32_t*>(a.slot_n)[slot] = n;
    const_cast<int32_t*>(a.slot_r)[slot] = R;
  }
  __threadfence();
  __syncwarp();
  if (lane == 0 && (long long)seq != s.hold_seq)
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(s.slot_ready + slot), "l"(seq + 1ull) : "memory");
  __syncwarp();
}

// Wait (bounded) until ligand seq's slot is staged; false when the wait ran out.
__device__ bool serve_wait(const ServeArgs& s, int slot, unsigned long long seq, int lane) {
  int ok = 0;
  if (lane == 0) {
    const long long c0 = clock64();
    unsigned sleep_ns = 128;
    for (;;) {
      if (ld_acquire_gpu(s.slot_ready + slot) == seq + 1ull) {
        ok = 1;
        break;
      }
      if (clock64() - c0 > s.wait_cycles) break;
      __nanosleep(sleep_ns);
      sleep_ns = sleep_ns < 2048u ? 2u * sleep_ns : 2048u;
    }
  }
  ok = __shfl_sync(FULL, ok, 0);
  __syncwarp();
  return ok != 0;
}

template <int S, int G, int B>
__global__ void __launch_bounds__(B == BUILD_LEAN ? 256 : 512, B == BUILD_LEAN ? 3 : 1)
    serve_kernel(const __grid_constant__ SearchArgs a, const __grid_constant__ ServeArgs sv) {
  static_assert(B != BUILD_COMPACT, "the server copies descriptors into each warp's buffers");
  constexpr bool PRUNE = B != BUILD_LEAN;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint8_t* sg = nullptr;
  size_t off = 0;
  if (G == GRID_SMEM) {
    sg = smem;
    off = (size_t)a.pk.bytes_pad;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + off);
    off += 16;
    if (!stage_grid(a, sg, mbar)) {
      if (threadIdx.x == 0) {
        atomicExch(a.err, ERR_STAGE_TIMEOUT);
        *reinterpret_cast<volatile int*>(sv.status) = ERR_STAGE_TIMEOUT;
        __threadfence_system();
      }
      return;
    }
  }
  float2* cs = reinterpret_cast<float2*>(smem + off);
  for (int k = threadIdx.x; k < a.A; k += blockDim.x) cs[k] = angle_entry(k, a.A);
  off += ((size_t)a.A * 8 + 15) / 16 * 16;
  __syncthreads();
  const int warp_bytes = warp_smem_bytes(a.nmax, a.fmax, a.mask_words, a.rmax, a.emax, false);
  WarpMem w = warp_mem(smem + off + (size_t)warp * warp_bytes, a.nmax, a.fmax, a.mask_words, a.rmax, a.emax, false);
  w.CS = cs;
  unsigned long long cur_seq = ~0ull;
  int e0 = 0;
  long long my_poll = clock64();
  const int gw = (int)(blockIdx.x * (blockDim.x >> 5)) + warp;
  // join the launch's warp count; a launch that closed before this warp was scheduled has
  // nothing left for it (a ticket it parked earlier waits for the next launch)
  int joined = 0;
  if (lane == 0) joined = serve_idle_step(sv, 0) ? 1 : 0;
  if (!__shfl_sync(FULL, joined, 0)) return;
  for (;;) {
    unsigned long long t = 0;
    int st = 0;
    if (lane == 0) st = serve_claim(sv, gw, &t, my_poll);
    st = __shfl_sync(FULL, st, 0);
    t = __shfl_sync(FULL, t, 0);
    if (st) break;
    const unsigned long long seq = t / (unsigned long long)sv.chunks;
    const int c = (int)(t % (unsigned long long)sv.chunks);
    const int slot = (int)(seq % (unsigned long long)sv.cap);
    // the first warp to reach ligand seq, whichever of its items it holds, stages the
    // slot: the warp holding the first item may have parked it and left an idle launch
    // while live warps took the later items once they were published
    unsigned long long prev = 0;
    if (lane == 0) prev = atomicMax(sv.slot_claim + slot, seq + 1ull);
    prev = __shfl_sync(FULL, prev, 0);
    if (prev < seq + 1ull) {
      serve_stage(a, sv, slot, seq, lane);
    } else if (!serve_wait(sv, slot, seq, lane)) {
      if (lane == 0) {
        *reinterpret_cast<volatile int*>(sv.status) = ERR_SLOT_TIMEOUT;
        __threadfence_system();
        serve_idle_step(sv, +1);  // gone: the idle warps need not wait for this one
      }
      break;
    }
    // item c covers positions [o0, o1) of the ligand's restarts (its list, or all in order);
    // items past a shorter list have nothing to search
    const int nres = __ldcg(sv.slot_nres + slot);
    const int o0 = c * sv.chunk, o1 = o0 + sv.chunk < nres ? o0 + sv.chunk : nres;
    if (o0 >= o1) continue;
    if (seq != cur_seq) {
      cur_seq = seq;
      e0 = load_ligand<false, true>(a, w, slot, lane);
    }
    for (int q = o0; q < o1; ++q) {
      const int o = nres < a.O ? (int)__ldcg(sv.slot_res + (size_t)slot * a.O + q) : q;
      search_pose<S, G, PRUNE, false, true>(a, sg, w, slot, o, e0, lane);
    }
    // completed right away: a ligand's result must not wait for this warp's next item
    complete<G, true>(a, sg, w, slot, o1 - o0, lane, &sv);
  }
}

// Raise a kernel's dynamic shared-memory limit to at least `bytes` on the current device.
// The limit is per function, so it only ever grows: jobs planned on other host threads
// with larger buffers keep a limit that covers their launches.
cudaError_t raise_smem_limit(const void* fn, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> limit;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> g(mu);
  size_t& cur = limit[{fn, dev}];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

// Resident blocks per SM of a kernel at a block size and dynamic shared memory, queried
// once per (kernel, device, shape) and remembered: jobs are planned per call, and the
// query costs more host time than the search of a single ligand's restarts.
cudaError_t blocks_per_sm(const void* fn, int threads, size_t smem, int* per_sm) {
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, int, size_t>, int> known;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const auto key = std::make_tuple(fn, dev, threads, smem);
  {
    std::lock_guard<std::mutex> g(mu);
    auto it = known.find(key);
    if (it != known.end()) {
      *per_sm = it->second;
      return cudaSuccess;
    }
  }
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, threads, smem);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> g(mu);
  known[key] = *per_sm;
  return cudaSuccess;
}

template <int S, int G, int B>
cudaError_t plan_t(const SearchArgs& a, int warps, size_t smem, int num_sms, LaunchCfg* cfg) {
  auto k = search_kernel<S, G, B>;
  cudaError_t e = raise_smem_limit((const void*)k, smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = blocks_per_sm((const void*)k, warps * 32, smem, &per_sm);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long blocks = (long long)per_sm * num_sms;
  const long long need = ((a.n_items + a.chunk - 1) / a.chunk + warps - 1) / warps;
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  cfg->fn = (const void*)k;
  cfg->blocks = (unsigned)blocks;
  cfg->threads = (unsigned)(warps * 32);
  cfg->smem = smem;
  return cudaSuccess;
}

// ids 1..12: wide builds (<= 128 registers), one block of up to 16 warps per SM, the grid
// staged when it fits; ids 13..15: lean builds (<= 80 registers) for up to 24 warps per
// SM; ids 16..20: compact builds (<= 96 registers, compact per-warp buffers) for about 20
// warps per SM with large ligands, or fewer warps (12, 16) that leave more of the SM's
// L1 to the texture path.
constexpr Tile kTiles[] = {{8, 1, BUILD_WIDE},     {8, 2, BUILD_WIDE},     {8, 4, BUILD_WIDE},
                           {4, 1, BUILD_WIDE},     {4, 2, BUILD_WIDE},     {4, 4, BUILD_WIDE},
                           {16, 1, BUILD_WIDE},    {16, 2, BUILD_WIDE},    {16, 4, BUILD_WIDE},
                           {2, 1, BUILD_WIDE},     {2, 2, BUILD_WIDE},     {2, 4, BUILD_WIDE},
                           {8, 1, BUILD_LEAN},     {8, 2, BUILD_LEAN},     {4, 2, BUILD_LEAN},
                           {20, 4, BUILD_COMPACT}, {20, 2, BUILD_COMPACT}, {10, 4, BUILD_COMPACT},
                           {16, 4, BUILD_COMPACT}, {12, 4, BUILD_COMPACT}};
constexpr int kLean8x1 = 13;

template <int B>
cudaError_t plan_build(const SearchArgs& a, const Tile& t, bool tex, size_t smem, int num_sms, LaunchCfg* cfg) {
  switch (t.slots * 2 + (tex ? 1 : 0)) {
    case 2: return plan_t<1, GRID_LDG, B>(a, t.warps, smem, num_sms, cfg);
    case 3: return plan_t<1, GRID_TEX, B>(a, t.warps, smem, num_sms, cfg);
    case 4: return plan_t<2, GRID_LDG, B>(a, t.warps, smem, num_sms, cfg);
    case 5: return plan_t<2, GRID_TEX, B>(a, t.warps, smem, num_sms, cfg);
    case 8: return plan_t<4, GRID_LDG, B>(a, t.warps, smem, num_sms, cfg);
    default: return plan_t<4, GRID_TEX, B>(a, t.warps, smem, num_sms, cfg);
  }
}

}  // namespace

int tile_count() { return (int)(sizeof(kTiles) / sizeof(kTiles[0])); }
Tile tile_get(int id) { return kTiles[id - 1]; }
int max_smem_grid_bytes() { return 200 * 1024; }

size_t search_smem_bytes(const SearchArgs& a, int tile, bool grid_in_smem) {
  const Tile t = tile_get(tile);
  const bool compact = t.build == BUILD_COMPACT;
  size_t s = (size_t)t.warps * (size_t)warp_smem_bytes(a.nmax, a.fmax, a.mask_words, a.rmax, a.emax, compact) +
             ((size_t)a.A * 8 + 15) / 16 * 16;
  if (grid_in_smem) s += (size_t)a.pk.bytes_pad + 16;
  return s;
}

int default_tile(const SearchArgs& a) {
  const int two = a.A >= 64 ? 1 : 0;  // two angles per lane once there are 64 angles
  // lean 8-warp blocks when three of them fit in an SM's 228 KB (1 KB reserved per block)
  if (3 * (search_smem_bytes(a, kLean8x1 + two, false) + 1024) <= 228 * 1024) return kLean8x1 + two;
  // else the wide 8-warp tile, giving up warps (8 -> 4 -> 2, same slots) until one block fits
  int t = 1 + two;
  for (int k = 0; k < 2 && search_smem_bytes(a, t, false) > 227 * 1024; ++k) t += k == 0 ? 3 : 6;
  return t;
}

cudaError_t plan_search(const SearchArgs& a, int tile, bool grid_in_smem, int num_sms, LaunchCfg* cfg) {
  const Tile t = tile_get(tile);
  const size_t smem = search_smem_bytes(a, tile, grid_in_smem);
  const bool tex = !grid_in_smem && a.pk.tex != 0;
  if (grid_in_smem) {
    if (!tile_stages_grid(t)) return cudaErrorInvalidConfiguration;
    switch (t.slots) {
      case 1: return plan_t<1, GRID_SMEM, BUILD_WIDE>(a, t.warps, smem, num_sms, cfg);
      case 2: return plan_t<2, GRID_SMEM, BUILD_WIDE>(a, t.warps, smem, num_sms, cfg);
      default: return plan_t<4, GRID_SMEM, BUILD_WIDE>(a, t.warps, smem, num_sms, cfg);
    }
  }
  switch (t.build) {
    case BUILD_LEAN: return plan_build<BUILD_LEAN>(a, t, tex, smem, num_sms, cfg);
    case BUILD_COMPACT: return plan_build<BUILD_COMPACT>(a, t, tex, smem, num_sms, cfg);
    default: return plan_build<BUILD_WIDE>(a, t, tex, smem, num_sms, cfg);
  }
}

namespace {

template <int S, int G, int B>
cudaError_t plan_serve_t(int warps, size_t smem, int num_sms, LaunchCfg* cfg) {
  auto k = serve_kernel<S, G, B>;
  cudaError_t e = raise_smem_limit((const void*)k, smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = blocks_per_sm((const void*)k, warps * 32, smem, &per_sm);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  cfg->fn = (const void*)k;
  cfg->blocks = (unsigned)(per_sm * num_sms);  // persistent: every SM full
  cfg->threads = (unsigned)(warps * 32);
  cfg->smem = smem;
  return cudaSuccess;
}

}  // namespace

cudaError_t plan_serve(const SearchArgs& a, int tile, bool grid_in_smem, int num_sms, LaunchCfg* cfg) {
  const Tile t = tile_get(tile);
  if (t.build == BUILD_COMPACT) return cudaErrorInvalidConfiguration;
  const size_t smem = search_smem_bytes(a, tile, grid_in_smem);
  if (grid_in_smem) {
    if (!tile_stages_grid(t)) return cudaErrorInvalidConfiguration;
    switch (t.slots) {
      case 1: return plan_serve_t<1, GRID_SMEM, BUILD_WIDE>(t.warps, smem, num_sms, cfg);
      case 2: return plan_serve_t<2, GRID_SMEM, BUILD_WIDE>(t.warps, smem, num_sms, cfg);
      default: return plan_serve_t<4, GRID_SMEM, BUILD_WIDE>(t.warps, smem, num_sms, cfg);
    }
  }
  if (!a.pk.tex) return cudaErrorInvalidConfiguration;  // the server reads the grid through the texture
  if (t.build == BUILD_LEAN) {
    if (t.slots == 1) return plan_serve_t<1, GRID_TEX, BUILD_LEAN>(t.warps, smem, num_sms, cfg);
    if (t.slots == 2) return plan_serve_t<2, GRID_TEX, BUILD_LEAN>(t.warps, smem, num_sms, cfg);
    return cudaErrorInvalidConfiguration;
  }
  switch (t.slots) {
    case 1: return plan_serve_t<1, GRID_TEX, BUILD_WIDE>(t.warps, smem, num_sms, cfg);
    case 2: return plan_serve_t<2, GRID_TEX, BUILD_WIDE>(t.warps, smem, num_sms, cfg);
    default: return plan_serve_t<4, GRID_TEX, BUILD_WIDE>(t.warps, smem, num_sms, cfg);
  }
}

cudaError_t launch_serve(const SearchArgs& a, const ServeArgs& sv, const LaunchCfg& cfg, cudaStream_t st) {
  void* args[] = {const_cast<SearchArgs*>(&a), const_cast<ServeArgs*>(&sv)};
  return cudaLaunchKernel(cfg.fn, dim3(cfg.blocks), dim3(cfg.threads), args, cfg.smem, st);
}

cudaError_t launch_restart_tables(const SearchArgs& a, cudaStream_t st) {
  SearchArgs t = a;  // rotations and quaternions of every restart only: no ligands
  t.L = 0;
  const int blocks = (int)std::min(1024LL, std::max(1LL, ((long long)a.O + 255) / 256));
  pose_setup_kernel<<<blocks, 256, 0, st>>>(t);
  return cudaGetLastError();
}

cudaError_t launch_search(const SearchArgs& a, const LaunchCfg& cfg, cudaStream_t st) {
  const long long need = std::max((long long)a.O, 32LL * a.L);
  const int blocks = (int)std::min(1024LL, std::max(1LL, (need + 255) / 256));
  pose_setup_kernel<<<blocks, 256, 0, st>>>(a);
  void* args[] = {const_cast<SearchArgs*>(&a)};
  return cudaLaunchKernel(cfg.fn, dim3(cfg.blocks), dim3(cfg.threads), args, cfg.smem, st);
}

}  // namespace gd
