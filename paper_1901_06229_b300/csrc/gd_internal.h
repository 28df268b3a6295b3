// Internal layout shared by the host runtime (gd_api.cu) and the search kernel
// (gd_search.cu).  Not part of the public ABI.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace gd {

// One rotamer as the kernel sees it.  Atoms of a ligand are renumbered in DFS
// preorder from atom 0, so the subtree under either end of a tree bond is one
// contiguous range [lo, hi); the rotating fragment is that range (comp = 0) or its
// complement (comp = 1).  p / q are the static / moving ends of the bond (preorder
// ids).  excl[excl_off .. excl_off + n_excl) lists the moving x static pairs whose
// graph distance is below min_bond_sep as (a | b << 8), sorted by the moving atom a:
// in a tree every moving-static path runs through q-p, so these are the pairs with
// dist(a,q) + 1 + dist(p,b) < min_bond_sep.
struct alignas(16) RotDesc {
  uint16_t p, q;
  uint16_t lo, hi;
  uint8_t comp;
  uint8_t n_excl;
  uint16_t pad;
  uint32_t excl_off;
};
static_assert(sizeof(RotDesc) == 16, "RotDesc layout");

// Words of one rotamer step's near-pair masks in a ligand of n atoms: one 32-bit word
// per moving atom and per 32 static atoms.
__host__ __device__ inline int step_mask_words(int n, const RotDesc& d) {
  const int sub = (int)d.hi - (int)d.lo, f = d.comp ? n - sub : sub;
  return f * ((n - f + 31) / 32);
}

struct PocketDev {
  const uint8_t* grid;   // cropped grid [cz][cy][cx]; cells outside the crop are 0
  int cx, cy, cz;        // crop extents (cells)
  int bytes_pad;         // cx*cy*cz rounded up to 16 (bulk-copy granule)
  float inv_h, h;        // 1 / spacing, spacing (A)
  float shift[3];        // n/2 - crop_lo per axis: cell = floor(x_rel * inv_h + shift)
  float centre[3];       // pocket centre (world): x_world = x_rel + centre
  unsigned long long tex;  // texture object over the crop (point sampling, border 0,
                           // unnormalised coordinates); 0: none (grid read through L1)
};

struct SearchArgs {
  PocketDev pk;
  // batch (preorder-packed)
  int L;
  const int32_t* atom_off;    // [L+1]
  const int32_t* rot_off;     // [L+1]
  const float4* xyz;          // [N] preorder, input coordinates (w unused)
  const uint8_t* perm;        // [N] preorder id -> input-order local id
  const RotDesc* rots;        // [Rt]
  const uint16_t* excl;       // [sum n_excl] excluded pairs (a | b << 8)
  const int32_t* order;       // [L] ligand processing order (largest cost first)
  long long n_items;          // L * O
  int chunk;                  // items a warp takes at a time (4 for large batches, else 1)
  const uint32_t* items;      // optional explicit (ligand, restart) list, rows li * O + o
  const int32_t* item_cnt;    // with items: restarts searched per ligand (>= 1)
  const int32_t* n_items_dev; // with items: list length (device scalar)
  // search parameters
  int na, nb, ng, O, A, reps;
  // The search keeps pose coordinates in grid units, g = x_rel * inv_h + shift (so a
  // point's cell is floor(g)); both squared distances are in those units.
  float thr2;                 // (bump_dist inv_h)^2
  float reach2;               // ((bump_dist + REACH_MARGIN) inv_h)^2: pairs farther apart at every angle skip the test
  int use_filter;             // 1: per-rotamer reach filter; 0: test every moving x static pair
  int mask_sweep;             // 1: always sweep the filter's masks, never its near list
  // outputs
  uint32_t* best_score;       // [L]
  int32_t* best_orient;       // [L]
  int16_t* best_angle;        // [reps * Rt]
  float* best_xyz;            // [3N]
  unsigned long long* evals;  // [L]
  unsigned long long* pair_tests;  // [L]
  unsigned long long* atom_moves;  // [L]
  // scratch
  uint32_t* pose_score;       // [L*O]
  int16_t* pose_pick;         // [O * reps * Rt]
  unsigned long long* pose_pairs;  // [L*O]
  int32_t* done;              // [L]   zeroed by the pose-setup kernel before every search
  unsigned long long* work;   // [1]   zeroed by the pose-setup kernel before every search
  int32_t* err;               // [1]   0 = fine, else error code (output block; zeroed at setup)
  // debug (may be null)
  uint8_t* bump_bits;         // [O * reps * A * Rt]
  int nmax;                   // largest ligand of the batch (per-warp buffer size)
  int mask_words;             // largest step_mask_words of the batch (>= 1)
  float4* xc;                 // [N] (scratch) centred input coordinates x0 - c_lig, preorder
  float* rmat;                // [O * 9] (scratch) restart rotation matrices, row-major
  float4* quat;               // [O] (scratch) restart unit quaternions (w >= 0)
  int fmax;                   // largest rotating fragment of the batch (>= 1)
  int rmax, emax;             // largest rotamer / excluded-pair count of one ligand (>= 1)
  unsigned long long* reach_tests;  // [L] (output) moving x static pairs checked by the reach filter
  unsigned long long* pose_reach;   // [L*O] (scratch)
  // rigid alignment sweep (off when rigid_n <= 1)
  int rigid_span;             // s: candidates are the (2s+1)^3 rotation vectors step * (i-s, j-s, k-s)
  float rigid_step;           // radians
  int rigid_n;                // (2s+1)^3 (identity first)
  int16_t* pose_rigid;        // [L*O] (scratch) chosen rigid candidate per restart
  int16_t* best_rigid;        // [L] (output) of the best restart
  int stage_extra_bytes;      // testing: bytes the grid-staging barrier expects beyond the grid
  // slot layout (the streaming server): ligand li's atoms start at li * slot_amax and its
  // rotamers at li * slot_rmax, with counts slot_n[li] / slot_r[li]; NULL: the CSR offsets
  const int32_t* slot_n;
  const int32_t* slot_r;
  int slot_amax, slot_rmax;
};

// The streaming server's persistent launch (see gd_server_create).  Ligand seq lives in
// slot seq % cap.  The host publishes ligands by raising *published (mapped host memory)
// after writing their records; warps take tickets for work items (item t: ligand
// t / chunks, restarts [4 (t % chunks), ...)) and start on one once it is published; a
// launch that ends idle parks its warps' unpublished tickets for the next launch.
struct ServeArgs {
  const unsigned long long* published;  // (mapped) ligands published so far
  const int* stop;                      // (mapped) 1: exit once every published item is claimed
  int* status;                          // (mapped) 0 fine, ERR_SLOT_TIMEOUT after a wait ran out
  unsigned long long* work;             // items claimed so far (device; persists across launches)
  unsigned long long* pub_dev;          // device copy of *published
  unsigned long long* stop_dev;         // device copy of *stop
  unsigned long long* last_poll;        // globaltimer of the last read of the mapped words
  unsigned long long* slot_ready;       // [cap] seq + 1 once the slot holds ligand seq
  unsigned long long* slot_claim;       // [cap] seq + 1 once a warp has taken the staging of ligand seq
  unsigned long long* result_seq;       // (mapped) [cap] seq + 1 once ligand seq's results are written
  const unsigned char* rec;             // (mapped) [cap] ligand records of rec_stride bytes
  long long rec_stride;
  int cap, emax;                        // slots; excluded pairs per slot
  int chunk, chunks;                    // restarts per item; items per ligand
  long long idle_cycles;                // an idle warp exits after this many SM cycles without work
  long long wait_cycles;                // bound (SM cycles) of a wait for a slot being staged
  long long hold_seq;                   // testing: the ligand whose slot is never released (-1)
  unsigned long long* polls;            // reads of the mapped control words (device counter)
  unsigned long long* parked;           // [warps of the launch] ticket + 1 a warp held when its launch ended idle
  unsigned long long* idle_state;       // this launch's warps: started << 31 | idle or gone | SERVE_CLOSING
                                        // (zeroed before every launch)
  int32_t* slot_nres;                   // [cap] restarts the slot's ligand searches (O: all of them)
  uint16_t* slot_res;                   // [cap * O] which ones, when fewer than O
};
constexpr unsigned long long SERVE_CLOSING = 1ull << 62;
constexpr unsigned long long SERVE_STARTED_ONE = 1ull << 31;

// A ligand record in the server's mapped host memory (slot s at rec + s * rec_stride):
// header, then xyz float4[amax] (preorder, w unused), perm uint8[amax], RotDesc[rmax]
// (excl_off relative to the record's excluded pairs), excl uint16[emax], restarts
// uint16[O] (the restarts to search, n_res of them; n_res 0: every restart in order).
struct ServeRecHeader {
  int32_t n, R, n_excl, n_res;
};
__host__ __device__ inline long long serve_rec_perm_dev(int amax) { return 16 + 16LL * amax; }
__host__ __device__ inline long long serve_rec_rots_dev(int amax) { return (16 + 17LL * amax + 15) / 16 * 16; }
__host__ __device__ inline long long serve_rec_excl_dev(int amax, int rmax) {
  return serve_rec_rots_dev(amax) + 16LL * rmax;
}
__host__ __device__ inline long long serve_rec_res_dev(int amax, int rmax, int emax) {
  return serve_rec_excl_dev(amax, rmax) + 2LL * emax;
}
__host__ __device__ inline long long serve_rec_bytes(int amax, int rmax, int emax, int O) {
  return (serve_rec_res_dev(amax, rmax, emax) + 2LL * O + 127) / 128 * 128;
}

// Margin of the reach filter (A).  FP32 rounding moves a rotated atom by ~1e-5 A at
// most, so a pair whose closest approach over the whole turn exceeds bump_dist by
// this margin can never be flagged by the per-angle test.
constexpr float REACH_MARGIN = 0.01f;

// Per-warp shared memory: X float4[nmax] | HR float2[nmax] (later the near-pair list,
// uint16[4 nmax]) | DP float4[fmax] | W2 float2[fmax] |
// MASK uint32[mask_words] | EXL uint16[emax] | RD RotDesc[rmax] | PC float4[32] (the
// coefficients of the near pairs being swept).  fmax / rmax / emax: the largest
// fragment, rotamer count and excluded-pair count of one ligand in the batch (>= 1).
// compact (the 96-register builds): no W2 (rebuilt from DP) and no EXL / RD (the
// descriptors and excluded pairs are read through L1).
__host__ __device__ inline int warp_smem_bytes(int nmax, int fmax, int mask_words, int rmax, int emax,
                                               bool compact = false) {
  auto a16 = [](int v) { return (v + 15) / 16 * 16; };
  if (compact) return a16(16 * nmax) + a16(8 * nmax) + a16(16 * fmax) + a16(4 * mask_words) + 32 * 16;
  return a16(16 * nmax) + a16(8 * nmax) + a16(16 * fmax) + a16(8 * fmax) + a16(4 * mask_words) + a16(2 * emax) +
         16 * rmax + 32 * 16;
}

// Atoms of a rotamer's rotating fragment in a ligand of n atoms.
__host__ __device__ inline int frag_atoms(int n, const RotDesc& d) {
  const int sub = (int)d.hi - (int)d.lo;
  return d.comp ? n - sub : sub;
}

enum : int { ERR_NONE = 0, ERR_STAGE_TIMEOUT = 1, ERR_SLOT_TIMEOUT = 2 };

// Items per work-queue grab: 4 once there are at least 8 per warp a full GPU holds
// (148 SMs x 32 warps), so chunking never idles warps on small batches.
inline int work_chunk(long long n_items) { return n_items >= 8LL * 148 * 32 ? 4 : 1; }

// pose_score of a restart that a subset launch leaves out (buffers are filled with it)
constexpr uint32_t NOT_SEARCHED = 0xFFFFFFFFu;

// Builds of the search kernel.
//   BUILD_WIDE:    <= 128 registers, one block of up to 16 warps per SM; the pocket grid
//                  is staged in shared memory when its crop fits; the reach filter prunes
//                  its static columns first.
//   BUILD_LEAN:    <= 80 registers (a little state spills) for up to 24 warps per SM; the
//                  grid is read through the texture path; no column pruning.
//   BUILD_COMPACT: <= 96 registers and smaller per-warp buffers (compact warp_smem_bytes)
//                  for about 20 warps per SM with the buffers of 250-atom ligands; texture
//                  path; column pruning.
enum : int { BUILD_WIDE = 0, BUILD_LEAN = 1, BUILD_COMPACT = 2 };

// Launch configuration of one tile.
struct Tile {
  int warps;        // warps (poses in flight) per block
  int slots;        // angles per lane evaluated together
  int build;        // BUILD_*
};
int tile_count();
Tile tile_get(int id);  // id in [1, tile_count()]

// Launch shape of the search kernel for one tile (kernel attributes and occupancy are
// queried here, outside any stream capture).
struct LaunchCfg {
  const void* fn = nullptr;
  unsigned blocks = 0, threads = 0;
  size_t smem = 0;
};
cudaError_t plan_search(const SearchArgs& a, int tile, bool grid_in_smem, int num_sms, LaunchCfg* cfg);
// The proposer's 48 features of every (ligand, restart) of a packed batch, rows
// li * O + o, as BF16 (Xb) and/or FP32 (Xf).
cudaError_t launch_features(const SearchArgs& a, __nv_bfloat16* Xb, float* Xf, int num_sms, cudaStream_t stream);
// Restart selection from predicted scores [L x O]: per ligand the top k, or the top kf
// (all O when kf >= O) when the top-k spread is below (rule 0) / above (rule 1) margin,
// written as an item list in queue order.
cudaError_t launch_selection(const SearchArgs& a, const float* pred, int k, int kf, float margin, int rule,
                             int32_t* cnt, uint16_t* topk, float* spread, int32_t* off, uint32_t* items,
                             int32_t* n_items, cudaStream_t stream);
// Launch the search: the pose-setup kernel (which also zeroes the work counter and the
// per-ligand completion counters) and the search kernel, on `stream`.
cudaError_t launch_search(const SearchArgs& a, const LaunchCfg& cfg, cudaStream_t stream);
// The streaming server's persistent launch (every SM full; lean and wide builds only) and
// the restart tables it reads (pose-setup kernel without ligands; a.work is written).
cudaError_t plan_serve(const SearchArgs& a, int tile, bool grid_in_smem, int num_sms, LaunchCfg* cfg);
cudaError_t launch_serve(const SearchArgs& a, const ServeArgs& sv, const LaunchCfg& cfg, cudaStream_t stream);
cudaError_t launch_restart_tables(const SearchArgs& a, cudaStream_t stream);
size_t search_smem_bytes(const SearchArgs& a, int tile, bool grid_in_smem);
int max_smem_grid_bytes();
// Tile used for tile 0 (the built-in default) given the batch's buffer sizes.
int default_tile(const SearchArgs& a);
// Register budget per thread of a tile's kernel.
inline int tile_max_regs(const Tile& t) {
  return t.build == BUILD_LEAN ? 80 : (t.build == BUILD_COMPACT ? 96 : 128);
}
// Whether a tile's kernel can stage the pocket grid in shared memory.
inline bool tile_stages_grid(const Tile& t) { return t.build == BUILD_WIDE; }

}  // namespace gd
