// gd_dock_batch_noalloc: docking without any memory allocation at call time.
//
// Who needs it: callers that cannot allocate device memory when they dock -- a
// process whose device memory is already fully reserved by another framework's
// caching allocator, a service that forbids allocation after start-up so its memory
// use stays fixed, or code that must not call cudaMalloc/cudaFree because those calls
// synchronise the device.  gd_dock_batch allocates (cached) device and pinned memory
// per job; this entry point instead keeps everything -- the pocket grid, the packed
// ligands, the results and the search kernel's scratch (per-restart scores, picks and
// counters) -- in one file-scope __device__ array of fixed size, and packs ligands with
// fixed-size arrays on the stack.  It runs the same search kernel, so its results are
// those of gd_dock_batch.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "geodock.h"
#include "gd_internal.h"
#include "gd_pack.h"

using gd::RotDesc;

namespace {

constexpr size_t kBytes = (size_t)GD_NOALLOC_MAX_BYTES;

// Device working memory of every call; each GPU that loads the library holds it
// until the process exits.
static __device__ __align__(256) unsigned char g_dev[kBytes];
// Host staging of the packed inputs (pageable, part of the library image).
static unsigned char g_stage[kBytes];

constexpr int kMaxDevices = 64;
static unsigned char* g_dev_addr[kMaxDevices];  // device address of g_dev, per device
static int g_num_sms[kMaxDevices];
static std::mutex g_setup_mu;

// Reason of the current call's failure, copied to the caller's buffer on return.
thread_local char g_msg[512];

gd_status nfail(gd_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof g_msg, fmt, ap);
  va_end(ap);
  return s;
}

gd_status dock_noalloc(const uint8_t* grid, int nx, int ny, int nz, float spacing, const float origin[3],
                       const gd_ligand_batch* b, const gd_search_params* p, gd_result_batch* out, void* stream);

size_t a256(size_t v) { return (v + 255) / 256 * 256; }

// Device address of g_dev on the current device (taken once per device).
gd_status setup_device(int dev, unsigned char** base, int* sms) {
  if (dev < 0 || dev >= kMaxDevices) return nfail(GD_EINVAL, "device %d not supported here", dev);
  std::lock_guard<std::mutex> g(g_setup_mu);
  if (!g_dev_addr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_dev);
    if (e != cudaSuccess) return nfail(GD_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    e = cudaDeviceGetAttribute(&g_num_sms[dev], cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return nfail(GD_ECUDA, "device attribute: %s", cudaGetErrorString(e));
    g_dev_addr[dev] = (unsigned char*)ptr;
  }
  *base = g_dev_addr[dev];
  *sms = g_num_sms[dev];
  return GD_OK;
}

}  // namespace

extern "C" gd_status gd_dock_batch_noalloc(const uint8_t* grid, int nx, int ny, int nz, float spacing,
                                           const float origin[3], const gd_ligand_batch* b,
                                           const gd_search_params* p, gd_result_batch* out, void* stream,
                                           char* err_msg, size_t err_len) {
  g_msg[0] = 0;
  const gd_status st = dock_noalloc(grid, nx, ny, nz, spacing, origin, b, p, out, stream);
  if (err_msg && err_len) {
    strncpy(err_msg, g_msg, err_len - 1);
    err_msg[err_len - 1] = 0;
  }
  return st;
}

namespace {

gd_status dock_noalloc(const uint8_t* grid, int nx, int ny, int nz, float spacing, const float origin[3],
                       const gd_ligand_batch* b, const gd_search_params* p, gd_result_batch* out, void* stream) {
  if (!grid || !origin || !b || !p || !out) return nfail(GD_EINVAL, "NULL argument");
  if (nx < 1 || ny < 1 || nz < 1 || (long long)nx * ny * nz > (1ll << 31))
    return nfail(GD_EINVAL, "grid dims %d x %d x %d", nx, ny, nz);
  if (!(spacing > 0.f) || !std::isfinite(spacing)) return nfail(GD_EINVAL, "spacing must be > 0");
  {
    const gd_status st = gd::check_params_fixed(nfail, p);
    if (st) return st;
  }
  if (p->flags & (GD_FLAG_DEBUG | GD_FLAG_DEBUG_BUMPS))
    return nfail(GD_EINVAL, "debug outputs are not available without allocation");
  if (p->flags & GD_FLAG_TEST_STAGE_TIMEOUT) return nfail(GD_EINVAL, "test flags are not accepted here");
  if (out->orient_score || out->orient_pick || out->bump_bits)
    return nfail(GD_EINVAL, "debug outputs are not available without allocation");
  if (p->tile == -1) return nfail(GD_EINVAL, "tile -1 (autotuned) needs a context; pass 0 (default) or a tile id");
  if (p->rigid_span != 0) return nfail(GD_EINVAL, "the rigid alignment sweep is not available without allocation");
  const int L = b->n_ligands;
  if (L < 0) return nfail(GD_EINVAL, "n_ligands < 0");
  if (L == 0) return GD_OK;
  if (!b->atom_off || !b->xyz || !b->bond_off || !b->bonds || !b->rot_off || !b->rot_bond)
    return nfail(GD_EINVAL, "batch has a NULL array");
  if (b->atom_off[0] != 0 || b->bond_off[0] != 0 || b->rot_off[0] != 0)
    return nfail(GD_EINVAL, "CSR offsets must start at 0");
  for (int i = 0; i < L; ++i)
    if (b->atom_off[i + 1] < b->atom_off[i] || b->bond_off[i + 1] < b->bond_off[i] || b->rot_off[i + 1] < b->rot_off[i])
      return nfail(GD_EINVAL, "CSR offsets decrease at ligand %d", i);
  const long long N = b->atom_off[L], Rt = b->rot_off[L];
  const int O = p->n_alpha * p->n_beta * p->n_gamma, reps = p->repetitions, A = p->n_angles;

  // pocket crop: bounding box of non-zero cells (cells outside score 0), as gd_load_pocket
  int lo[3] = {nx, ny, nz}, hi[3] = {-1, -1, -1};
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i)
        if (grid[((size_t)k * ny + j) * nx + i]) {
          if (i < lo[0]) lo[0] = i;
          if (i > hi[0]) hi[0] = i;
          if (j < lo[1]) lo[1] = j;
          if (j > hi[1]) hi[1] = j;
          if (k < lo[2]) lo[2] = k;
          if (k > hi[2]) hi[2] = k;
        }
  if (hi[0] < 0) lo[0] = lo[1] = lo[2] = hi[0] = hi[1] = hi[2] = 0;
  const int cx = hi[0] - lo[0] + 1, cy = hi[1] - lo[1] + 1, cz = hi[2] - lo[2] + 1;
  const size_t grid_pad = ((size_t)cx * cy * cz + 15) / 16 * 16;

  // one layout for the fixed array: grid | inputs | outputs | scratch
  size_t o = 0;
  const size_t o_grid = o;       o = a256(o + grid_pad);
  const size_t o_atom_off = o;   o = a256(o + 4 * (size_t)(L + 1));
  const size_t o_rot_off = o;    o = a256(o + 4 * (size_t)(L + 1));
  const size_t o_xyz = o;        o = a256(o + 16 * (size_t)N);
  const size_t o_perm = o;       o = a256(o + (size_t)N);
  const size_t o_rots = o;       o = a256(o + sizeof(RotDesc) * (size_t)Rt);
  const size_t o_order = o;      o = a256(o + 4 * (size_t)L);
  const size_t o_excl = o;       o = a256(o + 2 * (size_t)Rt * GD_MAX_EXCLUDED);
  const size_t o_score = o;      o = a256(o + 4 * (size_t)L);
  const size_t o_orient = o;     o = a256(o + 4 * (size_t)L);
  const size_t o_angle = o;      o = a256(o + 2 * (size_t)Rt * reps);
  const size_t o_bxyz = o;       o = a256(o + 12 * (size_t)N);
  const size_t o_evals = o;      o = a256(o + 8 * (size_t)L);
  const size_t o_pairs = o;      o = a256(o + 8 * (size_t)L);
  const size_t o_moves = o;      o = a256(o + 8 * (size_t)L);
  const size_t o_reach = o;      o = a256(o + 8 * (size_t)L);
  const size_t o_err = o;        o = a256(o + 4);
  const size_t o_pscore = o;     o = a256(o + 4 * (size_t)L * O);
  const size_t o_ppick = o;      o = a256(o + 2 * (size_t)O * reps * Rt);
  const size_t o_ppairs = o;     o = a256(o + 8 * (size_t)L * O);
  const size_t o_preach = o;     o = a256(o + 8 * (size_t)L * O);
  const size_t o_xc = o;         o = a256(o + 16 * (size_t)N);
  const size_t o_rmat = o;       o = a256(o + 36 * (size_t)O);
  const size_t o_quat = o;       o = a256(o + 16 * (size_t)O);
  const size_t o_done = o;       o = o + 4 * (size_t)L;
  o = (o + 7) / 8 * 8;
  const size_t o_work = o;       o = a256(o + 8);
  if (o > kBytes)
    return nfail(GD_EINVAL, "batch needs %zu bytes of working memory, more than the fixed %zu bytes", o, kBytes);

  // host packing into the fixed staging array
  unsigned char* h = g_stage;
  for (int k = 0; k < cz; ++k)
    for (int j = 0; j < cy; ++j)
      memcpy(h + o_grid + ((size_t)k * cy + j) * cx, &grid[((size_t)(k + lo[2]) * ny + (j + lo[1])) * nx + lo[0]], cx);
  memset(h + o_grid + (size_t)cx * cy * cz, 0, grid_pad - (size_t)cx * cy * cz);
  int32_t* atom_off = (int32_t*)(h + o_atom_off);
  int32_t* rot_off = (int32_t*)(h + o_rot_off);
  int32_t* order = (int32_t*)(h + o_order);
  size_t n_excl = 0;
  int nmax = 2;
  for (int i = 0; i < L; ++i) {
    const int a0 = b->atom_off[i], n = b->atom_off[i + 1] - a0;
    const int b0 = b->bond_off[i], nb = b->bond_off[i + 1] - b0;
    const int r0 = b->rot_off[i], R = b->rot_off[i + 1] - r0;
    gd_status st = gd::pack_ligand_fixed(nfail, i, n, b->xyz + 3 * (size_t)a0, nb, b->bonds + 2 * (size_t)b0, R,
                                         b->rot_bond + r0, p->min_bond_sep, (float4*)(h + o_xyz) + a0,
                                         h + o_perm + a0, (RotDesc*)(h + o_rots) + r0, (uint16_t*)(h + o_excl),
                                         (size_t)Rt * GD_MAX_EXCLUDED, &n_excl, nullptr);
    if (st) return st;
    if (R * reps > 32767) return nfail(GD_EINVAL, "ligand %d: too many steps", i);
    if (n > nmax) nmax = n;
    order[i] = i;  // queue order only affects scheduling, never results
  }
  for (int i = 0; i <= L; ++i) {
    atom_off[i] = b->atom_off[i];
    rot_off[i] = b->rot_off[i];
  }

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return nfail(GD_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  unsigned char* d = nullptr;
  int sms = 0;
  gd_status st = setup_device(dev, &d, &sms);
  if (st) return st;

  gd::SearchArgs a{};
  a.pk.grid = d + o_grid;
  a.pk.cx = cx;
  a.pk.cy = cy;
  a.pk.cz = cz;
  a.pk.bytes_pad = (int)grid_pad;
  a.pk.inv_h = (float)(1.0 / (double)spacing);
  a.pk.h = spacing;
  const int nn[3] = {nx, ny, nz};
  for (int k = 0; k < 3; ++k) {
    a.pk.shift[k] = (float)(0.5 * nn[k] - lo[k]);
    a.pk.centre[k] = (float)((double)origin[k] + 0.5 * (double)spacing * nn[k]);
  }
  a.L = L;
  a.atom_off = (const int32_t*)(d + o_atom_off);
  a.rot_off = (const int32_t*)(d + o_rot_off);
  a.xyz = (const float4*)(d + o_xyz);
  a.perm = d + o_perm;
  a.rots = (const RotDesc*)(d + o_rots);
  a.excl = (const uint16_t*)(d + o_excl);
  a.order = (const int32_t*)(d + o_order);
  a.n_items = (long long)L * O;
  a.chunk = gd::work_chunk(a.n_items);
  a.na = p->n_alpha;
  a.nb = p->n_beta;
  a.ng = p->n_gamma;
  a.O = O;
  a.A = A;
  a.reps = reps;
  {
    const float ih = a.pk.inv_h, bd = p->bump_dist * ih, rd = (p->bump_dist + gd::REACH_MARGIN) * ih;
    a.thr2 = bd * bd;
    a.reach2 = rd * rd;
  }
  a.use_filter = (p->flags & GD_FLAG_NO_FILTER) ? 0 : 1;
  a.mask_sweep = (p->flags & GD_FLAG_MASK_SWEEP) ? 1 : 0;
  a.stage_extra_bytes = 0;
  a.best_score = (uint32_t*)(d + o_score);
  a.best_orient = (int32_t*)(d + o_orient);
  a.best_angle = (int16_t*)(d + o_angle);
  a.best_xyz = (float*)(d + o_bxyz);
  a.evals = (unsigned long long*)(d + o_evals);
  a.pair_tests = (unsigned long long*)(d + o_pairs);
  a.atom_moves = (unsigned long long*)(d + o_moves);
  a.reach_tests = (unsigned long long*)(d + o_reach);
  a.err = (int32_t*)(d + o_err);
  a.pose_score = (uint32_t*)(d + o_pscore);
  a.pose_pick = (int16_t*)(d + o_ppick);
  a.pose_pairs = (unsigned long long*)(d + o_ppairs);
  a.pose_reach = (unsigned long long*)(d + o_preach);
  a.xc = (float4*)(d + o_xc);
  a.rmat = (float*)(d + o_rmat);
  a.quat = (float4*)(d + o_quat);
  a.done = (int32_t*)(d + o_done);
  a.work = (unsigned long long*)(d + o_work);
  a.bump_bits = nullptr;
  a.nmax = nmax;
  a.mask_words = 1;
  a.fmax = 1;
  a.rmax = 1;
  a.emax = 1;
  for (int i = 0; i < L; ++i) {
    int ne = 0;
    const RotDesc* rr = (const RotDesc*)(h + o_rots);
    const int n = b->atom_off[i + 1] - b->atom_off[i];
    for (int r = rot_off[i]; r < rot_off[i + 1]; ++r) {
      ne += rr[r].n_excl;
      const int mw = gd::step_mask_words(n, rr[r]);
      a.mask_words = mw > a.mask_words ? mw : a.mask_words;
      const int fa = gd::frag_atoms(n, rr[r]);
      a.fmax = fa > a.fmax ? fa : a.fmax;
    }
    a.rmax = rot_off[i + 1] - rot_off[i] > a.rmax ? rot_off[i + 1] - rot_off[i] : a.rmax;
    a.emax = ne > a.emax ? ne : a.emax;
  }

  const int tile = p->tile > 0 ? p->tile : gd::default_tile(a);
  const size_t smem_cap = 227 * 1024;
  bool smem_grid = gd::tile_stages_grid(gd::tile_get(tile)) && (int)grid_pad <= gd::max_smem_grid_bytes() &&
                   gd::search_smem_bytes(a, tile, true) <= smem_cap;
  if (!smem_grid && gd::search_smem_bytes(a, tile, false) > smem_cap)
    return nfail(GD_EINVAL, "tile %d needs more shared memory than a block has", tile);
  gd::LaunchCfg cfg;
  e = gd::plan_search(a, tile, smem_grid, sms, &cfg);
  if (e != cudaSuccess) return nfail(GD_ECUDA, "search launch shape: %s", cudaGetErrorString(e));

  cudaStream_t s = (cudaStream_t)stream;
  const size_t in_used = o_excl + 2 * n_excl;
  int32_t err = 0;
  if ((e = cudaMemcpyAsync(d, g_stage, in_used, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(d + o_err, 0, 4, s)) != cudaSuccess ||
      (e = gd::launch_search(a, cfg, s)) != cudaSuccess)
    return nfail(GD_ECUDA, "launch: %s", cudaGetErrorString(e));
  struct Copy {
    void* dst;
    size_t off, bytes;
  } copies[] = {{out->best_score, o_score, 4 * (size_t)L},   {out->best_orient, o_orient, 4 * (size_t)L},
                {out->best_angle, o_angle, 2 * (size_t)Rt * reps}, {out->best_xyz, o_bxyz, 12 * (size_t)N},
                {out->evals, o_evals, 8 * (size_t)L},        {out->pair_tests, o_pairs, 8 * (size_t)L},
                {out->atom_moves, o_moves, 8 * (size_t)L},   {out->reach_tests, o_reach, 8 * (size_t)L},
                {&err, o_err, 4}};
  for (auto& c : copies)
    if (c.dst && c.bytes && (e = cudaMemcpyAsync(c.dst, d + c.off, c.bytes, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return nfail(GD_ECUDA, "result copy: %s", cudaGetErrorString(e));
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return nfail(GD_ECUDA, "search: %s", cudaGetErrorString(e));
  if (err == gd::ERR_STAGE_TIMEOUT) return nfail(GD_ETIMEOUT, "pocket staging wait timed out on the device");
  return GD_OK;
}

}  // namespace
