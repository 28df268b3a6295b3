// Host runtime of libgeodock: contexts, pockets, batch validation and packing, job
// memory, CUDA-graph launch and the launch-tile autotuner.  Implements include/geodock.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <condition_variable>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "geodock.h"
#include "geodock_mlp.h"
#include "gd_internal.h"
#include "gd_pack.h"
#include "gd_peak.h"

// The search kernel packs atom ids into bytes (near pairs, the reach filter's column
// lists, which share the 512-byte coefficient buffer of a warp).
static_assert(GD_MAX_ATOMS <= 256, "atom ids must fit a byte");

using gd::RotDesc;
using gd::SearchArgs;


namespace {

thread_local std::string g_err;

gd_status fail(gd_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define GD_CUDA(call)                                                                       \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return fail(GD_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

// ---------------------------------------------------------------- context & memory

namespace {

// Host threads that pack batches, started once with the context (starting threads per
// batch cost more than packing a small batch).  run(T, fn) calls fn(0 .. T-1) on the
// caller and the workers and returns when all calls have returned; calls to run are
// serialised.
class HostPool {
 public:
  explicit HostPool(int workers) {
    for (int i = 0; i < workers; ++i) th_.emplace_back([this] { loop(); });
  }
  ~HostPool() {
    {
      std::lock_guard<std::mutex> g(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto& t : th_) t.join();
  }
  int threads() const { return (int)th_.size() + 1; }
  void run(int T, const std::function<void(int)>& fn) {
    std::lock_guard<std::mutex> serial(run_mu_);
    {
      std::lock_guard<std::mutex> g(mu_);
      fn_ = &fn;
      next_ = 1;
      T_ = T;
      pending_ = T - 1;
      ++gen_;
    }
    if (T > 1) cv_.notify_all();
    fn(0);
    std::unique_lock<std::mutex> lk(mu_);
    done_.wait(lk, [&] { return pending_ == 0; });
    fn_ = nullptr;
  }

 private:
  void loop() {
    uint64_t seen = 0;
    std::unique_lock<std::mutex> lk(mu_);
    for (;;) {
      cv_.wait(lk, [&] { return stop_ || gen_ != seen; });
      if (stop_) return;
      seen = gen_;
      while (next_ < T_) {
        const int t = next_++;
        const std::function<void(int)>* fn = fn_;
        lk.unlock();
        (*fn)(t);
        lk.lock();
        if (--pending_ == 0) done_.notify_all();
      }
    }
  }
  std::vector<std::thread> th_;
  std::mutex mu_, run_mu_;
  std::condition_variable cv_, done_;
  const std::function<void(int)>* fn_ = nullptr;
  int next_ = 0, T_ = 0, pending_ = 0;
  uint64_t gen_ = 0;
  bool stop_ = false;
};

// Packing threads (the caller included): the host's hardware threads, 1 to 16.  Packing
// is compute-bound (about 2-7 us per ligand and thread, depending on the host), and on a
// 16-thread host 16 packers beat 8 by 1.3-1.4x even with the caller's other threads
// running.
int pack_threads() { return std::max(1, std::min(16, (int)std::thread::hardware_concurrency())); }

}  // namespace

struct gd_ctx {
  int device = 0;
  int num_sms = 0;
  size_t budget = 0;  // 0: unlimited
  size_t used = 0;    // device bytes currently held (cached blocks included)
  cudaStream_t capture_stream = nullptr;
  std::mutex capture_mu;  // one graph capture at a time on capture_stream
  std::mutex mu;
  std::multimap<size_t, void*> dev_free;   // cached device blocks by size
  std::multimap<size_t, void*> host_free;  // cached pinned blocks by size
  std::unordered_map<void*, size_t> dev_size, host_size;  // size of every block allocated
  std::map<std::string, int> tuned;        // autotuned tile per workload signature
  std::vector<cudaEvent_t> events;         // completion events of released jobs, for reuse
  HostPool pool{pack_threads() - 1};        // batch packing
};

namespace {

// Blocks are rounded to 1 MiB (or a power of two below); a request takes the smallest
// cached block of at least its size and at most twice it, so jobs of similar shapes
// (a stream of batches of varying size) reuse blocks instead of allocating.
size_t size_class(size_t b) {
  if (b <= (1u << 20)) {
    size_t s = 4096;
    while (s < b) s <<= 1;
    return s;
  }
  return align_up(b, 1u << 20);
}

gd_status dev_alloc(gd_ctx* c, size_t bytes, void** out) {
  const size_t sz = size_class(bytes);
  {
    std::lock_guard<std::mutex> g(c->mu);
    auto it = c->dev_free.lower_bound(sz);
    if (it != c->dev_free.end() && it->first <= 2 * sz) {
      *out = it->second;
      c->dev_free.erase(it);
      return GD_OK;
    }
  }
  if (c->budget && c->used + sz > c->budget) {
    // drop cached blocks before refusing
    std::lock_guard<std::mutex> g(c->mu);
    for (auto& kv : c->dev_free) {
      cudaFree(kv.second);
      c->used -= kv.first;
      c->dev_size.erase(kv.second);
    }
    c->dev_free.clear();
    if (c->used + sz > c->budget)
      return fail(GD_EBUDGET, "device budget %zu B exceeded (held %zu B, need %zu B)", c->budget, c->used, sz);
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, sz);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(GD_ENOMEM, "cudaMalloc(%zu): %s", sz, cudaGetErrorString(e));
  }
  std::lock_guard<std::mutex> g(c->mu);
  c->used += sz;
  c->dev_size[p] = sz;
  *out = p;
  return GD_OK;
}

void dev_release(gd_ctx* c, void* p, size_t bytes) {
  if (!p) return;
  std::lock_guard<std::mutex> g(c->mu);
  auto it = c->dev_size.find(p);
  c->dev_free.emplace(it != c->dev_size.end() ? it->second : size_class(bytes), p);
}

gd_status host_alloc(gd_ctx* c, size_t bytes, void** out) {
  const size_t sz = size_class(bytes);
  {
    std::lock_guard<std::mutex> g(c->mu);
    auto it = c->host_free.lower_bound(sz);
    if (it != c->host_free.end() && it->first <= 2 * sz) {
      *out = it->second;
      c->host_free.erase(it);
      return GD_OK;
    }
  }
  void* p = nullptr;
  cudaError_t e = cudaMallocHost(&p, sz);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(GD_ENOMEM, "cudaMallocHost(%zu): %s", sz, cudaGetErrorString(e));
  }
  std::lock_guard<std::mutex> g(c->mu);
  c->host_size[p] = sz;
  *out = p;
  return GD_OK;
}

void host_release(gd_ctx* c, void* p, size_t bytes) {
  if (!p) return;
  std::lock_guard<std::mutex> g(c->mu);
  auto it = c->host_size.find(p);
  c->host_free.emplace(it != c->host_size.end() ? it->second : size_class(bytes), p);
}

}  // namespace

struct gd_pocket {
  gd::PocketDev dev{};
  void* buf = nullptr;
  size_t buf_bytes = 0;
  cudaArray_t arr = nullptr;  // the crop again as a 3D array, behind dev.tex
  size_t arr_bytes = 0;
  int nx = 0, ny = 0, nz = 0;
};

// ---------------------------------------------------------------- batch packing

namespace {

// Byte layout of a packed batch; the same offsets are used in pinned staging and in
// device memory so one copy moves the whole input.
struct InLayout {
  size_t atom_off, rot_off, xyz, perm, rots, order, excl, total;
};

InLayout in_layout(int L, long long N, long long Rt, long long n_excl) {
  InLayout l{};
  size_t o = 0;
  l.atom_off = o; o = align_up(o + 4 * (size_t)(L + 1), 256);
  l.rot_off = o;  o = align_up(o + 4 * (size_t)(L + 1), 256);
  l.xyz = o;      o = align_up(o + 16 * (size_t)N, 256);
  l.perm = o;     o = align_up(o + (size_t)N, 256);
  l.rots = o;     o = align_up(o + sizeof(RotDesc) * (size_t)Rt, 256);
  l.order = o;    o = align_up(o + 4 * (size_t)L, 256);
  l.excl = o;     o = align_up(o + 2 * (size_t)n_excl, 256);
  l.total = o;
  return l;
}

struct OutLayout {
  size_t best_score, best_orient, best_angle, best_xyz, evals, pair_tests, atom_moves, reach_tests, best_rigid, err,
      total;
};

OutLayout out_layout(int L, long long N, long long Rt, int reps) {
  OutLayout l{};
  size_t o = 0;
  l.best_score = o;  o = align_up(o + 4 * (size_t)L, 256);
  l.best_orient = o; o = align_up(o + 4 * (size_t)L, 256);
  l.best_angle = o;  o = align_up(o + 2 * (size_t)Rt * reps, 256);
  l.best_xyz = o;    o = align_up(o + 12 * (size_t)N, 256);
  l.evals = o;       o = align_up(o + 8 * (size_t)L, 256);
  l.pair_tests = o;  o = align_up(o + 8 * (size_t)L, 256);
  l.atom_moves = o;  o = align_up(o + 8 * (size_t)L, 256);
  l.reach_tests = o; o = align_up(o + 8 * (size_t)L, 256);
  l.best_rigid = o;  o = align_up(o + 2 * (size_t)L, 256);
  l.err = o;         o = align_up(o + 4, 256);
  l.total = o;
  return l;
}

struct ScratchLayout {
  size_t pose_score, pose_pick, pose_pairs, pose_reach, pose_rigid, xc, rmat, quat, done, work, bump, total;
};

ScratchLayout scratch_layout(int L, int O, long long N, long long Rt, int reps, int A, bool debug) {
  ScratchLayout l{};
  size_t o = 0;
  l.xc = o;         o = align_up(o + 16 * (size_t)N, 256);
  l.rmat = o;       o = align_up(o + 36 * (size_t)O, 256);
  l.quat = o;       o = align_up(o + 16 * (size_t)O, 256);
  l.pose_score = o; o = align_up(o + 4 * (size_t)L * O, 256);
  l.pose_pick = o;  o = align_up(o + 2 * (size_t)O * reps * Rt, 256);
  l.pose_pairs = o; o = align_up(o + 8 * (size_t)L * O, 256);
  l.pose_reach = o; o = align_up(o + 8 * (size_t)L * O, 256);
  l.pose_rigid = o; o = align_up(o + 2 * (size_t)L * O, 256);
  l.done = o;       o = o + 4 * (size_t)L;          // done and work are cleared by one memset
  o = align_up(o, 8);
  l.work = o;       o = align_up(o + 8, 256);
  l.bump = o;       o = align_up(o + (debug ? (size_t)O * reps * A * Rt : 0), 256);
  l.total = o;
  return l;
}

gd_status check_params(const gd_search_params* p) { return gd::check_params_fixed(fail, p); }

// Validate one ligand and write its preorder-packed atoms and rotamer descriptors
// (gd::pack_ligand_fixed), appending its excluded pairs to excl.
// cost: an estimate of its search work, used to order the work queue.
gd_status pack_ligand(int li, int n, const float* xyz, int nb, const int32_t* bonds, int R,
                      const int32_t* rot_bond, int min_sep, float4* out_xyz, uint8_t* out_perm,
                      RotDesc* out_rots, std::vector<uint16_t>& excl, double* cost) {
  const size_t old = excl.size();
  excl.resize(old + (size_t)std::min(std::max(R, 0), GD_MAX_ROTAMERS) * GD_MAX_EXCLUDED);
  size_t used = old;
  const gd_status st = gd::pack_ligand_fixed(fail, li, n, xyz, nb, bonds, R, rot_bond, min_sep, out_xyz, out_perm,
                                             out_rots, excl.data(), excl.size(), &used, cost);
  excl.resize(st ? old : used);
  return st;
}

}  // namespace

// ---------------------------------------------------------------- jobs

struct gd_job {
  gd_ctx* ctx = nullptr;
  int L = 0, O = 0, reps = 0, A = 0;
  long long N = 0, Rt = 0;
  bool debug = false;
  bool debug_bumps = false;
  bool grid_in_smem = false;
  int tile = 1;
  InLayout in{};
  OutLayout out{};
  ScratchLayout scr{};
  void* d_in = nullptr;
  void* d_out = nullptr;
  void* d_scr = nullptr;
  void* h_in = nullptr;
  size_t h_in_cap = 0;
  void* h_out = nullptr;
  void* h_dbg = nullptr;  // pose_score | pose_pick | bump (debug only)
  size_t dbg_bytes = 0;
  SearchArgs args{};
  gd::LaunchCfg cfg{};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;  // built at the job's second launch
  int launches = 0;                // searches enqueued so far
  // restart selection of the learned proposer (allocated on first use)
  void* d_sel = nullptr;
  size_t sel_bytes = 0;
  int32_t *sel_cnt = nullptr, *sel_off = nullptr, *sel_n = nullptr;
  uint16_t* sel_topk = nullptr;
  float* sel_spread = nullptr;
  uint32_t* sel_items = nullptr;
  cudaEvent_t done = nullptr;
  std::vector<int32_t> rot_off;  // host copy for result layout checks
};

namespace {

gd_status job_release(gd_ctx* c, gd_job* j) {
  if (j->done) cudaEventSynchronize(j->done);
  if (j->exec) cudaGraphExecDestroy(j->exec);
  if (j->graph) cudaGraphDestroy(j->graph);
  if (j->done) {  // completed (synchronised above): kept for the context's next job
    std::lock_guard<std::mutex> g(c->mu);
    c->events.push_back(j->done);
  }
  dev_release(c, j->d_in, j->in.total);
  dev_release(c, j->d_out, j->out.total);
  dev_release(c, j->d_scr, j->scr.total);
  dev_release(c, j->d_sel, j->sel_bytes);
  host_release(c, j->h_in, j->h_in_cap);
  host_release(c, j->h_out, j->out.total);
  host_release(c, j->h_dbg, j->dbg_bytes);
  delete j;
  return GD_OK;
}

std::string signature(const gd_pocket* pk, const gd_search_params* p, int nmax, bool smem) {
  char b[256];
  snprintf(b, sizeof b, "O%d_A%d_r%d_n%d_g%d_%dx%dx%d_f%d_s%d", p->n_alpha * p->n_beta * p->n_gamma, p->n_angles,
           p->repetitions, (nmax + 31) / 32, smem ? 1 : 0, pk->dev.cx, pk->dev.cy, pk->dev.cz,
           (p->flags & GD_FLAG_NO_FILTER) ? 0 : ((p->flags & GD_FLAG_MASK_SWEEP) ? 2 : 1), p->rigid_span);
  return b;
}

// Capture [pose setup (which also clears the search's counters), search kernel] once;
// replayed by every later launch of the job.  A job's first launch goes to the stream directly (capturing and instantiating a
// graph costs more host time than a single launch of a small job saves).
gd_status build_graph(gd_ctx* c, gd_job* j) {
  std::lock_guard<std::mutex> serial(c->capture_mu);  // host threads share the capture stream
  cudaStream_t s = c->capture_stream;
  GD_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  cudaError_t le = gd::launch_search(j->args, j->cfg, s);
  cudaGraph_t g = nullptr;
  cudaError_t ee = cudaStreamEndCapture(s, &g);
  if (le != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return fail(GD_ECUDA, "search launch: %s", cudaGetErrorString(le));
  }
  if (ee != cudaSuccess) return fail(GD_ECUDA, "graph capture: %s", cudaGetErrorString(ee));
  j->graph = g;
  GD_CUDA(cudaGraphInstantiate(&j->exec, g, 0));
  return GD_OK;
}

// The job's ligand i is batch ligand sel[i] (sel = NULL: ligand i, L = n_ligands); its
// atoms and rotamers are packed contiguously in that order.
gd_status make_job(gd_ctx* c, const gd_pocket* pk, const gd_ligand_batch* b, const int32_t* sel, int n_sel,
                   const gd_search_params* p, int tile, gd_job** out) {
  const int LB = b->n_ligands;
  if (LB < 0) return fail(GD_EINVAL, "n_ligands < 0");
  if (sel && n_sel < 0) return fail(GD_EINVAL, "n_sel < 0");
  const int L = sel ? n_sel : LB;
  if (LB > 0 && (!b->atom_off || !b->xyz || !b->bond_off || !b->bonds || !b->rot_off || !b->rot_bond))
    return fail(GD_EINVAL, "batch has a NULL array");
  if (LB > 0 && (b->atom_off[0] != 0 || b->bond_off[0] != 0 || b->rot_off[0] != 0))
    return fail(GD_EINVAL, "CSR offsets must start at 0");
  // destination offsets of the job's ligands (atoms, rotamers)
  std::vector<int32_t> dA(L + 1, 0), dR(L + 1, 0);
  for (int i = 0; i < L; ++i) {
    const int s = sel ? sel[i] : i;
    if (s < 0 || s >= LB) return fail(GD_EINVAL, "sel[%d] = %d outside [0, %d)", i, s, LB);
    if (b->atom_off[s + 1] < b->atom_off[s] || b->bond_off[s + 1] < b->bond_off[s] || b->rot_off[s + 1] < b->rot_off[s])
      return fail(GD_EINVAL, "CSR offsets decrease at ligand %d", s);
    const long long na = (long long)dA[i] + (b->atom_off[s + 1] - b->atom_off[s]);
    const long long nr = (long long)dR[i] + (b->rot_off[s + 1] - b->rot_off[s]);
    if (na > INT32_MAX || nr > INT32_MAX) return fail(GD_EINVAL, "batch too large");
    dA[i + 1] = (int32_t)na;
    dR[i + 1] = (int32_t)nr;
  }
  const long long N = dA[L], Rt = dR[L];
  gd_job* j = new gd_job();
  j->ctx = c;
  j->L = L;
  j->O = p->n_alpha * p->n_beta * p->n_gamma;
  j->reps = p->repetitions;
  j->A = p->n_angles;
  j->N = N;
  j->Rt = Rt;
  j->debug = (p->flags & (GD_FLAG_DEBUG | GD_FLAG_DEBUG_BUMPS)) != 0;
  j->debug_bumps = (p->flags & GD_FLAG_DEBUG_BUMPS) != 0;
  // validate and pack: atoms / permutation / descriptors go straight into pinned
  // staging (their sizes are known); exclusions are gathered first and copied after
  j->in = in_layout(L, N, Rt, 0);
  j->out = out_layout(L, N, Rt, j->reps);
  j->scr = scratch_layout(L, j->O, N, Rt, j->reps, j->A, j->debug_bumps);
  const size_t in_cap = j->in.total + align_up(2 * (size_t)Rt * GD_MAX_EXCLUDED, 256);
  gd_status st;
  if ((st = host_alloc(c, in_cap, &j->h_in))) {
    job_release(c, j);
    return st;
  }
  j->h_in_cap = in_cap;
  if ((st = host_alloc(c, j->out.total, &j->h_out))) {
    job_release(c, j);
    return st;
  }
  char* h = (char*)j->h_in;
  int32_t* atom_off = (int32_t*)(h + j->in.atom_off);
  int32_t* rot_off = (int32_t*)(h + j->in.rot_off);
  float4* xyz = (float4*)(h + j->in.xyz);
  uint8_t* perm = (uint8_t*)(h + j->in.perm);
  RotDesc* rots = (RotDesc*)(h + j->in.rots);
  int32_t* order = (int32_t*)(h + j->in.order);
  // ligands are packed by the context's host threads over contiguous ranges; each keeps its
  // own exclusion list, concatenated afterwards in ligand order
  std::vector<double> cost(L);
  const int T = std::max(1, std::min(c->pool.threads(), L / 64));
  struct Part {
    int l0 = 0, l1 = 0, nmax = 2, bad = -1;
    gd_status st = GD_OK;
    std::string err;
    std::vector<uint16_t> excl;
  };
  std::vector<Part> parts(T);
  auto work = [&](Part& pt) {
    for (int i = pt.l0; i < pt.l1; ++i) {
      const int s = sel ? sel[i] : i;
      const int a0 = b->atom_off[s], n = b->atom_off[s + 1] - a0;
      const int b0 = b->bond_off[s], nb = b->bond_off[s + 1] - b0;
      const int r0 = b->rot_off[s], R = b->rot_off[s + 1] - r0;
      gd_status s2 = pack_ligand(s, n, b->xyz + 3 * (size_t)a0, nb, b->bonds + 2 * (size_t)b0, R, b->rot_bond + r0,
                                 p->min_bond_sep, xyz + dA[i], perm + dA[i], rots + dR[i], pt.excl, &cost[i]);
      if (!s2 && R * j->reps > 32767) s2 = fail(GD_EINVAL, "ligand %d: too many steps", s);
      if (s2) {
        pt.st = s2;
        pt.bad = s;
        pt.err = g_err;  // the message lives in this thread's g_err
        return;
      }
      pt.nmax = std::max(pt.nmax, n);
    }
  };
  for (int t = 0; t < T; ++t) {
    parts[t].l0 = (int)((long long)L * t / T);
    parts[t].l1 = (int)((long long)L * (t + 1) / T);
  }
  c->pool.run(T, [&](int t) { work(parts[t]); });
  int nmax = 2;
  size_t n_excl = 0;
  for (auto& pt : parts) {
    if (pt.st) {
      job_release(c, j);
      g_err = pt.err;
      return pt.st;
    }
    nmax = std::max(nmax, pt.nmax);
    n_excl += pt.excl.size();
  }
  j->in = in_layout(L, N, Rt, (long long)n_excl);
  {
    size_t base = 0;
    for (auto& pt : parts) {
      if (base)
        for (long long r = dR[pt.l0]; r < dR[pt.l1]; ++r) rots[r].excl_off += (uint32_t)base;
      if (!pt.excl.empty()) memcpy(h + j->in.excl + 2 * base, pt.excl.data(), 2 * pt.excl.size());
      base += pt.excl.size();
    }
  }
  memcpy(atom_off, dA.data(), sizeof(int32_t) * (L + 1));
  memcpy(rot_off, dR.data(), sizeof(int32_t) * (L + 1));
  j->rot_off.assign(rot_off, rot_off + L + 1);
  for (int i = 0; i < L; ++i) order[i] = i;
  std::stable_sort(order, order + L, [&](int x, int y) { return cost[x] > cost[y]; });

  if ((st = dev_alloc(c, j->in.total, &j->d_in)) || (st = dev_alloc(c, j->out.total, &j->d_out)) ||
      (st = dev_alloc(c, j->scr.total, &j->d_scr))) {
    job_release(c, j);
    return st;
  }
  if (j->debug) {
    j->dbg_bytes = j->scr.total;
    if ((st = host_alloc(c, j->dbg_bytes, &j->h_dbg))) {
      job_release(c, j);
      return st;
    }
  }
  // kernel arguments
  SearchArgs& a = j->args;
  a.pk = pk->dev;
  a.L = L;
  char* d = (char*)j->d_in;
  a.atom_off = (const int32_t*)(d + j->in.atom_off);
  a.rot_off = (const int32_t*)(d + j->in.rot_off);
  a.xyz = (const float4*)(d + j->in.xyz);
  a.perm = (const uint8_t*)(d + j->in.perm);
  a.rots = (const RotDesc*)(d + j->in.rots);
  a.order = (const int32_t*)(d + j->in.order);
  a.excl = (const uint16_t*)(d + j->in.excl);
  a.n_items = (long long)L * j->O;
  a.chunk = gd::work_chunk(a.n_items);
  a.na = p->n_alpha;
  a.nb = p->n_beta;
  a.ng = p->n_gamma;
  a.O = j->O;
  a.A = j->A;
  a.reps = j->reps;
  {
    const float ih = a.pk.inv_h, bd = p->bump_dist * ih, rd = (p->bump_dist + gd::REACH_MARGIN) * ih;
    a.thr2 = bd * bd;
    a.reach2 = rd * rd;
  }
  a.use_filter = (p->flags & GD_FLAG_NO_FILTER) ? 0 : 1;
  a.mask_sweep = (p->flags & GD_FLAG_MASK_SWEEP) ? 1 : 0;
  a.stage_extra_bytes = (p->flags & GD_FLAG_TEST_STAGE_TIMEOUT) ? 16 : 0;
  char* o = (char*)j->d_out;
  a.best_score = (uint32_t*)(o + j->out.best_score);
  a.best_orient = (int32_t*)(o + j->out.best_orient);
  a.best_angle = (int16_t*)(o + j->out.best_angle);
  a.best_xyz = (float*)(o + j->out.best_xyz);
  a.evals = (unsigned long long*)(o + j->out.evals);
  a.pair_tests = (unsigned long long*)(o + j->out.pair_tests);
  a.atom_moves = (unsigned long long*)(o + j->out.atom_moves);
  a.reach_tests = (unsigned long long*)(o + j->out.reach_tests);
  a.best_rigid = (int16_t*)(o + j->out.best_rigid);
  a.rigid_span = p->rigid_span;
  a.rigid_step = p->rigid_step;
  a.rigid_n = p->rigid_span > 0 ? (2 * p->rigid_span + 1) * (2 * p->rigid_span + 1) * (2 * p->rigid_span + 1) : 0;
  char* s = (char*)j->d_scr;
  a.pose_score = (uint32_t*)(s + j->scr.pose_score);
  a.pose_pick = (int16_t*)(s + j->scr.pose_pick);
  a.pose_pairs = (unsigned long long*)(s + j->scr.pose_pairs);
  a.pose_reach = (unsigned long long*)(s + j->scr.pose_reach);
  a.pose_rigid = (int16_t*)(s + j->scr.pose_rigid);
  a.xc = (float4*)(s + j->scr.xc);
  a.rmat = (float*)(s + j->scr.rmat);
  a.quat = (float4*)(s + j->scr.quat);
  a.done = (int32_t*)(s + j->scr.done);
  a.work = (unsigned long long*)(s + j->scr.work);
  a.err = (int32_t*)(o + j->out.err);
  a.bump_bits = j->debug_bumps ? (uint8_t*)(s + j->scr.bump) : nullptr;
  a.nmax = nmax;
  a.mask_words = 1;
  a.fmax = 1;
  a.rmax = 1;
  a.emax = 1;
  for (int i = 0; i < L; ++i) {
    int ne = 0;
    const int n = dA[i + 1] - dA[i];
    for (int r = rot_off[i]; r < rot_off[i + 1]; ++r) {
      ne += rots[r].n_excl;
      a.mask_words = std::max(a.mask_words, gd::step_mask_words(n, rots[r]));
      a.fmax = std::max(a.fmax, gd::frag_atoms(n, rots[r]));
    }
    a.rmax = std::max(a.rmax, rot_off[i + 1] - rot_off[i]);
    a.emax = std::max(a.emax, ne);
  }
  // tile (0: chosen from the batch's buffer sizes) and grid staging mode
  const size_t smem_cap = 227 * 1024;
  if (tile == 0) tile = gd::default_tile(a);
  j->tile = tile;
  j->grid_in_smem = gd::tile_stages_grid(gd::tile_get(tile)) && pk->dev.bytes_pad <= gd::max_smem_grid_bytes() &&
                    gd::search_smem_bytes(a, tile, true) <= smem_cap;
  if (!j->grid_in_smem && gd::search_smem_bytes(a, tile, false) > smem_cap) {
    job_release(c, j);
    return fail(GD_EINVAL, "tile %d needs more shared memory than a block has", tile);
  }
  {
    std::lock_guard<std::mutex> g(c->mu);
    if (!c->events.empty()) {
      j->done = c->events.back();
      c->events.pop_back();
    }
  }
  if (!j->done) GD_CUDA(cudaEventCreateWithFlags(&j->done, cudaEventDisableTiming));
  if (L > 0) {  // launch shape (kernel attributes and occupancy: queried outside any capture)
    cudaError_t pe = gd::plan_search(j->args, j->tile, j->grid_in_smem, c->num_sms, &j->cfg);
    if (pe != cudaSuccess) {
      job_release(c, j);
      return fail(GD_ECUDA, "search launch shape: %s", cudaGetErrorString(pe));
    }
  }
  *out = j;
  return GD_OK;
}

gd_status enqueue_search(gd_job* j, cudaStream_t s) {
  if (j->L == 0) return GD_OK;
  if (!j->exec && j->launches == 0) {  // first launch: straight to the stream
    GD_CUDA(gd::launch_search(j->args, j->cfg, s));
  } else {  // relaunched: capture once, replay from then on
    if (!j->exec) {
      gd_status st = build_graph(j->ctx, j);
      if (st) return st;
    }
    GD_CUDA(cudaGraphLaunch(j->exec, s));
  }
  ++j->launches;
  GD_CUDA(cudaEventRecord(j->done, s));  // releasing the job waits for this launch
  return GD_OK;
}

gd_status enqueue_download(gd_job* j, cudaStream_t s) {
  GD_CUDA(cudaMemcpyAsync(j->h_out, j->d_out, j->out.total, cudaMemcpyDeviceToHost, s));
  if (j->debug) GD_CUDA(cudaMemcpyAsync(j->h_dbg, j->d_scr, j->dbg_bytes, cudaMemcpyDeviceToHost, s));
  GD_CUDA(cudaEventRecord(j->done, s));
  return GD_OK;
}

}  // namespace

// ---------------------------------------------------------------- C ABI

extern "C" {

const char* gd_last_error(gd_ctx*) { return g_err.c_str(); }

gd_status gd_create(gd_ctx** out, int device, size_t budget) {
  if (!out) return fail(GD_EINVAL, "out is NULL");
  int count = 0;
  GD_CUDA(cudaGetDeviceCount(&count));
  if (device < 0 || device >= count) return fail(GD_EINVAL, "device %d of %d", device, count);
  GD_CUDA(cudaSetDevice(device));
  gd_ctx* c = new gd_ctx();
  c->device = device;
  c->budget = budget;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  cudaError_t e = cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete c;
    return fail(GD_ECUDA, "stream: %s", cudaGetErrorString(e));
  }
  *out = c;
  g_err.clear();
  return GD_OK;
}

gd_status gd_destroy(gd_ctx* c) {
  if (!c) return GD_OK;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  for (auto& kv : c->dev_free) cudaFree(kv.second);
  for (auto& kv : c->host_free) cudaFreeHost(kv.second);
  for (cudaEvent_t e : c->events) cudaEventDestroy(e);
  if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
  delete c;
  return GD_OK;
}

gd_status gd_load_pocket(gd_ctx* c, const uint8_t* grid, int nx, int ny, int nz, float h, const float origin[3],
                         gd_pocket** out) {
  if (!c || !grid || !origin || !out) return fail(GD_EINVAL, "NULL argument");
  if (nx < 1 || ny < 1 || nz < 1 || (long long)nx * ny * nz > (1ll << 31))
    return fail(GD_EINVAL, "grid dims %d x %d x %d", nx, ny, nz);
  if (!(h > 0.f) || !std::isfinite(h)) return fail(GD_EINVAL, "spacing must be > 0");
  for (int d = 0; d < 3; ++d)
    if (!std::isfinite(origin[d])) return fail(GD_EINVAL, "origin not finite");
  cudaSetDevice(c->device);
  // crop to the bounding box of non-zero cells: every cell outside it scores 0
  int lo[3] = {nx, ny, nz}, hi[3] = {-1, -1, -1};
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i)
        if (grid[((size_t)k * ny + j) * nx + i]) {
          lo[0] = std::min(lo[0], i); hi[0] = std::max(hi[0], i);
          lo[1] = std::min(lo[1], j); hi[1] = std::max(hi[1], j);
          lo[2] = std::min(lo[2], k); hi[2] = std::max(hi[2], k);
        }
  if (hi[0] < 0) lo[0] = lo[1] = lo[2] = hi[0] = hi[1] = hi[2] = 0;  // all zero: one zero cell
  const int cx = hi[0] - lo[0] + 1, cy = hi[1] - lo[1] + 1, cz = hi[2] - lo[2] + 1;
  const size_t bytes = (size_t)cx * cy * cz, pad = align_up(bytes, 16);
  std::vector<uint8_t> crop(pad, 0);
  for (int k = 0; k < cz; ++k)
    for (int j = 0; j < cy; ++j)
      memcpy(&crop[((size_t)k * cy + j) * cx], &grid[((size_t)(k + lo[2]) * ny + (j + lo[1])) * nx + lo[0]], cx);
  gd_pocket* P = new gd_pocket();
  gd_status st = dev_alloc(c, pad, &P->buf);
  if (st) {
    delete P;
    return st;
  }
  P->buf_bytes = pad;
  cudaError_t e = cudaMemcpy(P->buf, crop.data(), pad, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    dev_release(c, P->buf, pad);
    delete P;
    return fail(GD_ECUDA, "pocket upload: %s", cudaGetErrorString(e));
  }
  // the same crop as a 3D array behind a texture object (point sampling, border 0)
  {
    const size_t abytes = (size_t)cx * cy * cz;
    bool over = false;
    {
      std::lock_guard<std::mutex> g(c->mu);
      over = c->budget && c->used + abytes > c->budget;
    }
    if (over) {
      dev_release(c, P->buf, pad);
      delete P;
      return fail(GD_EBUDGET, "device budget %zu B exceeded by the pocket texture", c->budget);
    }
    cudaChannelFormatDesc cd = cudaCreateChannelDesc<unsigned char>();
    const cudaExtent ext = make_cudaExtent(cx, cy, cz);
    e = cudaMalloc3DArray(&P->arr, &cd, ext);
    if (e == cudaSuccess) {
      cudaMemcpy3DParms cp = {};
      cp.srcPtr = make_cudaPitchedPtr(crop.data(), cx, cx, cy);
      cp.dstArray = P->arr;
      cp.extent = ext;
      cp.kind = cudaMemcpyHostToDevice;
      e = cudaMemcpy3D(&cp);
    }
    cudaTextureObject_t tex = 0;
    if (e == cudaSuccess) {
      cudaResourceDesc rd = {};
      rd.resType = cudaResourceTypeArray;
      rd.res.array.array = P->arr;
      cudaTextureDesc td = {};
      td.addressMode[0] = td.addressMode[1] = td.addressMode[2] = cudaAddressModeBorder;
      td.filterMode = cudaFilterModePoint;
      td.readMode = cudaReadModeElementType;
      td.normalizedCoords = 0;
      e = cudaCreateTextureObject(&tex, &rd, &td, nullptr);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (P->arr) cudaFreeArray(P->arr);
      dev_release(c, P->buf, pad);
      delete P;
      return fail(GD_ECUDA, "pocket texture: %s", cudaGetErrorString(e));
    }
    P->arr_bytes = abytes;
    P->dev.tex = (unsigned long long)tex;
    std::lock_guard<std::mutex> g(c->mu);
    c->used += abytes;
  }
  P->nx = nx; P->ny = ny; P->nz = nz;
  gd::PocketDev& d = P->dev;
  d.grid = (const uint8_t*)P->buf;
  d.cx = cx; d.cy = cy; d.cz = cz;
  d.bytes_pad = (int)pad;
  d.inv_h = (float)(1.0 / (double)h);
  d.h = h;
  const int n[3] = {nx, ny, nz};
  for (int a = 0; a < 3; ++a) {
    d.shift[a] = (float)(0.5 * n[a] - lo[a]);
    d.centre[a] = (float)((double)origin[a] + 0.5 * (double)h * n[a]);
  }
  *out = P;
  return GD_OK;
}

gd_status gd_free_pocket(gd_ctx* c, gd_pocket* P) {
  if (!c || !P) return GD_OK;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();  // a queued job may still read the grid
  dev_release(c, P->buf, P->buf_bytes);
  if (P->dev.tex) cudaDestroyTextureObject((cudaTextureObject_t)P->dev.tex);
  if (P->arr) {
    cudaFreeArray(P->arr);
    std::lock_guard<std::mutex> g(c->mu);
    c->used -= P->arr_bytes;
  }
  delete P;
  return GD_OK;
}

gd_status gd_check_batch(const gd_ligand_batch* b, const gd_search_params* p) {
  if (!b) return fail(GD_EINVAL, "batch is NULL");
  gd_status st = check_params(p);
  if (st) return st;
  const int L = b->n_ligands;
  if (L < 0) return fail(GD_EINVAL, "n_ligands < 0");
  if (L == 0) return GD_OK;
  if (!b->atom_off || !b->xyz || !b->bond_off || !b->bonds || !b->rot_off || !b->rot_bond)
    return fail(GD_EINVAL, "batch has a NULL array");
  if (b->atom_off[0] != 0 || b->bond_off[0] != 0 || b->rot_off[0] != 0)
    return fail(GD_EINVAL, "CSR offsets must start at 0");
  std::vector<float4> xyz;
  std::vector<uint8_t> perm;
  std::vector<RotDesc> rots;
  std::vector<uint16_t> excl;
  for (int i = 0; i < L; ++i) {
    if (b->atom_off[i + 1] < b->atom_off[i] || b->bond_off[i + 1] < b->bond_off[i] || b->rot_off[i + 1] < b->rot_off[i])
      return fail(GD_EINVAL, "CSR offsets decrease at ligand %d", i);
    const int a0 = b->atom_off[i], n = b->atom_off[i + 1] - a0;
    const int b0 = b->bond_off[i], nb = b->bond_off[i + 1] - b0;
    const int r0 = b->rot_off[i], R = b->rot_off[i + 1] - r0;
    xyz.resize(std::max(n, 0));
    perm.resize(std::max(n, 0));
    rots.resize(std::max(R, 0));
    double cost;
    if ((st = pack_ligand(i, n, b->xyz + 3 * (size_t)a0, nb, b->bonds + 2 * (size_t)b0, R, b->rot_bond + r0,
                          p->min_bond_sep, xyz.data(), perm.data(), rots.data(), excl, &cost)))
      return st;
  }
  g_err.clear();
  return GD_OK;
}

int gd_tile_count(void) { return gd::tile_count(); }

gd_status gd_tile_info(int tile, int* warps, int* slots, int* max_regs) {
  if (tile < 1 || tile > gd::tile_count()) return fail(GD_EINVAL, "tile %d out of range", tile);
  gd::Tile t = gd::tile_get(tile);
  if (warps) *warps = t.warps;
  if (slots) *slots = t.slots;
  if (max_regs) *max_regs = gd::tile_max_regs(t);
  return GD_OK;
}

gd_status gd_measure_peaks(int device, void* stream, double* ffma_per_s, double* lds_u8_per_s) {
  GD_CUDA(cudaSetDevice(device));
  GD_CUDA(gd::measure_peaks(static_cast<cudaStream_t>(stream), ffma_per_s, lds_u8_per_s));
  return GD_OK;
}

gd_status gd_autotune(gd_ctx* c, const gd_pocket* pk, const gd_ligand_batch* b, const gd_search_params* p,
                      int max_ligands, void* stream, int* best_tile, float* best_ms) {
  if (!c || !pk || !b || !p) return fail(GD_EINVAL, "NULL argument");
  gd_status st = check_params(p);
  if (st) return st;
  cudaSetDevice(c->device);
  gd_ligand_batch sub = *b;
  if (max_ligands > 0 && sub.n_ligands > max_ligands) sub.n_ligands = max_ligands;
  gd_search_params q = *p;
  q.flags &= ~(GD_FLAG_DEBUG | GD_FLAG_DEBUG_BUMPS | GD_FLAG_TEST_STAGE_TIMEOUT);
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  GD_CUDA(cudaEventCreate(&e0));
  GD_CUDA(cudaEventCreate(&e1));
  int best = 0, nmax = 0;
  float bms = 1e30f;
  for (int t = 1; t <= gd::tile_count(); ++t) {
    gd::Tile tl = gd::tile_get(t);
    if (tl.slots > 1 && 32 * (tl.slots / 2) >= p->n_angles) continue;  // idle lanes only
    gd_job* j = nullptr;
    if (make_job(c, pk, &sub, nullptr, 0, &q, t, &j)) continue;
    nmax = j->args.nmax;
    cudaMemcpyAsync(j->d_in, j->h_in, j->in.total, cudaMemcpyHostToDevice, s);
    cudaMemsetAsync((char*)j->d_out + j->out.err, 0, 4, s);
    enqueue_search(j, s);  // warm-up
    cudaEventRecord(e0, s);
    for (int r = 0; r < 3; ++r) enqueue_search(j, s);
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    job_release(c, j);
    if (e != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return fail(GD_ECUDA, "autotune tile %d: %s", t, cudaGetErrorString(e));
    }
    ms /= 3.f;
    if (ms < bms) {
      bms = ms;
      best = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!best) return fail(GD_EINVAL, "no tile could run this batch");
  {
    std::lock_guard<std::mutex> g(c->mu);
    c->tuned[signature(pk, p, nmax, pk->dev.bytes_pad <= gd::max_smem_grid_bytes())] = best;
  }
  if (best_tile) *best_tile = best;
  if (best_ms) *best_ms = bms;
  g_err.clear();
  return GD_OK;
}

namespace {

// Validate, pack and upload a batch (its ligands sel[0 .. n_sel) when sel is not NULL)
// on `stream`; the search is not launched.
gd_status prepare(gd_ctx* c, const gd_pocket* pk, const gd_ligand_batch* b, const int32_t* sel, int n_sel,
                  const gd_search_params* p, void* stream, gd_job** out) {
  if (!c || !pk || !b || !out) return fail(GD_EINVAL, "NULL argument");
  gd_status st = check_params(p);
  if (st) return st;
  cudaSetDevice(c->device);
  int tile = p->tile;  // 0 is resolved once the batch is packed
  if (tile == -1) {
    int nmax = 2;
    for (int i = 0; i < (sel ? n_sel : b->n_ligands); ++i) {
      const int s = sel ? sel[i] : i;
      if (s >= 0 && s < b->n_ligands) nmax = std::max(nmax, b->atom_off[s + 1] - b->atom_off[s]);
    }
    const std::string sig = signature(pk, p, nmax, pk->dev.bytes_pad <= gd::max_smem_grid_bytes());
    int found = 0;
    {
      std::lock_guard<std::mutex> g(c->mu);
      auto it = c->tuned.find(sig);
      if (it != c->tuned.end()) found = it->second;
    }
    if (!found && (st = gd_autotune(c, pk, b, p, 256, stream, &found, nullptr))) return st;
    tile = found;
  }
  gd_job* j = nullptr;
  if ((st = make_job(c, pk, b, sel, n_sel, p, tile, &j))) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(j->d_in, j->h_in, j->in.total, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync((char*)j->d_out + j->out.err, 0, 4, s);
  if (e == cudaSuccess) e = cudaEventRecord(j->done, s);
  if (e != cudaSuccess) {
    job_release(c, j);
    return fail(GD_ECUDA, "upload: %s", cudaGetErrorString(e));
  }
  *out = j;
  return GD_OK;
}

}  // namespace

gd_status gd_prepare_batch(gd_ctx* c, const gd_pocket* pk, const gd_ligand_batch* b, const gd_search_params* p,
                           void* stream, gd_job** out) {
  gd_status st = prepare(c, pk, b, nullptr, 0, p, stream, out);
  if (!st) g_err.clear();
  return st;
}

gd_status gd_prepare_batch_sel(gd_ctx* c, const gd_pocket* pk, const gd_ligand_batch* b, const int32_t* sel,
                               int32_t n_sel, const gd_search_params* p, void* stream, gd_job** out) {
  if (!sel && n_sel) return fail(GD_EINVAL, "NULL sel");
  static const int32_t none = 0;
  gd_status st = prepare(c, pk, b, sel ? sel : &none, n_sel, p, stream, out);
  if (!st) g_err.clear();
  return st;
}

gd_status gd_dock_batch(gd_ctx* c, const gd_pocket* pk, const gd_ligand_batch* b, const gd_search_params* p,
                        void* stream, gd_job** out) {
  gd_job* j = nullptr;
  gd_status st = prepare(c, pk, b, nullptr, 0, p, stream, &j);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = enqueue_search(j, s)) || (st = enqueue_download(j, s))) {
    job_release(c, j);
    return st;
  }
  *out = j;
  g_err.clear();
  return GD_OK;
}

gd_status gd_job_features(gd_ctx* c, gd_job* j, void* x_bf16, float* x_f32, void* stream) {
  if (!c || !j) return fail(GD_EINVAL, "NULL argument");
  if (!x_bf16 && !x_f32) return fail(GD_EINVAL, "no output");
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = gd::launch_features(j->args, (__nv_bfloat16*)x_bf16, x_f32, c->num_sms, s);
  if (e == cudaSuccess) e = cudaEventRecord(j->done, s);
  if (e != cudaSuccess) return fail(GD_ECUDA, "features: %s", cudaGetErrorString(e));
  return GD_OK;
}

gd_status gd_job_launch_proposed(gd_ctx* c, gd_job* j, const float* pred, int k, float margin, int rule,
                                 void* stream) {
  return gd_job_launch_proposed_fb(c, j, pred, k, j ? j->O : 0, margin, rule, stream);
}

gd_status gd_job_launch_proposed_fb(gd_ctx* c, gd_job* j, const float* pred, int k, int k_fallback, float margin,
                                    int rule, void* stream) {
  if (!c || !j || !pred) return fail(GD_EINVAL, "NULL argument");
  if (j->O > 256) return fail(GD_EINVAL, "restart selection supports at most 256 restarts (have %d)", j->O);
  if (k < 1 || k > j->O) return fail(GD_EINVAL, "k = %d outside [1, %d]", k, j->O);
  if (k_fallback < k || k_fallback > j->O)
    return fail(GD_EINVAL, "k_fallback = %d outside [k = %d, %d]", k_fallback, k, j->O);
  if (j->L == 0) return GD_OK;
  cudaSetDevice(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t L = (size_t)j->L, O = (size_t)j->O;
  if (!j->d_sel) {
    size_t o = 0;
    const size_t o_cnt = o;    o = align_up(o + 4 * L, 256);
    const size_t o_off = o;    o = align_up(o + 4 * L, 256);
    const size_t o_n = o;      o = align_up(o + 4, 256);
    const size_t o_topk = o;   o = align_up(o + 2 * L * O, 256);
    const size_t o_spr = o;    o = align_up(o + 4 * L, 256);
    const size_t o_items = o;  o = align_up(o + 4 * L * O, 256);
    gd_status st = dev_alloc(c, o, &j->d_sel);
    if (st) return st;
    j->sel_bytes = o;
    char* b = (char*)j->d_sel;
    j->sel_cnt = (int32_t*)(b + o_cnt);
    j->sel_off = (int32_t*)(b + o_off);
    j->sel_n = (int32_t*)(b + o_n);
    j->sel_topk = (uint16_t*)(b + o_topk);
    j->sel_spread = (float*)(b + o_spr);
    j->sel_items = (uint32_t*)(b + o_items);
  }
  SearchArgs a = j->args;
  a.items = j->sel_items;
  a.item_cnt = j->sel_cnt;
  a.n_items_dev = j->sel_n;
  gd::LaunchCfg cfg;
  cudaError_t e = gd::plan_search(a, j->tile, j->grid_in_smem, c->num_sms, &cfg);
  if (e == cudaSuccess)
    e = gd::launch_selection(a, pred, k, k_fallback, margin, rule, j->sel_cnt, j->sel_topk, j->sel_spread, j->sel_off,
                             j->sel_items, j->sel_n, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.pose_score, 0xFF, 4 * L * O, s);
  if (e == cudaSuccess) e = gd::launch_search(a, cfg, s);
  if (e == cudaSuccess) e = cudaEventRecord(j->done, s);
  if (e != cudaSuccess) return fail(GD_ECUDA, "proposed search: %s", cudaGetErrorString(e));
  return GD_OK;
}

gd_status gd_job_selection(gd_ctx* c, gd_job* j, int32_t* counts, float* spreads) {
  if (!c || !j) return fail(GD_EINVAL, "NULL argument");
  if (!j->d_sel) return fail(GD_EINVAL, "no proposed search was launched on this job");
  cudaSetDevice(c->device);
  GD_CUDA(cudaEventSynchronize(j->done));
  if (counts) GD_CUDA(cudaMemcpy(counts, j->sel_cnt, 4 * (size_t)j->L, cudaMemcpyDeviceToHost));
  if (spreads) GD_CUDA(cudaMemcpy(spreads, j->sel_spread, 4 * (size_t)j->L, cudaMemcpyDeviceToHost));
  return GD_OK;
}

gd_status gd_job_launch(gd_ctx* c, gd_job* j, void* stream) {
  if (!c || !j) return fail(GD_EINVAL, "NULL argument");
  cudaSetDevice(c->device);
  return enqueue_search(j, (cudaStream_t)stream);
}

gd_status gd_job_download(gd_ctx* c, gd_job* j, void* stream) {
  if (!c || !j) return fail(GD_EINVAL, "NULL argument");
  cudaSetDevice(c->device);
  return enqueue_download(j, (cudaStream_t)stream);
}

gd_status gd_fetch_results(gd_ctx* c, gd_job* j, gd_result_batch* r, int blocking) {
  if (!c || !j || !r) return fail(GD_EINVAL, "NULL argument");
  cudaSetDevice(c->device);
  if (blocking) {
    GD_CUDA(cudaEventSynchronize(j->done));
  } else {
    cudaError_t e = cudaEventQuery(j->done);
    if (e == cudaErrorNotReady) return GD_ENOTREADY;
    if (e != cudaSuccess) return fail(GD_ECUDA, "job: %s", cudaGetErrorString(e));
  }
  if (j->L == 0) return GD_OK;
  const char* h = (const char*)j->h_out;
  int32_t err = 0;  // the kernel's error word travels with the results
  memcpy(&err, h + j->out.err, 4);
  if (err == gd::ERR_STAGE_TIMEOUT) return fail(GD_ETIMEOUT, "pocket staging wait timed out on the device");
  const int L = j->L;
  if (r->best_score) memcpy(r->best_score, h + j->out.best_score, 4 * (size_t)L);
  if (r->best_orient) memcpy(r->best_orient, h + j->out.best_orient, 4 * (size_t)L);
  if (r->best_angle) memcpy(r->best_angle, h + j->out.best_angle, 2 * (size_t)j->Rt * j->reps);
  if (r->best_xyz) memcpy(r->best_xyz, h + j->out.best_xyz, 12 * (size_t)j->N);
  if (r->evals) memcpy(r->evals, h + j->out.evals, 8 * (size_t)L);
  if (r->pair_tests) memcpy(r->pair_tests, h + j->out.pair_tests, 8 * (size_t)L);
  if (r->atom_moves) memcpy(r->atom_moves, h + j->out.atom_moves, 8 * (size_t)L);
  if (r->reach_tests) memcpy(r->reach_tests, h + j->out.reach_tests, 8 * (size_t)L);
  if (r->best_rigid) memcpy(r->best_rigid, h + j->out.best_rigid, 2 * (size_t)L);
  if (r->orient_score || r->orient_pick || r->bump_bits || r->orient_rigid) {
    if (!j->debug) return fail(GD_EINVAL, "debug outputs need GD_FLAG_DEBUG at dock time");
    if (r->bump_bits && !j->debug_bumps) return fail(GD_EINVAL, "bump_bits need GD_FLAG_DEBUG_BUMPS at dock time");
    const char* dh = (const char*)j->h_dbg;
    if (r->orient_score) memcpy(r->orient_score, dh + j->scr.pose_score, 4 * (size_t)L * j->O);
    if (r->orient_pick) memcpy(r->orient_pick, dh + j->scr.pose_pick, 2 * (size_t)j->O * j->reps * j->Rt);
    if (r->orient_rigid) memcpy(r->orient_rigid, dh + j->scr.pose_rigid, 2 * (size_t)L * j->O);
    if (r->bump_bits) memcpy(r->bump_bits, dh + j->scr.bump, (size_t)j->O * j->reps * j->A * j->Rt);
  }
  return GD_OK;
}

gd_status gd_job_bytes(gd_ctx* c, const gd_job* j, uint64_t* h2d, uint64_t* d2h) {
  if (!c || !j) return fail(GD_EINVAL, "NULL argument");
  if (h2d) *h2d = j->L ? (uint64_t)j->in.total : 0;
  if (d2h) *d2h = (uint64_t)j->out.total + (j->debug ? (uint64_t)j->dbg_bytes : 0);
  return GD_OK;
}

gd_status gd_job_info(gd_ctx* c, const gd_job* j, int* tile, int* grid_in_smem, int* blocks, int* threads,
                      size_t* smem_bytes) {
  if (!c || !j) return fail(GD_EINVAL, "NULL argument");
  if (tile) *tile = j->tile;
  if (grid_in_smem) *grid_in_smem = j->grid_in_smem ? 1 : 0;
  if (blocks) *blocks = (int)j->cfg.blocks;
  if (threads) *threads = (int)j->cfg.threads;
  if (smem_bytes) *smem_bytes = j->cfg.smem;
  return GD_OK;
}

gd_status gd_job_free(gd_ctx* c, gd_job* j) {
  if (!c || !j) return GD_OK;
  cudaSetDevice(c->device);
  return job_release(c, j);
}

}  // extern "C"

// ---------------------------------------------------------------- streaming server
//
// Host side of the persistent search launch that ligands join while it runs (declared
// with gd_server_create).  Mapped (zero-copy) host memory holds the control words the
// launch polls, one packed record per slot and one result row per slot; the device holds
// the slots' search data and per-restart scratch.  Ligand seq lives in slot seq % cap;
// a slot is reused only once its ligand's results were returned to the caller.

struct gd_server {
  gd_ctx* ctx = nullptr;
  int O = 0, reps = 0, A = 0, cap = 0, amax = 0, rmax = 0, emax = 0, tile = 0, min_sep = 3;
  bool grid_in_smem = false;
  SearchArgs args{};
  gd::ServeArgs sv{};
  gd::LaunchCfg cfg{};
  cudaStream_t stream = nullptr;
  cudaEvent_t ended = nullptr;
  bool running = false;
  // mapped host memory: control words | records | result rows
  char* h_map = nullptr;
  volatile unsigned long long* h_published = nullptr;
  volatile int* h_stop = nullptr;
  volatile int* h_status = nullptr;
  volatile unsigned long long* h_result_seq = nullptr;
  char* h_rec = nullptr;
  uint32_t* h_score = nullptr;
  int32_t* h_orient = nullptr;
  uint64_t *h_evals = nullptr, *h_pairs = nullptr, *h_moves = nullptr, *h_reach = nullptr;
  int16_t* h_rigid = nullptr;
  int16_t* h_angle = nullptr;
  float* h_xyz = nullptr;
  // device memory
  void* d_mem = nullptr;
  size_t dev_bytes = 0;
  unsigned long long* d_work = nullptr;
  // bookkeeping
  unsigned long long next_seq = 0;      // ligands published
  unsigned long long oldest = 0;        // no ligand before this one is still outstanding
  unsigned long long launches = 0, idle_exits = 0, finished = 0;
  std::vector<unsigned long long> owner;  // per slot: seq + 1 of the ligand in it, 0 if free
  std::vector<int32_t> nat, nrot;         // per slot: atoms and rotamers of that ligand
};

namespace {

// Device-side bounds are counted in SM cycles (the clock every SM has); at the maximum
// clock of 2.032 GHz these are the times named, at lower clocks longer.
constexpr double SERVE_CYCLES_PER_NS = 2.032;
constexpr long long SERVE_WAIT_CYCLES = (long long)(0.5e9 * SERVE_CYCLES_PER_NS);       // a slot being staged
constexpr long long SERVE_TEST_WAIT_CYCLES = (long long)(0.2e9 * SERVE_CYCLES_PER_NS);  // ... held by a test
constexpr double SERVE_POLL_LIMIT_S = 30.0;  // a blocking gd_server_poll gives up after this long

// Whether some published ligand has no results yet.
bool server_unfinished(const gd_server* s) {
  for (unsigned long long q = s->oldest; q < s->next_seq; ++q) {
    const int slot = (int)(q % (unsigned long long)s->cap);
    if (s->owner[slot] == q + 1 && s->h_result_seq[slot] != q + 1) return true;
  }
  return false;
}

// Notice a launch that ended; launch again if a published ligand has no results yet (its
// items, or tickets parked for them, wait for a launch).
gd_status server_pump(gd_server* s) {
  if (s->running) {
    const cudaError_t e = cudaEventQuery(s->ended);
    if (e == cudaErrorNotReady) return GD_OK;
    if (e != cudaSuccess) return fail(GD_ECUDA, "server launch: %s", cudaGetErrorString(e));
    s->running = false;
    if (!*s->h_stop && *s->h_status == gd::ERR_NONE) ++s->idle_exits;
  }
  if (*s->h_status != gd::ERR_NONE)
    return fail(GD_ETIMEOUT, *s->h_status == gd::ERR_SLOT_TIMEOUT ? "a server wait for a staged slot timed out"
                                                                   : "the server's pocket staging wait timed out");
  if (*s->h_stop || !server_unfinished(s)) return GD_OK;
  GD_CUDA(cudaMemsetAsync(s->sv.idle_state, 0, sizeof(unsigned long long), s->stream));
  GD_CUDA(gd::launch_serve(s->args, s->sv, s->cfg, s->stream));
  GD_CUDA(cudaEventRecord(s->ended, s->stream));
  s->running = true;
  ++s->launches;
  return GD_OK;
}

void server_free(gd_server* s) {
  if (s->stream) cudaStreamSynchronize(s->stream);
  if (s->ended) cudaEventDestroy(s->ended);
  if (s->stream) cudaStreamDestroy(s->stream);
  if (s->h_map) cudaFreeHost(s->h_map);
  dev_release(s->ctx, s->d_mem, s->dev_bytes);
  delete s;
}

}  // namespace

extern "C" {

gd_status gd_server_create(gd_ctx* c, const gd_pocket* pk, const gd_search_params* p, int capacity, int max_atoms,
                           int max_rotamers, int max_excluded, int idle_ms, gd_server** out) {
  if (!c || !pk || !p || !out) return fail(GD_EINVAL, "NULL argument");
  gd_status st = check_params(p);
  if (st) return st;
  if (p->flags & (GD_FLAG_DEBUG | GD_FLAG_DEBUG_BUMPS | GD_FLAG_TEST_STAGE_TIMEOUT))
    return fail(GD_EINVAL, "the server keeps no debug outputs and takes no test flags");
  if (capacity < 1 || capacity > (1 << 20)) return fail(GD_EINVAL, "capacity %d outside [1, 2^20]", capacity);
  if (max_atoms < 2 || max_atoms > GD_MAX_ATOMS) return fail(GD_EINVAL, "max_atoms %d outside [2, %d]", max_atoms,
                                                             GD_MAX_ATOMS);
  if (max_rotamers < 0 || max_rotamers > GD_MAX_ROTAMERS)
    return fail(GD_EINVAL, "max_rotamers %d outside [0, %d]", max_rotamers, GD_MAX_ROTAMERS);
  if (max_excluded == 0) max_excluded = 16 * std::max(1, max_rotamers);
  if (max_excluded < 1 || max_excluded > GD_MAX_EXCLUDED * std::max(1, max_rotamers))
    return fail(GD_EINVAL, "max_excluded %d outside [1, %d]", max_excluded, GD_MAX_EXCLUDED * std::max(1, max_rotamers));
  if (idle_ms < 1 || idle_ms > 60000) return fail(GD_EINVAL, "idle_ms %d outside [1, 60000]", idle_ms);
  const int O = p->n_alpha * p->n_beta * p->n_gamma;
  if (max_rotamers * p->repetitions > 32767) return fail(GD_EINVAL, "too many steps per ligand");
  cudaSetDevice(c->device);
  gd_server* s = new gd_server();
  s->ctx = c;
  s->O = O;
  s->reps = p->repetitions;
  s->A = p->n_angles;
  s->cap = capacity;
  s->amax = (max_atoms + 3) / 4 * 4;  // 4-byte aligned per-slot permutation rows
  s->rmax = std::max(1, max_rotamers);
  s->emax = max_excluded;
  s->min_sep = p->min_bond_sep;
  s->owner.assign(capacity, 0);
  s->nat.assign(capacity, 0);
  s->nrot.assign(capacity, 0);
  const long long cap = capacity, amax = s->amax, rmax = s->rmax, emax = s->emax;
  const long long rec_stride = gd::serve_rec_bytes(s->amax, s->rmax, s->emax, O);
  // mapped host memory
  size_t o = 0;
  const size_t o_ctrl = o;   o = align_up(o + 256, 256);
  const size_t o_rec = o;    o = align_up(o + (size_t)(cap * rec_stride), 256);
  const size_t o_rseq = o;   o = align_up(o + 8 * cap, 256);
  const size_t o_score = o;  o = align_up(o + 4 * cap, 256);
  const size_t o_orient = o; o = align_up(o + 4 * cap, 256);
  const size_t o_evals = o;  o = align_up(o + 8 * cap, 256);
  const size_t o_pairs = o;  o = align_up(o + 8 * cap, 256);
  const size_t o_moves = o;  o = align_up(o + 8 * cap, 256);
  const size_t o_reach = o;  o = align_up(o + 8 * cap, 256);
  const size_t o_rigid = o;  o = align_up(o + 2 * cap, 256);
  const size_t o_angle = o;  o = align_up(o + 2 * (size_t)(cap * rmax * s->reps), 256);
  const size_t o_xyz = o;    o = align_up(o + 12 * (size_t)(cap * amax), 256);
  const size_t map_bytes = o;
  cudaError_t e = cudaHostAlloc((void**)&s->h_map, map_bytes, cudaHostAllocMapped);
  if (e != cudaSuccess) {
    cudaGetLastError();
    s->h_map = nullptr;
    server_free(s);
    return fail(GD_ENOMEM, "cudaHostAlloc(%zu, mapped): %s", map_bytes, cudaGetErrorString(e));
  }
  memset(s->h_map, 0, map_bytes);
  char* h = s->h_map;
  s->h_published = (volatile unsigned long long*)(h + o_ctrl);
  s->h_stop = (volatile int*)(h + o_ctrl + 8);
  s->h_status = (volatile int*)(h + o_ctrl + 12);
  s->h_rec = h + o_rec;
  s->h_result_seq = (volatile unsigned long long*)(h + o_rseq);
  s->h_score = (uint32_t*)(h + o_score);
  s->h_orient = (int32_t*)(h + o_orient);
  s->h_evals = (uint64_t*)(h + o_evals);
  s->h_pairs = (uint64_t*)(h + o_pairs);
  s->h_moves = (uint64_t*)(h + o_moves);
  s->h_reach = (uint64_t*)(h + o_reach);
  s->h_rigid = (int16_t*)(h + o_rigid);
  s->h_angle = (int16_t*)(h + o_angle);
  s->h_xyz = (float*)(h + o_xyz);
  char* hd = nullptr;  // the same memory as the device addresses it
  e = cudaHostGetDevicePointer((void**)&hd, s->h_map, 0);
  if (e != cudaSuccess) {
    server_free(s);
    return fail(GD_ECUDA, "cudaHostGetDevicePointer: %s", cudaGetErrorString(e));
  }
  // device memory
  o = 0;
  const size_t d_work = o;    o += 8;
  const size_t d_pub = o;     o += 8;
  const size_t d_stop = o;    o += 8;
  const size_t d_poll = o;    o += 8;
  const size_t d_polls = o;   o += 8;
  const size_t d_idle = o;    o += 8;
  const size_t d_dummy = o;   o = align_up(o + 8, 256);
  const size_t d_parked = o;  o = align_up(o + 8 * (size_t)c->num_sms * 64, 256);  // every resident warp
  const size_t d_ready = o;   o = align_up(o + 8 * cap, 256);
  const size_t d_claim = o;   o = align_up(o + 8 * cap, 256);
  const size_t d_nres = o;    o = align_up(o + 4 * cap, 256);
  const size_t d_done = o;    o = align_up(o + 4 * cap, 256);
  const size_t d_n = o;       o = align_up(o + 4 * cap, 256);
  const size_t d_r = o;       o = align_up(o + 4 * cap, 256);
  const size_t d_err = o;     o = align_up(o + 4, 256);
  const size_t d_xc = o;      o = align_up(o + 16 * (size_t)(cap * amax), 256);
  const size_t d_perm = o;    o = align_up(o + (size_t)(cap * amax), 256);
  const size_t d_rots = o;    o = align_up(o + 16 * (size_t)(cap * rmax), 256);
  const size_t d_excl = o;    o = align_up(o + 2 * (size_t)(cap * emax), 256);
  const size_t d_pscore = o;  o = align_up(o + 4 * (size_t)(cap * O), 256);
  const size_t d_ppick = o;   o = align_up(o + 2 * (size_t)(cap * rmax * s->reps * O), 256);
  const size_t d_ppairs = o;  o = align_up(o + 8 * (size_t)(cap * O), 256);
  const size_t d_preach = o;  o = align_up(o + 8 * (size_t)(cap * O), 256);
  const size_t d_prigid = o;  o = align_up(o + 2 * (size_t)(cap * O), 256);
  const size_t d_rmat = o;    o = align_up(o + 36 * (size_t)O, 256);
  const size_t d_quat = o;    o = align_up(o + 16 * (size_t)O, 256);
  const size_t d_res = o;     o = align_up(o + 2 * (size_t)cap * O, 256);
  s->dev_bytes = o;
  if ((st = dev_alloc(c, s->dev_bytes, &s->d_mem))) {
    s->d_mem = nullptr;
    server_free(s);
    return st;
  }
  char* d = (char*)s->d_mem;
  s->d_work = (unsigned long long*)(d + d_work);
  e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ended, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMemsetAsync(d, 0, d_xc, s->stream);  // counters, slot words
  if (e != cudaSuccess) {
    server_free(s);
    return fail(GD_ECUDA, "server set-up: %s", cudaGetErrorString(e));
  }
  // search arguments in the slot layout
  SearchArgs& a = s->args;
  a.pk = pk->dev;
  a.L = capacity;
  a.xc = (float4*)(d + d_xc);
  a.perm = (const uint8_t*)(d + d_perm);
  a.rots = (const RotDesc*)(d + d_rots);
  a.excl = (const uint16_t*)(d + d_excl);
  a.slot_n = (const int32_t*)(d + d_n);
  a.slot_r = (const int32_t*)(d + d_r);
  a.slot_amax = s->amax;
  a.slot_rmax = s->rmax;
  a.na = p->n_alpha;
  a.nb = p->n_beta;
  a.ng = p->n_gamma;
  a.O = O;
  a.A = p->n_angles;
  a.reps = p->repetitions;
  {
    const float ih = a.pk.inv_h, bd = p->bump_dist * ih, rd = (p->bump_dist + gd::REACH_MARGIN) * ih;
    a.thr2 = bd * bd;
    a.reach2 = rd * rd;
  }
  a.use_filter = (p->flags & GD_FLAG_NO_FILTER) ? 0 : 1;
  a.mask_sweep = (p->flags & GD_FLAG_MASK_SWEEP) ? 1 : 0;
  a.rigid_span = p->rigid_span;
  a.rigid_step = p->rigid_step;
  a.rigid_n = p->rigid_span > 0 ? (2 * p->rigid_span + 1) * (2 * p->rigid_span + 1) * (2 * p->rigid_span + 1) : 0;
  a.best_score = (uint32_t*)(hd + o_score);
  a.best_orient = (int32_t*)(hd + o_orient);
  a.best_angle = (int16_t*)(hd + o_angle);
  a.best_xyz = (float*)(hd + o_xyz);
  a.evals = (unsigned long long*)(hd + o_evals);
  a.pair_tests = (unsigned long long*)(hd + o_pairs);
  a.atom_moves = (unsigned long long*)(hd + o_moves);
  a.reach_tests = (unsigned long long*)(hd + o_reach);
  a.best_rigid = (int16_t*)(hd + o_rigid);
  a.pose_score = (uint32_t*)(d + d_pscore);
  a.pose_pick = (int16_t*)(d + d_ppick);
  a.pose_pairs = (unsigned long long*)(d + d_ppairs);
  a.pose_reach = (unsigned long long*)(d + d_preach);
  a.pose_rigid = (int16_t*)(d + d_prigid);
  a.rmat = (float*)(d + d_rmat);
  a.quat = (float4*)(d + d_quat);
  a.done = (int32_t*)(d + d_done);
  a.work = (unsigned long long*)(d + d_dummy);  // written by the restart-table launch only
  a.err = (int32_t*)(d + d_err);
  a.bump_bits = nullptr;
  // per-warp buffers sized for the largest ligand the server accepts: the fragment is the
  // smaller side of its bond (at most half the atoms)
  a.nmax = s->amax;
  a.fmax = std::max(1, s->amax / 2);
  a.mask_words = 1;
  for (int f = 1; f <= s->amax / 2; ++f) a.mask_words = std::max(a.mask_words, f * ((s->amax - f + 31) / 32));
  a.rmax = s->rmax;
  a.emax = s->emax;
  // tile: the built-in default (never a compact one) unless the caller named one
  int tile = p->tile;
  if (tile < 0) {
    server_free(s);
    return fail(GD_EINVAL, "the server takes tile 0 (default) or a lean or wide tile id");
  }
  if (tile == 0) {  // the wide tile with the most warps whose buffers fit a block (16, 8, 4, 2)
    const int two = a.A >= 64 ? 1 : 0;
    const int ids[4] = {7 + two, 1 + two, 4 + two, 10 + two};
    tile = ids[3];
    for (int id : ids)
      if (gd::search_smem_bytes(a, id, false) <= 227 * 1024) {
        tile = id;
        break;
      }
  }
  if (gd::tile_get(tile).build == gd::BUILD_COMPACT) {
    server_free(s);
    return fail(GD_EINVAL, "tile %d is a compact build: the server needs a lean or wide tile", tile);
  }
  const size_t smem_cap = 227 * 1024;
  s->tile = tile;
  s->grid_in_smem = gd::tile_stages_grid(gd::tile_get(tile)) && pk->dev.bytes_pad <= gd::max_smem_grid_bytes() &&
                    gd::search_smem_bytes(a, tile, true) <= smem_cap;
  if (!s->grid_in_smem && gd::search_smem_bytes(a, tile, false) > smem_cap) {
    server_free(s);
    return fail(GD_EINVAL, "tile %d needs more shared memory than a block has for %d-atom ligands", tile, max_atoms);
  }
  e = gd::plan_serve(a, tile, s->grid_in_smem, c->num_sms, &s->cfg);
  if (e != cudaSuccess) {
    server_free(s);
    return fail(GD_ECUDA, "server launch shape: %s", cudaGetErrorString(e));
  }
  gd::ServeArgs& v = s->sv;
  v.published = (const unsigned long long*)(hd + o_ctrl);
  v.stop = (const int*)(hd + o_ctrl + 8);
  v.status = (int*)(hd + o_ctrl + 12);
  v.work = s->d_work;
  v.pub_dev = (unsigned long long*)(d + d_pub);
  v.stop_dev = (unsigned long long*)(d + d_stop);
  v.last_poll = (unsigned long long*)(d + d_poll);
  v.slot_ready = (unsigned long long*)(d + d_ready);
  v.slot_claim = (unsigned long long*)(d + d_claim);
  v.slot_nres = (int32_t*)(d + d_nres);
  v.slot_res = (uint16_t*)(d + d_res);
  v.result_seq = (unsigned long long*)(hd + o_rseq);
  v.rec = (const unsigned char*)(hd + o_rec);
  v.rec_stride = rec_stride;
  v.cap = capacity;
  v.emax = s->emax;
  v.chunk = 4;
  v.chunks = (O + 3) / 4;
  v.idle_cycles = (long long)((double)idle_ms * 1e6 * SERVE_CYCLES_PER_NS);
  v.wait_cycles = SERVE_WAIT_CYCLES;
  v.polls = (unsigned long long*)(d + d_polls);
  v.parked = (unsigned long long*)(d + d_parked);
  v.idle_state = (unsigned long long*)(d + d_idle);
  v.hold_seq = -1;
  e = gd::launch_restart_tables(a, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    server_free(s);
    return fail(GD_ECUDA, "restart tables: %s", cudaGetErrorString(e));
  }
  *out = s;
  g_err.clear();
  return GD_OK;
}

namespace {

// gd_server_submit(_restarts): restarts NULL searches every restart of each ligand; else
// ligand i of the submission searches restarts[i * res_stride .. + n_restarts[i]).
gd_status server_submit(gd_server* s, const gd_ligand_batch* b, const int32_t* sel, int32_t n_sel,
                        const uint16_t* restarts, const int32_t* n_restarts, int32_t res_stride, uint64_t* first_seq) {
  if (!s || !b) return fail(GD_EINVAL, "NULL argument");
  cudaSetDevice(s->ctx->device);
  const int LB = b->n_ligands;
  const int n = sel ? n_sel : LB;
  if (LB < 0 || n < 0) return fail(GD_EINVAL, "negative ligand count");
  if (n > 0 && (!b->atom_off || !b->xyz || !b->bond_off || !b->bonds || !b->rot_off || !b->rot_bond))
    return fail(GD_EINVAL, "batch has a NULL array");
  if (n > s->cap) return fail(GD_EINVAL, "%d ligands for %d slots", n, s->cap);
  if (*s->h_status != gd::ERR_NONE) return fail(GD_ETIMEOUT, "a server wait for a staged slot timed out");
  for (int i = 0; i < n; ++i)
    if (s->owner[(s->next_seq + i) % s->cap]) return fail(GD_EBUSY, "no free slot: return finished results first");
  const long long stride = s->sv.rec_stride;
  for (int i = 0; i < n; ++i) {
    const int li = sel ? sel[i] : i;
    if (li < 0 || li >= LB) return fail(GD_EINVAL, "sel[%d] = %d outside [0, %d)", i, li, LB);
  }
  if (restarts) {
    if (!n_restarts) return fail(GD_EINVAL, "restart lists without their lengths");
    std::vector<unsigned char> seen((size_t)s->O);
    for (int i = 0; i < n; ++i) {
      const int k = n_restarts[i];
      if (k < 1 || k > s->O || k > res_stride)
        return fail(GD_EINVAL, "ligand %d of the submission: %d restarts outside [1, min(%d, stride %d)]", i, k, s->O,
                    res_stride);
      std::fill(seen.begin(), seen.end(), 0);
      for (int q = 0; q < k; ++q) {
        const int o = restarts[(size_t)i * res_stride + q];
        if (o >= s->O) return fail(GD_EINVAL, "ligand %d of the submission: restart %d outside [0, %d)", i, o, s->O);
        if (seen[o]) return fail(GD_EINVAL, "ligand %d of the submission: restart %d listed twice", i, o);
        seen[o] = 1;
      }
    }
  }
  // pack each ligand into its slot's record, on the context's packing threads for large
  // submissions (contiguous ranges; the first failure in submission order is reported)
  struct Part {
    int i0 = 0, i1 = 0, bad = -1;
    gd_status st = GD_OK;
    std::string err;
  };
  const int T = std::max(1, std::min(s->ctx->pool.threads(), n / 32));
  std::vector<Part> parts(T);
  for (int t = 0; t < T; ++t) {
    parts[t].i0 = (int)((long long)n * t / T);
    parts[t].i1 = (int)((long long)n * (t + 1) / T);
  }
  auto work = [&](Part& pt) {
    for (int i = pt.i0; i < pt.i1; ++i) {
      const int li = sel ? sel[i] : i;
      const int a0 = b->atom_off[li], na = b->atom_off[li + 1] - a0;
      const int b0 = b->bond_off[li], nb = b->bond_off[li + 1] - b0;
      const int r0 = b->rot_off[li], R = b->rot_off[li + 1] - r0;
      gd_status st = GD_OK;
      if (na > s->amax || na < 0) st = fail(GD_EINVAL, "ligand %d: %d atoms > the server's %d", li, na, s->amax);
      else if (R > s->rmax || R < 0) st = fail(GD_EINVAL, "ligand %d: %d rotamers > the server's %d", li, R, s->rmax);
      const int slot = (int)((s->next_seq + i) % s->cap);
      char* rec = s->h_rec + (size_t)slot * (size_t)stride;
      size_t ne = 0;
      if (!st)
        st = gd::pack_ligand_fixed(fail, li, na, b->xyz + 3 * (size_t)a0, nb, b->bonds + 2 * (size_t)b0, R,
                                   b->rot_bond + r0, s->min_sep, (float4*)(rec + 16),
                                   (uint8_t*)(rec + gd::serve_rec_perm_dev(s->amax)),
                                   (RotDesc*)(rec + gd::serve_rec_rots_dev(s->amax)),
                                   (uint16_t*)(rec + gd::serve_rec_excl_dev(s->amax, s->rmax)), (size_t)s->emax, &ne,
                                   nullptr);
      if (st) {
        pt.st = st;
        pt.bad = i;
        pt.err = g_err;  // the message lives in this thread's g_err
        return;
      }
      // every restart listed is the same as none listed: all of them, in order
      const int32_t nres = restarts && n_restarts[i] < s->O ? n_restarts[i] : 0;
      if (nres)
        memcpy(rec + gd::serve_rec_res_dev(s->amax, s->rmax, s->emax), restarts + (size_t)i * res_stride,
               2 * (size_t)nres);
      const gd::ServeRecHeader hdr{na, R, (int32_t)ne, nres};
      memcpy(rec, &hdr, sizeof hdr);
      s->nat[slot] = na;
      s->nrot[slot] = R;
    }
  };
  if (T == 1) work(parts[0]);
  else s->ctx->pool.run(T, [&](int t) { work(parts[t]); });
  for (auto& pt : parts)
    if (pt.st) {  // nothing of this call is published: the slots stay free
      g_err = pt.err;
      return pt.st;
    }
  for (int i = 0; i < n; ++i) s->owner[(s->next_seq + i) % s->cap] = s->next_seq + i + 1;
  if (first_seq) *first_seq = s->next_seq;
  s->next_seq += n;
  std::atomic_thread_fence(std::memory_order_seq_cst);  // the records before the count
  *s->h_published = s->next_seq;
  std::atomic_thread_fence(std::memory_order_seq_cst);
  return server_pump(s);
}

}  // namespace

gd_status gd_server_submit(gd_server* s, const gd_ligand_batch* b, const int32_t* sel, int32_t n_sel,
                           uint64_t* first_seq) {
  return server_submit(s, b, sel, n_sel, nullptr, nullptr, 0, first_seq);
}

gd_status gd_server_submit_restarts(gd_server* s, const gd_ligand_batch* b, const int32_t* sel, int32_t n_sel,
                                    const uint16_t* restarts, const int32_t* n_restarts, int32_t stride,
                                    uint64_t* first_seq) {
  if (!restarts) return fail(GD_EINVAL, "NULL restart lists");
  return server_submit(s, b, sel, n_sel, restarts, n_restarts, stride, first_seq);
}

gd_status gd_server_reserve_sms(gd_server* s, int free_sms) {
  if (!s) return fail(GD_EINVAL, "NULL argument");
  if (s->launches) return fail(GD_EBUSY, "the server has launched already: reserve SMs before the first submission");
  if (free_sms < 0 || free_sms >= s->ctx->num_sms)
    return fail(GD_EINVAL, "free_sms = %d outside [0, %d)", free_sms, s->ctx->num_sms);
  cudaSetDevice(s->ctx->device);
  const cudaError_t e = gd::plan_serve(s->args, s->tile, s->grid_in_smem, s->ctx->num_sms - free_sms, &s->cfg);
  if (e != cudaSuccess) return fail(GD_ECUDA, "server launch shape: %s", cudaGetErrorString(e));
  g_err.clear();
  return GD_OK;
}

gd_status gd_server_poll(gd_server* s, uint64_t seq, gd_result_batch* r, int blocking) {
  if (!s || !r) return fail(GD_EINVAL, "NULL argument");
  if (r->orient_score || r->orient_pick || r->bump_bits || r->orient_rigid)
    return fail(GD_EINVAL, "the server keeps no debug outputs");
  cudaSetDevice(s->ctx->device);
  const int slot = (int)(seq % (uint64_t)s->cap);
  if (seq >= s->next_seq || s->owner[slot] != seq + 1) return fail(GD_EINVAL, "ligand %llu is not outstanding",
                                                                   (unsigned long long)seq);
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    gd_status st = server_pump(s);
    if (st) return st;
    if (s->h_result_seq[slot] == seq + 1) break;
    if (!blocking) return GD_ENOTREADY;
    if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > SERVE_POLL_LIMIT_S)
      return fail(GD_ETIMEOUT, "no result for ligand %llu within %.0f s", (unsigned long long)seq, SERVE_POLL_LIMIT_S);
    std::this_thread::yield();
  }
  std::atomic_thread_fence(std::memory_order_acquire);
  const int na = s->nat[slot], R = s->nrot[slot];
  if (r->best_score) r->best_score[0] = s->h_score[slot];
  if (r->best_orient) r->best_orient[0] = s->h_orient[slot];
  if (r->best_angle) memcpy(r->best_angle, s->h_angle + (size_t)slot * s->rmax * s->reps, 2 * (size_t)R * s->reps);
  if (r->best_xyz) memcpy(r->best_xyz, s->h_xyz + 3 * (size_t)slot * s->amax, 12 * (size_t)na);
  if (r->evals) r->evals[0] = s->h_evals[slot];
  if (r->pair_tests) r->pair_tests[0] = s->h_pairs[slot];
  if (r->atom_moves) r->atom_moves[0] = s->h_moves[slot];
  if (r->reach_tests) r->reach_tests[0] = s->h_reach[slot];
  if (r->best_rigid) r->best_rigid[0] = s->h_rigid[slot];
  s->owner[slot] = 0;
  ++s->finished;
  return GD_OK;
}

gd_status gd_server_collect(gd_server* s, uint64_t* seqs, uint32_t* score, int32_t* orient, int max, int* n_out) {
  if (!s || !n_out || max < 0) return fail(GD_EINVAL, "bad argument");
  cudaSetDevice(s->ctx->device);
  *n_out = 0;
  gd_status st = server_pump(s);
  if (st) return st;
  int k = 0;
  for (unsigned long long q = s->oldest; q < s->next_seq && k < max; ++q) {
    const int slot = (int)(q % (unsigned long long)s->cap);
    if (s->owner[slot] != q + 1) {  // returned already
      if (q == s->oldest) ++s->oldest;
      continue;
    }
    if (s->h_result_seq[slot] != q + 1) continue;
    std::atomic_thread_fence(std::memory_order_acquire);
    if (seqs) seqs[k] = q;
    if (score) score[k] = s->h_score[slot];
    if (orient) orient[k] = s->h_orient[slot];
    s->owner[slot] = 0;
    ++s->finished;
    ++k;
    if (q == s->oldest) ++s->oldest;
  }
  *n_out = k;
  return GD_OK;
}

gd_status gd_server_stats(gd_server* s, uint64_t* launches, uint64_t* idle_exits, uint64_t* published,
                          uint64_t* finished, uint64_t* claimed_items, uint64_t* control_reads) {
  if (!s) return fail(GD_EINVAL, "NULL argument");
  cudaSetDevice(s->ctx->device);
  if (s->running && cudaEventQuery(s->ended) == cudaSuccess) server_pump(s);
  if (launches) *launches = s->launches;
  if (idle_exits) *idle_exits = s->idle_exits;
  if (published) *published = s->next_seq;
  if (finished) *finished = s->finished;
  if (claimed_items || control_reads) {  // device counters, read on a stream of their own (the launch may run)
    unsigned long long v[2] = {0, 0};
    cudaStream_t st = nullptr;
    GD_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    cudaError_t e = cudaMemcpyAsync(&v[0], s->sv.work, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&v[1], s->sv.polls, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    if (e != cudaSuccess) return fail(GD_ECUDA, "server counters: %s", cudaGetErrorString(e));
    if (claimed_items) *claimed_items = v[0];
    if (control_reads) *control_reads = v[1];
  }
  return GD_OK;
}

gd_status gd_server_test_hold(gd_server* s, int64_t hold_seq) {
  if (!s) return fail(GD_EINVAL, "NULL argument");
  cudaSetDevice(s->ctx->device);
  // the hold and the wait bound travel with the launch parameters: a running launch is
  // left to end (it does once idle), and the next one takes them
  s->sv.hold_seq = hold_seq;
  s->sv.wait_cycles = hold_seq >= 0 ? SERVE_TEST_WAIT_CYCLES : SERVE_WAIT_CYCLES;
  if (s->running) {
    GD_CUDA(cudaEventSynchronize(s->ended));
    s->running = false;
    if (!*s->h_stop && *s->h_status == gd::ERR_NONE) ++s->idle_exits;
  }
  return GD_OK;
}

gd_status gd_server_destroy(gd_server* s) {
  if (!s) return GD_OK;
  cudaSetDevice(s->ctx->device);
  *s->h_stop = 1;
  std::atomic_thread_fence(std::memory_order_seq_cst);
  server_free(s);
  return GD_OK;
}

}  // extern "C"
