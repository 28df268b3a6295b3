/* geodock.h -- C ABI of the B300 GeoDock pose-search library (libgeodock.so).
 *
 * The calls follow the paper's problem statement: a target pocket is loaded once
 * (Listing 1, "load(pocket)"), a library of ligands -- atoms plus rotamers, the bonds
 * that split a ligand into two fragments rotating about the bond axis (Sec. 1) -- is
 * docked against it, data crosses the host/device boundary once on the way in and
 * once on the way out (Sec. 4.1), and only the best pose and score of every ligand
 * come back (Sec. 4.1, "we only extract the result at the end").
 *
 * Method computed for every ligand (Sec. 3.1, Listing 1; Sec. 4.1, Listing 2):
 *   for each restart o of an Euler-angle grid (generate_starting_pose):
 *     x <- c_pocket + R_o (x - c_lig)                 rigid placement (align phase)
 *     repeat `repetitions` times, for each rotamer r in order (optimize_pose):
 *       rotate the smaller side of bond r about the bond axis by 2 pi k / A,
 *       k = 0..A-1; a candidate is rejected when a moving and a static atom at
 *       graph distance >= min_bond_sep come closer than bump_dist (BumpCheck);
 *       the others are scored as the sum of pocket-grid cells under the atoms
 *       (scoring function, Sec. 3.2); the best angle is kept (ties: smallest k).
 *   the best restart (ties: smallest o) is the ligand's pose.
 * Arithmetic: FP32 on the device.  Scores are exact integers.
 *
 * Conventions: every call returns a gd_status; nothing else crosses the ABI (no
 * exceptions, no exit).  On failure gd_last_error() holds a one-line reason for the
 * calling thread.  One context per thread, or external locking.  Streams are
 * cudaStream_t passed as void* (NULL = the legacy default stream).
 */
#ifndef GEODOCK_H
#define GEODOCK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int gd_status;
#define GD_OK 0
#define GD_EINVAL 1      /* malformed input or parameter (reason in gd_last_error) */
#define GD_ENOMEM 2      /* host or device allocation failed */
#define GD_EBUDGET 3     /* the request would exceed the context's device-memory budget */
#define GD_ECUDA 4       /* a CUDA runtime call failed */
#define GD_ETIMEOUT 5    /* a bounded device-side wait ran out (kernel returned early) */
#define GD_EBUSY 6       /* the object is still in use by queued device work */
#define GD_ENOTREADY 7   /* non-blocking fetch: results not ready yet */

/* Limits checked by every entry point. */
#define GD_MAX_ATOMS 256        /* atoms per ligand */
#define GD_MAX_ROTAMERS 128     /* rotamers per ligand */
#define GD_MAX_ANGLES 1024      /* angles per rotamer sweep */
#define GD_MAX_ORIENT 65535     /* restart orientations */
#define GD_MAX_REPS 16          /* optimize_pose repetitions */
#define GD_MAX_EXCLUDED 128     /* moving x static pairs closer than min_bond_sep bonds, per rotamer */
#define GD_MAX_EXCLUDED_ATOM 32 /* ... and per moving atom */

/* Flags of gd_search_params.flags */
#define GD_FLAG_DEBUG 1         /* keep per-orientation scores and picks (orient_score, orient_pick) */
#define GD_FLAG_DEBUG_BUMPS 2   /* also keep per-candidate bump bits (bump_bits) */
#define GD_FLAG_NO_FILTER 4     /* test every moving x static pair at every angle (no reach
                                   filter); results are identical, only slower */
#define GD_FLAG_MASK_SWEEP 8    /* sweep every step's angles over the reach filter's bit masks
                                   instead of its compacted near list (the path a step takes
                                   when the list overflows); results are identical */
#define GD_FLAG_TEST_STAGE_TIMEOUT 16 /* testing only: the pocket-staging barrier of kernels that
                                   stage the grid in shared memory expects 16 bytes more than
                                   are copied, so its bounded wait (about 2 s) runs out; the job
                                   then reports GD_ETIMEOUT and the context stays usable.
                                   Ignored by autotuning; rejected by gd_dock_batch_noalloc. */

typedef struct gd_ctx gd_ctx;
typedef struct gd_pocket gd_pocket;
typedef struct gd_job gd_job;

/* Ligand library in CSR form, host memory, owned by the caller.  The library copies
 * what it needs before gd_dock_batch returns.
 *   atom_off[L+1]  first atom of ligand i (atoms of ligand i: atom_off[i] .. atom_off[i+1]-1)
 *   xyz[3*N]       coordinates in Angstrom, x y z per atom
 *   bond_off[L+1]  first bond of ligand i
 *   bonds[2*B]     bond endpoints as ligand-local atom ids; the bonds of a ligand form a tree
 *   rot_off[L+1]   first rotamer of ligand i
 *   rot_bond[Rt]   rotamer r of ligand i = its bond rot_bond[rot_off[i]+r] (ligand-local),
 *                  swept in this order; a rotamer on a terminal bond is rejected. */
typedef struct {
  int32_t n_ligands;
  const int32_t* atom_off;
  const float* xyz;
  const int32_t* bond_off;
  const int32_t* bonds;
  const int32_t* rot_off;
  const int32_t* rot_bond;
} gd_ligand_batch;

/* Search settings.  Restart o = (i*n_beta + j)*n_gamma + k uses the ZYZ Euler angles
 * (2 pi i/n_alpha, pi (j+1/2)/n_beta, 2 pi k/n_gamma).  tile: 0 = built-in default
 * (an 8-warp tile: the 80-register kernel when three of its blocks fit in an SM's shared
 * memory, else the 128-register one, with fewer warps if 8 do not fit), -1 = autotuned
 * (cached per context), > 0 = a tile id from gd_tile_count(); the tile changes speed
 * only, never results.
 * rigid_span s > 0 adds the rigid alignment sweep of align_ligand (Sec. 3.1, 4.1) after
 * each restart's placement: the (2s+1)^3 rotations about the pocket centre by rotation
 * vectors rigid_step * (i-s, j-s, k-s), i, j, k in [0, 2s] (identity first, then the
 * others in (i, j, k) order), are scored rigidly and the best (ties: the earlier one)
 * is kept before optimize_pose.  s <= 3; 0 = off. */
typedef struct {
  int32_t n_alpha, n_beta, n_gamma;
  int32_t n_angles;
  float bump_dist;
  int32_t min_bond_sep;
  int32_t repetitions;
  int32_t flags;
  int32_t tile;
  int32_t rigid_span;
  float rigid_step;
} gd_search_params;

/* Results, caller-allocated host buffers (sizes from the batch it came from):
 *   best_score[L]          integer score of the best pose
 *   best_orient[L]         its restart index o
 *   best_angle[reps*Rt]    its angle index per step, ligand i at rot_off[i]*reps,
 *                          step = rep*R_i + r; -1 where every candidate was bumped
 *   best_xyz[3*N]          its final coordinates, atoms in input order
 *   evals[L]               candidates evaluated (O * reps * R_i * A)
 *   pair_tests[L]          moving x static pair tests performed: with the reach filter,
 *                          each step's near pairs at every angle; without it, every
 *                          eligible pair of each moving atom at every angle not yet
 *                          bumped (early exit per atom)
 *   atom_moves[L]          fragment atoms rotated and scored (O * reps * A * sum_r f_r,
 *                          f_r = atoms of fragment r)
 *   best_rigid[L]          rigid-sweep candidate kept for the best restart (0 without sweep)
 *   reach_tests[L]         moving x static pairs checked once per rotamer step by the
 *                          reach filter (a pair that cannot come within bump_dist at any
 *                          angle is not tested per angle)
 * Debug outputs (NULL to skip):
 *   orient_score[L*O]      final score of every restart            (GD_FLAG_DEBUG)
 *   orient_pick[O*reps*Rt] picks of every restart, ligand i at rot_off[i]*reps*O,
 *                          then o*reps*R_i + step                  (GD_FLAG_DEBUG)
 *   orient_rigid[L*O]      rigid-sweep candidate kept by every restart (GD_FLAG_DEBUG)
 *   bump_bits[sum_i O*reps*R_i*A]  1 if the candidate was bumped   (GD_FLAG_DEBUG_BUMPS), ligand i at
 *                          O*reps*A*rot_off[i], then ((o*reps*R_i + step)*A + k) */
typedef struct {
  uint32_t* best_score;
  int32_t* best_orient;
  int16_t* best_angle;
  float* best_xyz;
  uint64_t* evals;
  uint64_t* pair_tests;
  uint64_t* atom_moves;
  uint64_t* reach_tests;
  uint32_t* orient_score;
  int16_t* orient_pick;
  uint8_t* bump_bits;
  int16_t* best_rigid;
  int16_t* orient_rigid;
} gd_result_batch;

/* Create a context on CUDA device `device`.  mem_budget_bytes caps the device memory
 * the context may hold (0 = no cap). */
gd_status gd_create(gd_ctx** ctx, int device, size_t mem_budget_bytes);
/* Wait for the context's work and free everything it owns. */
gd_status gd_destroy(gd_ctx* ctx);
/* Thread-local reason of the last failure on this thread ("" if none). */
const char* gd_last_error(gd_ctx* ctx);

/* load(pocket), Listing 1: upload a uint8 score grid laid out [nz][ny][nx] (x fastest),
 * cell (i,j,k) covering origin + h*[i,i+1) x h*[j,j+1) x h*[k,k+1).  Cells outside the
 * grid score 0.  The grid is copied; the caller keeps ownership of `grid`. */
gd_status gd_load_pocket(gd_ctx* ctx, const uint8_t* grid, int nx, int ny, int nz, float spacing,
                         const float origin[3], gd_pocket** out);
gd_status gd_free_pocket(gd_ctx* ctx, gd_pocket* pocket);

/* Dock a ligand library (the outer loop of Listing 1).  Validates and packs the
 * batch, copies it to the device on `stream`, launches the search and queues the
 * copy of the results back; returns without waiting.  The caller may free `batch`
 * on return.  The job owns its device memory until gd_job_free. */
gd_status gd_dock_batch(gd_ctx* ctx, const gd_pocket* pocket, const gd_ligand_batch* batch,
                        const gd_search_params* params, void* stream, gd_job** out);
/* The first half of gd_dock_batch: validate, pack and copy the batch to the device on
 * `stream`, without searching.  Search it later with gd_job_launch (every restart) or
 * gd_job_launch_subset (chosen restarts), then gd_job_download + gd_fetch_results. */
gd_status gd_prepare_batch(gd_ctx* ctx, const gd_pocket* pocket, const gd_ligand_batch* batch,
                           const gd_search_params* params, void* stream, gd_job** out);
/* gd_prepare_batch over the ligands sel[0 .. n_sel) of `batch`, in that order, without
 * building a sub-batch: the job's ligand i is batch ligand sel[i] (a ligand may be
 * listed more than once), and its results are laid out as for a batch of those ligands.
 * Only the selected ligands are read and validated.  For a caller that keeps one large
 * library on the host and docks parts of it as they are needed (a streaming screen).
 * GD_EINVAL when an index is outside [0, n_ligands) or sel is NULL with n_sel > 0. */
gd_status gd_prepare_batch_sel(gd_ctx* ctx, const gd_pocket* pocket, const gd_ligand_batch* batch,
                               const int32_t* sel, int32_t n_sel, const gd_search_params* params, void* stream,
                               gd_job** out);
/* Copy a job's results into `out`.  blocking = 0 returns GD_ENOTREADY while the device
 * is still working. */
gd_status gd_fetch_results(gd_ctx* ctx, gd_job* job, gd_result_batch* out, int blocking);
/* Run the search of an existing job again on its device-resident inputs (no host
 * copies; the results stay on the device until gd_job_download). */
gd_status gd_job_launch(gd_ctx* ctx, gd_job* job, void* stream);
/* Queue the device-to-host copy of a job's current results (read with gd_fetch_results). */
gd_status gd_job_download(gd_ctx* ctx, gd_job* job, void* stream);
/* Bytes one gd_dock_batch of this job moves host->device (packed inputs) and
 * device->host (results, plus debug arrays when requested). */
gd_status gd_job_bytes(gd_ctx* ctx, const gd_job* job, uint64_t* h2d_bytes, uint64_t* d2h_bytes);
/* Launch shape of a job's search (the persistent launch of a3-a10): the tile it runs,
 * whether its kernel stages the pocket grid in shared memory (1: a bulk async copy per
 * block) or reads it through the texture / L1 path (0), and the blocks, threads per
 * block and dynamic shared memory per block of the launch (blocks = 0 for an empty
 * batch).  Any output pointer may be NULL. */
gd_status gd_job_info(gd_ctx* ctx, const gd_job* job, int* tile, int* grid_in_smem, int* blocks, int* threads,
                      size_t* smem_bytes);
/* Wait for the job's queued work and release it. */
gd_status gd_job_free(gd_ctx* ctx, gd_job* job);

/* Validate a batch and parameters on the host only, without a device: the checks
 * gd_dock_batch makes before it touches the GPU (tree bonds, atom/rotamer limits,
 * terminal rotamers, excluded-pair limit, finite coordinates, parameter ranges).
 * Returns GD_OK or GD_EINVAL with the reason in gd_last_error(NULL). */
gd_status gd_check_batch(const gd_ligand_batch* batch, const gd_search_params* params);

/* Launch tiles: number of ids (1..count) and, for one id, the warps per block, the
 * angles per lane and the register budget per thread of its kernel (128: the pocket
 * grid is staged in shared memory when it fits; 80: a little state spills to local
 * memory, but up to 24 warps stay resident per SM and the grid is read through the
 * texture path; 96: smaller per-warp buffers -- the rotamer descriptors and excluded pairs
 * read through L1, the turn's u x d term rebuilt per use -- so that about 20 warps with
 * the buffers of 250-atom ligands fit an SM).  Any output pointer may be NULL. */
int gd_tile_count(void);
gd_status gd_tile_info(int tile, int* warps_per_block, int* angles_per_lane, int* max_registers);
/* Time every tile on the batch (or its first max_ligands ligands) and return the
 * fastest; the choice is cached in the context for gd_search_params.tile = -1. */
gd_status gd_autotune(gd_ctx* ctx, const gd_pocket* pocket, const gd_ligand_batch* batch,
                      const gd_search_params* params, int max_ligands, void* stream, int* best_tile,
                      float* best_ms);

/* Peaks of the pipes that bound the search kernel, measured on `device` (made the
 * calling thread's current device) by two microbenchmarks launched on `stream`
 * (NULL: the legacy default stream): every SM full of 256-thread blocks, enough
 * independent work per warp to hide latency, best of three timed launches, about 50 ms
 * in all.  *ffma_per_s: FP32 fused multiply-adds per second, counted per lane (the unit
 * of the search's algorithmic FP32 count); *lds_u8_per_s: shared-memory byte loads per
 * second, counted per lane.  Either pointer may be NULL.  GD_ECUDA on a CUDA failure;
 * no device memory stays allocated. */
gd_status gd_measure_peaks(int device, void* stream, double* ffma_per_s, double* lds_u8_per_s);

/* ---- Streaming server: continuous batching into one persistent launch -------------
 * The paper's hybrid version hands each ligand to whichever thread becomes free (Sec. 4.2,
 * Listing 3: one task per ligand), and its MPI master sends a node new ligands as soon as
 * it finishes the last ones (Sec. 5); here ligands that arrive over time join a search
 * launch that is already running.  A server owns `capacity` slots
 * for ligands of at most max_atoms atoms, max_rotamers rotamers and max_excluded excluded
 * pairs in all (0: 16 per rotamer), in device memory counted against the context's
 * budget, plus mapped (zero-copy) host memory for its ligand records, results and
 * control words.  gd_server_submit validates and packs ligands into free slots on the
 * host and publishes them; a persistent launch on the server's own stream takes work,
 * 4 restarts of one ligand at a time, as soon as it is published, copies each ligand's record into
 * its slot when it starts the first of them, searches every restart exactly as gd_dock_batch
 * does (same results, bit for bit) and writes each ligand's results to host memory as soon
 * as its last restart is done.  A launch ends once every one of its warps has waited
 * `idle_ms` without work (work that arrives as it ends waits for the next launch); any
 * later call that finds published work unfinished launches it again.  Waits on the device are bounded by the SM
 * clock: a warp that waits longer than about 0.5 s for a slot being staged sets an error,
 * which the next gd_server_poll / gd_server_collect reports as GD_ETIMEOUT (the server
 * must then be destroyed; the context stays usable); a blocking gd_server_poll gives up
 * with GD_ETIMEOUT after 30 s without the result.  tile: 0 = the wide tile with the most warps
 * whose buffers, sized for the server's largest ligand, fit a block; > 0 a lean or wide
 * tile (compact tiles, 16-20, are rejected).  Destroy a server before its pocket and its
 * context.  Not thread-safe: one host thread per
 * server, or external locking.
 * Results of ligand seq (numbered from 0 in submission order): gd_server_poll copies them
 * into a one-ligand gd_result_batch (best_score[1], best_orient[1], best_angle[reps*R],
 * best_xyz[3*n], counters[1]; debug arrays must be NULL) and frees the slot;
 * gd_server_collect returns the score and best restart of every finished ligand not
 * yet returned, oldest first, and frees their slots.  A slot is reused only after its
 * ligand's results were returned; gd_server_submit answers GD_EBUSY when fewer than
 * n_sel slots are free. */
typedef struct gd_server gd_server;
gd_status gd_server_create(gd_ctx* ctx, const gd_pocket* pocket, const gd_search_params* params, int capacity,
                           int max_atoms, int max_rotamers, int max_excluded, int idle_ms, gd_server** out);
/* Submit ligands sel[0 .. n_sel) of `batch` (sel NULL: all of it, in order); the first gets
 * sequence number *first_seq, the others the following ones. */
gd_status gd_server_submit(gd_server* srv, const gd_ligand_batch* batch, const int32_t* sel, int32_t n_sel,
                           uint64_t* first_seq);
/* As gd_server_submit, but ligand i of the submission searches only the restarts
 * restarts[i * stride .. + n_restarts[i]) (host memory, copied before the call returns;
 * distinct ids in [0, O), 1 <= n_restarts[i] <= min(O, stride)), as gd_job_launch_proposed
 * does for the restarts a selection chose: its results are the best over those restarts
 * (ties to the smaller restart), bit for bit what the proposed search gives for the same
 * restarts, and its counters count those restarts.  This is the learned screen's path
 * into the running launch (Sec. 3.1's restart loop over a subset of the restarts). */
gd_status gd_server_submit_restarts(gd_server* srv, const gd_ligand_batch* batch, const int32_t* sel, int32_t n_sel,
                                    const uint16_t* restarts, const int32_t* n_restarts, int32_t stride,
                                    uint64_t* first_seq);
/* Leave free_sms of the device's SMs out of the server's launch, for other kernels that
 * run beside it (e.g. the proposer's features and network for the next arrivals).  They
 * stay free when the server's tile holds one block per SM (a wide tile whose buffers need
 * most of an SM's shared memory); with smaller blocks it only shrinks the launch.  Call it
 * before the first submission (GD_EBUSY afterwards); GD_EINVAL unless 0 <= free_sms < SMs. */
gd_status gd_server_reserve_sms(gd_server* srv, int free_sms);
/* Results of ligand seq; blocking = 0 returns GD_ENOTREADY while it is searched. */
gd_status gd_server_poll(gd_server* srv, uint64_t seq, gd_result_batch* out, int blocking);
/* Up to max finished ligands: their sequence numbers, best scores and best restarts (any
 * output pointer may be NULL); *n_out of them. */
gd_status gd_server_collect(gd_server* srv, uint64_t* seq, uint32_t* best_score, int32_t* best_orient, int max,
                            int* n_out);
/* Counters: launches started, launches that ended idle, ligands published, ligands whose
 * results were returned, work-item tickets taken on the device (4 restarts each; up to
 * one per warp runs ahead of the published work) and reads of the mapped control words by
 * the device.  Any pointer may be NULL. */
gd_status gd_server_stats(gd_server* srv, uint64_t* launches, uint64_t* idle_exits, uint64_t* published,
                          uint64_t* finished, uint64_t* claimed_items, uint64_t* control_reads);
/* Testing only: the slot of ligand hold_seq is never released to the warps that wait
 * for it, so their bounded waits run out (0.2 s here) and the server reports GD_ETIMEOUT;
 * -1 turns it off.  Takes effect for ligands submitted afterwards. */
gd_status gd_server_test_hold(gd_server* srv, int64_t hold_seq);
/* Stop the launch once every published ligand has been claimed, wait for it and free
 * everything. */
gd_status gd_server_destroy(gd_server* srv);

/* ---- Docking without allocation --------------------------------------------------
 * The paper has no counterpart: this serves callers that cannot allocate device memory
 * when they dock -- a process whose device memory is already fully reserved by
 * another framework's caching allocator, a service that forbids allocation after
 * start-up so its memory footprint stays fixed, or code that must avoid cudaMalloc /
 * cudaFree because they synchronise the whole device.
 *
 * gd_dock_batch_noalloc docks like gd_dock_batch + gd_fetch_results (same search
 * kernel, same results) but calls no cudaMalloc, cudaFree, cudaMallocHost or other
 * allocating routine and needs no context.  Its working memory -- the cropped pocket
 * grid, the packed ligands, the results and the kernel's scratch (per-restart scores,
 * picks and counters) -- is one file-scope __device__ array of GD_NOALLOC_MAX_BYTES
 * (64 MiB) that every GPU which loads the library holds until the process exits, plus
 * a host staging array of the same size.  Inputs: the pocket grid and the batch in
 * host memory (layouts as for gd_load_pocket / gd_ligand_batch); outputs: the caller's
 * host buffers of `out` (debug arrays must be NULL; GD_FLAG_DEBUG* are rejected).
 * The call is synchronous on `stream` (results are in `out` on return).
 * Limits: a batch whose grid, inputs, results and scratch need more than
 * GD_NOALLOC_MAX_BYTES is rejected with GD_EINVAL (about 20*L*O + 2*O*reps*Rt +
 * 300*Rt + 48*N + 64*L bytes plus the cropped grid); tile -1 (autotuned) is rejected,
 * since there is no context to keep an autotuned choice (0 = the built-in default, or a
 * tile id); rigid_span must be 0.  Ligands and parameters are validated by the same code
 * as gd_dock_batch and gd_check_batch, with the same messages.
 * Set-up: the first call on a device (the current device) looks up the array's device
 * address with cudaGetSymbolAddress; make that first call before any stream capture.
 * Concurrency: every call shares the one array and its contents persist between calls
 * (the kernel clears what must start at zero), so calls that overlap on the GPU -- from
 * two threads, or on two streams -- race and must be serialised by the caller.
 * err_msg (optional, err_len bytes) receives a one-line reason on failure. */
#define GD_NOALLOC_MAX_BYTES (64u << 20)
gd_status gd_dock_batch_noalloc(const uint8_t* grid, int nx, int ny, int nz, float spacing,
                                const float origin[3], const gd_ligand_batch* batch,
                                const gd_search_params* params, gd_result_batch* out, void* stream,
                                char* err_msg, size_t err_len);

#ifdef __cplusplus
}
#endif
#endif /* GEODOCK_H */
