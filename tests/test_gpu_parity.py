"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Small workloads are compared element by element (every restart's picks and score,
every candidate's bump flag); the full-size workloads run in the benchmark's launch
configuration and are compared on sampled ligands and restarts.
"""
import numpy as np
import pytest

import oracle
from paper_1901_06229_b300 import geodock as gdk
from paper_1901_06229_b300 import synth
from parity import Stats, check_ligand, check_pose_vs_oracle, compare_debug
from test_oracle_pins import modular_pocket, textured_pocket

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = gdk.Context(0)
    yield c
    c.close()


def run(ctx, w_pocket, batch, params, debug=True, bumps=True, tile=0, no_filter=False, mask_sweep=False,
        info=None):
    pk = ctx.load_pocket(w_pocket)
    job = ctx.dock_batch(pk, batch, params, debug=debug, bumps=bumps, tile=tile, no_filter=no_filter,
                         mask_sweep=mask_sweep)
    out = job.fetch()
    if info is not None and batch.n_ligands:
        info.update(job.info())
    job.free()
    pk.free()
    return out


# Least share of a workload's rotamer steps that must be compared with the oracle: the
# rest are steps after a restart legitimately parted from the oracle's trajectory at a
# fragile step.  Measured shares are printed with every comparison.
MIN_COMPARED = 0.95


def full_compare(ctx, pocket, batch, params, tile=0, min_exact=1, no_filter=False, mask_sweep=False,
                 min_compared=MIN_COMPARED, info=None):
    gpu = run(ctx, pocket, batch, params, tile=tile, no_filter=no_filter, mask_sweep=mask_sweep, info=info)
    orc = oracle.dock_batch(batch, pocket, params, n_threads=8, debug=True)
    st = compare_debug(gpu, orc, batch, params)
    print(dict(st), "compared", st.compared_fraction())
    assert st.get("scores_exact", 0) >= min_exact
    if st.get("steps_total", 0):
        assert st.compared_fraction() >= min_compared, st.compared_fraction()
    return gpu, orc, st


def test_single_ligand_workload(ctx):
    w = synth.workload_single()
    _, _, st = full_compare(ctx, w.pocket, w.batch, w.params)
    assert st["restarts"] == 64


def test_single_ligand_textured_pocket(ctx):
    w = synth.workload_single()
    gpu, orc, st = full_compare(ctx, textured_pocket(), w.batch, w.params, min_exact=40)
    assert (orc["orient_pick"] > 0).sum() > 20, "pocket should make the search move fragments"


def test_modular_grid_many_boundaries(ctx):
    P = modular_pocket(40, 40, 40, 0.5, origin=(-10.0, -10.0, -10.0))
    lig = [synth.gen_ligand(synth.SplitMix64(synth.ligand_seed(99, s)), 18, 3) for s in range(3)]
    full_compare(ctx, P, synth.pack(lig), synth.SearchParams(2, 3, 2, 32), min_exact=10)


def test_batched_subset_elementwise(ctx):
    w = synth.workload_batched(24)
    _, _, st = full_compare(ctx, w.pocket, w.batch, w.params, min_exact=1000)
    assert st["restarts"] == 24 * 256


@pytest.mark.parametrize("tile", [0, 16, 17])
def test_large_ligands_reduced_restarts(ctx, tile):
    """Large ligands against the oracle with the default tile and the compact builds
    (96 registers, descriptors read through L1, (u x d) rebuilt from the axis frame)."""
    w = synth.workload_large(6)
    params = synth.SearchParams(2, 2, 2, 128)
    _, _, st = full_compare(ctx, w.pocket, w.batch, params, min_exact=40, tile=tile)
    assert st["restarts"] == 48


@pytest.mark.parametrize("tile", [1, 2, 3, 10])
@pytest.mark.parametrize("which", ["single", "batched"])
def test_grid_staged_in_shared_memory_matches_oracle(ctx, which, tile):
    """The 128-register tiles stage the cropped pocket grid into each block's shared
    memory by bulk async copies (32 KB single-ligand crop, 162.6 KB batched crop): every
    pick, bump flag and score against the oracle, with the staging checked on the job."""
    w = synth.workload_single() if which == "single" else synth.workload_batched(24)
    info = {}
    _, _, st = full_compare(ctx, w.pocket, w.batch, w.params, tile=tile, min_exact=50, info=info)
    print(info)
    assert info["grid_in_smem"] and info["tile"] == tile
    assert st["restarts"] == w.batch.n_ligands * w.params.n_orient


def dense_exclusion_ligand(seed, min_sep, n_atoms=256, n_rot=128):
    """A tree whose rotamers are the internal bonds with the most excluded pairs that
    stay within the per-rotamer (128) and per-atom (32) limits at ``min_sep``."""
    import collections
    lig = synth.gen_ligand(synth.SplitMix64(synth.ligand_seed(4242, seed)), n_atoms, 0)
    adj = collections.defaultdict(list)
    for u, v in lig.bonds.tolist():
        adj[u].append(v)
        adj[v].append(u)

    def hops(src, block):  # bond distance from src, not crossing to block
        d, q = {src: 0}, collections.deque([src])
        while q:
            u = q.popleft()
            for v in adj[u]:
                if v != block and v not in d:
                    d[v] = d[u] + 1
                    q.append(v)
        return d

    ranked = []
    for e, (p, q) in enumerate(lig.bonds.tolist()):
        if len(adj[p]) < 2 or len(adj[q]) < 2:
            continue
        a, b = hops(q, p), hops(p, q)
        pairs = [(m, t) for m, dm in a.items() for t, dt in b.items() if dm + dt + 1 < min_sep]
        per_atom = collections.Counter(m for m, _ in pairs) + collections.Counter(t for _, t in pairs)
        if len(pairs) <= 128 and max(per_atom.values()) <= 32:
            ranked.append((-len(pairs), e))
    chosen = sorted(e for _, e in sorted(ranked)[:n_rot])
    return synth.Ligand(lig.xyz, lig.bonds, np.asarray(chosen, np.int32)), -sum(c for c, _ in sorted(ranked)[:n_rot])


@pytest.mark.parametrize("case", ["ragged_angles", "one_angle", "odd_euler", "reps2", "min_sep4",
                                  "bump25", "rigid_only", "two_atoms", "max_atoms", "rigid_sweep",
                                  "rigid_sweep_span2", "max_exclusions", "max_angles", "many_restarts",
                                  "max_reps"])
def test_edge_cases(ctx, case):
    pocket = textured_pocket()
    rng = lambda s: synth.SplitMix64(synth.ligand_seed(4242, s))
    ligs = [synth.gen_ligand(rng(s), n, r) for s, (n, r) in enumerate([(20, 3), (31, 5), (14, 2)])]
    params = synth.SearchParams(2, 2, 2, 40)
    if case == "ragged_angles":
        params = synth.SearchParams(2, 2, 2, 33)
    elif case == "one_angle":
        params = synth.SearchParams(2, 2, 2, 1)
    elif case == "odd_euler":
        params = synth.SearchParams(3, 5, 2, 32)
    elif case == "reps2":
        params = synth.SearchParams(2, 2, 2, 32, repetitions=2)
    elif case == "min_sep4":
        params = synth.SearchParams(2, 2, 2, 32, min_bond_sep=4)
    elif case == "bump25":
        params = synth.SearchParams(2, 2, 2, 32, bump_dist=2.5)
    elif case == "rigid_only":
        ligs = [synth.gen_ligand(rng(10 + s), 12, 0) for s in range(3)]
        params = synth.SearchParams(4, 4, 4, 32)
    elif case == "two_atoms":
        ligs = [synth.gen_ligand(rng(20), 2, 0), synth.gen_ligand(rng(21), 9, 1)]
    elif case == "rigid_sweep":
        params = synth.SearchParams(2, 2, 2, 32, rigid_span=1, rigid_step=0.12)
    elif case == "rigid_sweep_span2":
        params = synth.SearchParams(2, 2, 2, 32, repetitions=2, rigid_span=2, rigid_step=0.07)
    elif case == "max_atoms":
        big = synth.workload_large(1).pocket
        ligs = [synth.gen_ligand(rng(30), 256, 40)]
        pocket, params = big, synth.SearchParams(1, 2, 1, 64)
    elif case == "max_angles":  # GD_MAX_ANGLES: a step sweeps its angles in 16 passes of 64
        params = synth.SearchParams(1, 2, 1, 1024)
    elif case == "many_restarts":  # 1,000 restarts (10 x 10 x 10), ragged against the work chunks
        params = synth.SearchParams(10, 10, 10, 16)
    elif case == "max_reps":  # GD_MAX_REPS repetitions of the rotamer loop
        params = synth.SearchParams(1, 2, 1, 24, repetitions=16)
    elif case == "max_exclusions":  # 128 rotamers, ~7.7k excluded pairs: ~205 KB of warp buffers
        lig, n_excl = dense_exclusion_ligand(60, 7)
        assert len(lig.rot_bond) == 128 and n_excl > 7000
        ligs = [lig]
        pocket, params = synth.workload_large(1).pocket, synth.SearchParams(2, 2, 2, 64, min_bond_sep=7)
    full_compare(ctx, pocket, synth.pack(ligs), params, min_exact=1)


def test_rigid_sweep_on_the_batched_workload(ctx):
    w = synth.workload_batched(16)
    p = w.params
    params = synth.SearchParams(p.n_alpha, p.n_beta, p.n_gamma, p.n_angles, rigid_span=1, rigid_step=0.1)
    gpu, orc, st = full_compare(ctx, w.pocket, w.batch, params, min_exact=1000)
    assert st.get("rigid_compared", 0) > 1000
    assert (orc["orient_rigid"] != 0).mean() > 0.1  # the sweep moves many restarts


def test_unfiltered_sweep_matches_oracle(ctx):
    w = synth.workload_batched(12)
    full_compare(ctx, w.pocket, w.batch, w.params, min_exact=1000, no_filter=True)


@pytest.mark.parametrize("which", ["batched", "large", "min_sep4", "bump25"])
def test_reach_filter_is_exact(ctx, which):
    """The per-rotamer reach filter only skips pair tests that cannot fire: every output
    but the work counters is bitwise identical to testing every pair at every angle."""
    if which == "batched":
        w = synth.workload_batched(48)
        pocket, batch, params = w.pocket, w.batch, w.params
    else:
        w = synth.workload_large(4)
        pocket, batch = w.pocket, w.batch
        params = synth.SearchParams(2, 2, 2, 128)
        if which == "min_sep4":
            params = synth.SearchParams(2, 2, 2, 64, min_bond_sep=4)
        elif which == "bump25":
            params = synth.SearchParams(2, 2, 2, 64, bump_dist=2.5)
    a = run(ctx, pocket, batch, params, no_filter=False)
    b = run(ctx, pocket, batch, params, no_filter=True)
    m = run(ctx, pocket, batch, params, mask_sweep=True)
    for k in a:
        np.testing.assert_array_equal(a[k], m[k], err_msg=f"mask sweep: {k}")  # counters too
        if k in ("pair_tests", "reach_tests"):
            continue
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    assert a["pair_tests"].sum() < b["pair_tests"].sum()
    assert b["reach_tests"].sum() == 0 and a["reach_tests"].sum() > 0


@pytest.mark.parametrize("tile", [9, 14, 16])
def test_mask_sweep_matches_oracle(ctx, tile):
    """The overflow path of the reach filter (sweeping its bit masks) against the oracle,
    on ligands whose static side spans several 32-atom mask words."""
    w = synth.workload_large(3)
    full_compare(ctx, w.pocket, w.batch, synth.SearchParams(2, 2, 2, 64), tile=tile, min_exact=4, mask_sweep=True)


def _near_pairs(x, lig, rb, params):
    """Reach-filter count of rotamer bond rb at coordinates x (FP64, on the CPU): moving x
    static pairs at bond separation >= min_bond_sep whose (h, rho) about the bond axis
    lie within bump_dist + 0.01 A."""
    mv, p, q, dist = oracle.fragment(len(x), lig.bonds, rb)
    u = (x[q] - x[p]) / np.linalg.norm(x[q] - x[p])
    r = x - x[p]
    h = r @ u
    rho = np.sqrt(np.maximum((r * r).sum(1) - h * h, 0.0))
    A, B = np.nonzero(mv)[0], np.nonzero(~mv)[0]
    d2 = (h[A, None] - h[None, B]) ** 2 + (rho[A, None] - rho[None, B]) ** 2
    return int(((d2 < (params.bump_dist + 0.01) ** 2) & (dist[np.ix_(A, B)] >= params.min_bond_sep)).sum())


def test_near_list_overflow_takes_the_mask_sweep(ctx):
    """A step whose near pairs exceed the list (8 x n_max) sweeps the bit masks instead:
    results equal the forced mask sweep and the oracle."""
    lig = synth.gen_ligand(synth.SplitMix64(synth.ligand_seed(4343, 96)), 96, 12)
    small = synth.gen_ligand(synth.SplitMix64(synth.ligand_seed(4343, 40)), 40, 5)
    batch, pocket = synth.pack([lig, small]), textured_pocket()
    params = synth.SearchParams(2, 2, 2, 32, bump_dist=3.5)
    # the first step of every restart starts from a rigid motion of the input pose
    x0 = oracle.place(lig.xyz, 0, params, pocket)
    assert _near_pairs(x0, lig, int(lig.rot_bond[0]), params) > 8 * 96 + 100
    a = run(ctx, pocket, batch, params)
    m = run(ctx, pocket, batch, params, mask_sweep=True)
    for k in a:
        np.testing.assert_array_equal(a[k], m[k], err_msg=k)
    full_compare(ctx, pocket, batch, params, min_exact=1)


def test_empty_batch(ctx):
    w = synth.workload_single()
    out = run(ctx, w.pocket, synth.pack([]), w.params)
    assert len(out["best_score"]) == 0


def test_all_zero_pocket(ctx):
    w = synth.workload_single()
    zero = synth.Pocket(grid=np.zeros((8, 9, 10), np.uint8), spacing=0.5, origin=np.zeros(3, np.float32))
    out = run(ctx, zero, w.batch, w.params)
    assert out["best_score"][0] == 0 and out["best_orient"][0] == 0
    assert np.all(out["orient_score"] == 0) and np.all(out["orient_pick"] <= 0)


def test_tiles_give_identical_results(ctx):
    w = synth.workload_batched(32)
    ref = None
    for t in range(1, gdk.tile_count() + 1):
        out = run(ctx, w.pocket, w.batch, w.params, tile=t)
        if ref is None:
            ref = out
            continue
        for k in ref:
            if k in ("pair_tests", "reach_tests"):  # work counters depend on the early exit
                continue
            np.testing.assert_array_equal(out[k], ref[k], err_msg=f"tile {t}: {k}")


def test_relaunch_on_resident_inputs_is_deterministic(ctx):
    import torch
    w = synth.workload_batched(16)
    pk = ctx.load_pocket(w.pocket)
    s = torch.cuda.Stream()
    job = ctx.dock_batch(pk, w.batch, w.params, stream=s, debug=True)
    first = job.fetch()
    for _ in range(3):
        job.launch(stream=s)
    job.download(stream=s)
    again = job.fetch()
    for k in first:
        np.testing.assert_array_equal(first[k], again[k], err_msg=k)
    job.free()
    pk.free()


def _subset(gpu, batch, params, idx):
    """Results of a GPU run restricted to ligands idx, laid out as for batch.subset(idx)."""
    O, reps = params.n_orient, params.repetitions
    ro, ao = np.asarray(batch.rot_off, np.int64), np.asarray(batch.atom_off, np.int64)
    out = {k: [] for k in ("best_score", "best_orient", "best_angle", "best_xyz", "evals", "pair_tests",
                           "atom_moves", "orient_score", "orient_pick")}
    for i in idx:
        for k in ("best_score", "best_orient", "evals", "pair_tests", "atom_moves"):
            out[k].append(gpu[k][i:i + 1])
        out["orient_score"].append(gpu["orient_score"][i:i + 1])
        out["best_angle"].append(gpu["best_angle"][ro[i] * reps: ro[i + 1] * reps])
        out["best_xyz"].append(gpu["best_xyz"][ao[i]: ao[i + 1]])
        out["orient_pick"].append(gpu["orient_pick"][ro[i] * reps * O: ro[i + 1] * reps * O])
    return {k: np.concatenate(v) for k, v in out.items()}


def test_full_size_batched_sampled(ctx):
    """4,096 ligands, 256 restarts, 64 angles, autotuned tile (the benchmark's launch)."""
    w = synth.workload_batched(4096)
    gpu = run(ctx, w.pocket, w.batch, w.params, debug=True, bumps=False, tile=-1)
    idx = np.random.default_rng(7).choice(4096, size=48, replace=False)
    sub = w.batch.subset(idx)
    orc = oracle.dock_batch(sub, w.pocket, w.params, n_threads=8, debug=False)
    st = compare_debug(_subset(gpu, w.batch, w.params, idx), orc, sub, w.params, bumps=False)
    print(dict(st), "compared", st.compared_fraction())
    assert st["scores_exact"] > 0.9 * st["restarts"]
    assert st.compared_fraction() >= MIN_COMPARED
    # properties that hold for every ligand of the batch
    assert np.all(gpu["best_score"] == gpu["orient_score"].max(axis=1))
    assert np.all(gpu["best_orient"] == gpu["orient_score"].argmax(axis=1))
    R = np.diff(w.batch.rot_off)
    assert np.all(gpu["evals"] == 256 * 64 * R)


def test_full_size_large_sampled(ctx):
    """512 ligands of 100-250 atoms, 128^3 pocket (texture grid path), 128 angles, the
    benchmark's autotuned launch: 64 sampled ligands x 8 restarts (the ligand's best and 7
    drawn at random) against oracle.dock_pose, step by step along the oracle's trajectory."""
    from concurrent.futures import ThreadPoolExecutor
    w = synth.workload_large(512)
    gpu = run(ctx, w.pocket, w.batch, w.params, debug=True, bumps=False, tile=-1)
    st = Stats()
    rng = np.random.default_rng(11)
    cases = []
    for i in rng.choice(512, size=64, replace=False):
        best = int(gpu["best_orient"][i])
        others = [int(o) for o in rng.choice(np.setdiff1d(np.arange(256), [best]), size=7, replace=False)]
        cases += [(int(i), o, o == best) for o in [best] + others]

    def one(case):
        i, o, is_best = case
        ref, same = check_pose_vs_oracle(gpu, w.batch, w.params, w.pocket, i, o, Stats(), oracle)
        return ref, same

    # the oracle releases the GIL: one pose per thread (statistics are summed below)
    with ThreadPoolExecutor(8) as ex:
        results = list(ex.map(one, cases))
    coords = 0
    for (i, o, is_best), (ref, same) in zip(cases, results):
        check_pose_vs_oracle(gpu, w.batch, w.params, w.pocket, i, o, st, _Cached(ref))
        if is_best and same:
            a0, a1 = w.batch.atom_off[i], w.batch.atom_off[i + 1]
            d = np.abs(gpu["best_xyz"][a0:a1] - ref["xyz"]).max()
            assert d <= 1e-4, d
            coords += 1
    print(dict(st), "compared", st.compared_fraction(), "coordinates", coords)
    assert st["sampled_restarts"] == 512
    assert st.compared_fraction() >= MIN_COMPARED
    assert coords >= 48
    assert np.all(gpu["best_score"] == gpu["orient_score"].max(axis=1))


class _Cached:
    """Stands in for the oracle module with one precomputed dock_pose result."""

    def __init__(self, ref):
        self.ref = ref

    def dock_pose(self, *args, **kw):
        return self.ref
