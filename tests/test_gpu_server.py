"""The streaming server: ligands submitted over time join one running search launch.

Each result must be bit-for-bit what gd_dock_batch gives the same ligand (the server runs
the same search on its slots), whether the ligand is submitted alone or while others are
being searched, when slots are reused, and across launches that end idle and start
again.  A slot held back on the device (test hook) makes the bounded waits run out: the
server then reports GD_ETIMEOUT and the context stays usable.
"""
import time

import numpy as np
import pytest

from paper_1901_06229_b300 import geodock as gdk
from paper_1901_06229_b300 import synth

pytestmark = pytest.mark.gpu

KEYS = ("best_score", "best_orient", "best_angle", "best_xyz", "evals", "pair_tests", "atom_moves", "reach_tests",
        "best_rigid")


@pytest.fixture(scope="module")
def ctx():
    c = gdk.Context(0)
    yield c
    c.close()


def _alone(ctx, pk, batch, params, i):
    job = ctx.dock_batch(pk, batch.subset([i]), params)
    out = job.fetch()
    job.free()
    return out


def _same(got, ref, what):
    for k in KEYS:
        np.testing.assert_array_equal(got[k], ref[k], err_msg=f"{what}: {k}")


def test_results_equal_dock_batch_alone_and_in_the_mix(ctx):
    w = synth.workload_stream(96, seed_offset=70)
    pk = ctx.load_pocket(w.pocket)
    srv = gdk.Server(ctx, pk, w.params, capacity=256, max_atoms=256, max_rotamers=48)
    # one ligand alone, then the rest in waves that arrive while earlier ones are searched
    s0 = srv.submit(w.batch, [0])
    alone = srv.poll(s0)
    seqs = {}
    order = np.random.default_rng(3).permutation(np.arange(1, 96))
    for wave in np.array_split(order, 6):
        first = srv.submit(w.batch, wave)
        for k, i in enumerate(wave):
            seqs[first + k] = int(i)
        time.sleep(0.002)
    got = {q: srv.poll(q) for q in sorted(seqs)}
    print(srv.stats())
    ref = ctx.dock_batch(pk, w.batch, w.params).fetch()
    ao, ro = np.asarray(w.batch.atom_off), np.asarray(w.batch.rot_off)
    view = lambda r, i: dict(best_score=r["best_score"][i:i + 1], best_orient=r["best_orient"][i:i + 1],
                             best_angle=r["best_angle"][ro[i]:ro[i + 1]], best_xyz=r["best_xyz"][ao[i]:ao[i + 1]],
                             evals=r["evals"][i:i + 1], pair_tests=r["pair_tests"][i:i + 1],
                             atom_moves=r["atom_moves"][i:i + 1], reach_tests=r["reach_tests"][i:i + 1],
                             best_rigid=r["best_rigid"][i:i + 1])
    _same(alone, view(ref, 0), "ligand 0 alone")
    _same(alone, _alone(ctx, pk, w.batch, w.params, 0), "ligand 0 as a one-ligand batch")
    for q, i in seqs.items():
        _same(got[q], view(ref, i), f"ligand {i} in the mix")
    srv.close()
    pk.free()


def test_slots_are_reused_and_idle_launches_restart(ctx):
    w = synth.workload_stream(80, seed_offset=71)
    pk = ctx.load_pocket(w.pocket)
    srv = gdk.Server(ctx, pk, w.params, capacity=16, max_atoms=256, max_rotamers=48, idle_ms=20)
    ref = ctx.dock_batch(pk, w.batch, w.params).fetch()
    got_s, got_o, first_of = {}, {}, {}
    nxt = done = 0
    t_end = time.time() + 60
    for phase_end in (40, 80):  # between the phases the launch runs out of work and ends
        while done < phase_end:
            assert time.time() < t_end, (done, nxt, srv.stats())
            while nxt < phase_end:
                try:
                    q = srv.submit(w.batch, [nxt])
                except gdk.GeoDockError as e:
                    assert e.status == gdk.GD_EBUSY  # all 16 slots hold unreturned ligands
                    break
                first_of[q] = nxt
                nxt += 1
            seq, sc, ob = srv.collect()
            for q, a, b in zip(seq.tolist(), sc.tolist(), ob.tolist()):
                got_s[first_of[q]], got_o[first_of[q]] = a, b
            done += len(seq)
        time.sleep(0.1)
    st = srv.stats()
    print(st)
    assert st["launches"] >= 2 and st["idle_exits"] >= 1 and st["finished"] == 80
    np.testing.assert_array_equal([got_s[i] for i in range(80)], ref["best_score"])
    np.testing.assert_array_equal([got_o[i] for i in range(80)], ref["best_orient"])
    small = gdk.Server(ctx, pk, w.params, capacity=4, max_atoms=20, max_rotamers=8)
    with pytest.raises(gdk.GeoDockError) as e:  # a ligand larger than the server's slots
        small.submit(w.batch, [int(np.argmax(np.diff(w.batch.atom_off)))])
    assert e.value.status == gdk.GD_EINVAL
    small.close()
    srv.close()
    pk.free()


def test_ligands_published_while_idle_warps_park_their_tickets(ctx):
    """Batches arriving just as the idle launch's warps give up: warps claimed their
    tickets at different times (some at once, some after their last item), so they run
    out of idle time one after another, and a batch published in between must neither
    find a ligand's first item parked by a warp that has left while live warps hold its
    later items (the launch closes only when every warp is idle, and the first warp to
    reach a ligand stages it), nor lose the items of a batch published as the launch
    closes (parked, taken up by the next launch).  No wait runs out and every result is
    gd_dock_batch's.  The arrival time sweeps from half an idle timeout after a batch's
    last result to past the launch's close."""
    w = synth.workload_stream(48, seed_offset=73)
    pk = ctx.load_pocket(w.pocket)
    idle_ms = 10
    srv = gdk.Server(ctx, pk, w.params, capacity=64, max_atoms=256, max_rotamers=48, idle_ms=idle_ms)
    ref = ctx.dock_batch(pk, w.batch, w.params).fetch()
    cycles = 30
    t_batch = 0.0
    for c in range(cycles):
        t_sub = time.perf_counter()
        first = srv.submit(w.batch)
        got = {}
        while len(got) < 48:
            assert time.perf_counter() < t_sub + 30, (c, len(got), srv.stats())
            seq, sc, ob = srv.collect()
            for q, a, b in zip(seq.tolist(), sc.tolist(), ob.tolist()):
                got[q - first] = (a, b)
        t_batch += time.perf_counter() - t_sub
        np.testing.assert_array_equal([got[i][0] for i in range(48)], ref["best_score"], err_msg=f"cycle {c}")
        np.testing.assert_array_equal([got[i][1] for i in range(48)], ref["best_orient"], err_msg=f"cycle {c}")
        # the next batch lands between 0.5 and 2 idle timeouts after this one's last result
        wake = time.perf_counter() + 1e-3 * idle_ms * (0.5 + 1.5 * c / (cycles - 1))
        while time.perf_counter() < wake:
            pass
    st = srv.stats()
    print(st, "batch ms", round(1e3 * t_batch / cycles, 2))
    assert st["finished"] == 48 * cycles and st["launches"] >= 2
    srv.close()
    pk.free()


def test_restart_lists_match_the_proposed_search(ctx):
    """Ligands submitted with restart lists (gd_server_submit_restarts) search only those
    restarts: every result is bit for bit what gd_job_launch_proposed gives when its
    selection picks the same restarts -- predictions made so that the top 16 are a
    ligand's list of 16, or so that the top-16 spread sends it to its best 128, its list
    of 128 -- alone and in the mix, with SMs left out of the launch."""
    import torch
    L, O = 64, 256
    w = synth.workload_stream(L, seed_offset=74)
    pk = ctx.load_pocket(w.pocket)
    rng = np.random.default_rng(5)
    lists = np.zeros((L, 128), np.uint16)
    counts = np.where(rng.random(L) < 0.25, 128, 16).astype(np.int32)
    pred = np.zeros((L, O), np.float32)
    for i in range(L):
        k = int(counts[i])
        chosen = rng.choice(O, size=k, replace=False)
        lists[i, :k] = chosen
        # decreasing in list order: a spread of 0.015 over a list of 16 (no fallback at
        # margin 0.5), of 1.05 over the first 16 of a list of 128 (fallback to its 128)
        pred[i, chosen] = (1.0 - 0.001 * np.arange(k)) if k == 16 else (10.0 - 0.07 * np.arange(k))
    job = ctx.prepare_batch(pk, w.batch, w.params)
    y = torch.tensor(pred.reshape(-1), device="cuda")
    job.launch_proposed(y, 16, 0.5, 1, torch.cuda.current_stream(), k_fallback=128)
    job.download(torch.cuda.current_stream())
    ref = job.fetch()
    cnt, _ = job.selection()
    np.testing.assert_array_equal(cnt, counts)
    job.free()
    srv = gdk.Server(ctx, pk, w.params, capacity=128, max_atoms=256, max_rotamers=48, free_sms=16)
    with pytest.raises(gdk.GeoDockError) as e:  # a restart listed twice
        bad = lists[:1].copy()
        bad[0, 1] = bad[0, 0]
        srv.submit(w.batch, [0], restarts=bad, n_restarts=counts[:1])
    assert e.value.status == gdk.GD_EINVAL
    q = srv.submit(w.batch, [0], restarts=lists[:1], n_restarts=counts[:1])
    seqs, got = {q: 0}, {q: srv.poll(q)}  # ligand 0 alone first
    for wave in (np.arange(1, 33), np.arange(33, L)):  # then the rest in two overlapping waves
        first = srv.submit(w.batch, wave, restarts=lists[wave], n_restarts=counts[wave])
        for k, i in enumerate(wave):
            seqs[first + k] = int(i)
    got.update({qq: srv.poll(qq) for qq in seqs if qq != q})
    with pytest.raises(gdk.GeoDockError) as e:  # SMs can only be reserved before the first launch
        ctx._check(gdk.load().gd_server_reserve_sms(srv.h, 8))
    assert e.value.status == gdk.GD_EBUSY
    print(srv.stats())
    srv.close()
    ao, ro = np.asarray(w.batch.atom_off), np.asarray(w.batch.rot_off)
    for qq, i in seqs.items():
        view = dict(best_score=ref["best_score"][i:i + 1], best_orient=ref["best_orient"][i:i + 1],
                    best_angle=ref["best_angle"][ro[i]:ro[i + 1]], best_xyz=ref["best_xyz"][ao[i]:ao[i + 1]],
                    evals=ref["evals"][i:i + 1], pair_tests=ref["pair_tests"][i:i + 1],
                    atom_moves=ref["atom_moves"][i:i + 1], reach_tests=ref["reach_tests"][i:i + 1],
                    best_rigid=ref["best_rigid"][i:i + 1])
        _same(got[qq], view, f"ligand {i} ({counts[i]} restarts)")
    pk.free()


def test_a_held_slot_times_out_and_the_context_stays_usable(ctx):
    w = synth.workload_stream(8, seed_offset=72)
    pk = ctx.load_pocket(w.pocket)
    srv = gdk.Server(ctx, pk, w.params, capacity=8, max_atoms=256, max_rotamers=48, idle_ms=50)
    srv.test_hold(2)  # ligand 2's slot is never released to its later work items
    first = srv.submit(w.batch)
    t0 = time.time()
    with pytest.raises(gdk.GeoDockError) as e:
        for q in range(first, first + 8):
            srv.poll(q)
    print(f"timed out after {time.time() - t0:.2f} s: {e.value}")
    assert e.value.status == gdk.GD_ETIMEOUT
    srv.close()
    out = ctx.dock_batch(pk, w.batch, w.params).fetch()  # the context still docks
    assert len(out["best_score"]) == 8 and np.all(out["best_score"] > 0)
    pk.free()
