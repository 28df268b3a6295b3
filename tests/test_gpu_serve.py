"""Streaming screen: continuous batching gives every ligand the result it gets alone,
and admission by device-memory budget delays work without changing results."""
import numpy as np
import pytest

from paper_1901_06229_b300 import geodock as gdk
from paper_1901_06229_b300 import mlp, serve, synth

pytestmark = pytest.mark.gpu


def _alone(ctx, pk, w, net, i, k, margin, k_fallback=None):
    import torch
    b = w.batch.subset([i])
    job = ctx.prepare_batch(pk, b, w.params)
    X = torch.empty((w.params.n_orient, 48), dtype=torch.bfloat16, device="cuda")
    y = torch.empty(w.params.n_orient, device="cuda")
    job.features(x_bf16=X)
    net.predict(X, y)
    job.launch_proposed(y, k, margin, 1, k_fallback=k_fallback)
    job.download()
    out = job.fetch()
    job.free()
    return int(out["best_score"][0]), int(out["best_orient"][0])


def _median_spread(ctx, pk, w, net, k):
    import torch
    job = ctx.prepare_batch(pk, w.batch, w.params)
    L, O = w.batch.n_ligands, w.params.n_orient
    X = torch.empty((L * O, 48), dtype=torch.bfloat16, device="cuda")
    y = torch.empty(L * O, device="cuda")
    job.features(x_bf16=X)
    net.predict(X, y)
    job.launch_proposed(y, k, 1e30, 1)
    _, spread = job.selection()
    job.free()
    return float(np.median(spread))


@pytest.fixture(scope="module")
def setup():
    import torch
    ctx = gdk.Context(0)
    w = synth.workload_stream(400, seed_offset=77)
    pk = ctx.load_pocket(w.pocket)
    net = mlp.MLP(0, seed=5, max_batch=1024)  # untrained: consistency does not need a good model
    margin = _median_spread(ctx, pk, w, net, 16)  # about half of the ligands fall back
    yield ctx, pk, w, net, margin
    net.close()
    pk.free()
    ctx.close()


def test_results_are_the_same_alone_and_in_the_mix(setup):
    ctx, pk, w, net, margin = setup
    arr = serve.poisson_arrivals(w.batch.n_ligands, 20000.0, seed=3)
    scr = serve.Screen(ctx, pk, w.params, net, k=16, margin=margin, max_batch=64, max_inflight=3)
    res = scr.run(w, arr)
    s = res.summary()
    print(s)
    assert res.batches > 3 and max(res.batch_sizes) > 1
    assert 0 < np.mean(res.restarts == 256) < 1  # both pruned and fallback ligands
    assert np.all(res.latency > 0)
    for i in np.random.default_rng(0).choice(w.batch.n_ligands, 40, replace=False):
        assert _alone(ctx, pk, w, net, int(i), 16, margin) == (int(res.best_score[i]), int(res.best_orient[i]))


def test_bounded_fallback_in_the_mix(setup):
    """The screen with a bounded fallback (ligands that fall back search their 64
    best-predicted restarts) gives every ligand the result it gets alone."""
    ctx, pk, w, net, margin = setup
    arr = serve.poisson_arrivals(w.batch.n_ligands, 20000.0, seed=4)
    scr = serve.Screen(ctx, pk, w.params, net, k=16, margin=margin, max_batch=64, max_inflight=3, k_fallback=64)
    res = scr.run(w, arr)
    assert set(np.unique(res.restarts)) == {16, 64}  # both pruned and fallback ligands
    for i in np.random.default_rng(1).choice(w.batch.n_ligands, 40, replace=False):
        got = (int(res.best_score[i]), int(res.best_orient[i]))
        assert _alone(ctx, pk, w, net, int(i), 16, margin, k_fallback=64) == got


def test_requests_cycling_over_the_library(setup):
    """Requests that name library ligands (each ligand asked for twice, the second time
    while other batches run) get the same result as the ligand's first request."""
    ctx, pk, w, net, margin = setup
    n = w.batch.n_ligands
    lig = np.concatenate([np.arange(n), np.random.default_rng(5).permutation(n)])
    arr = serve.poisson_arrivals(2 * n, 40000.0, seed=6)
    res = serve.Screen(ctx, pk, w.params, net, k=16, margin=margin, max_batch=64, max_inflight=3).run(
        w, arr, ligand_of=lig)
    first = np.full(n, -1)
    for r in range(2 * n):
        if first[lig[r]] < 0:
            first[lig[r]] = r
        else:
            q = first[lig[r]]
            assert (res.best_score[r], res.best_orient[r]) == (res.best_score[q], res.best_orient[q])
    assert res.batches > 3


def test_memory_budget_admission(setup):
    ctx0, pk0, w, net, margin = setup
    arr = np.zeros(w.batch.n_ligands)  # everything arrives at once
    free_run = serve.Screen(ctx0, pk0, w.params, net, k=16, margin=margin, max_batch=100, max_inflight=4).run(w, arr)
    # a budget that holds the pocket and about one batch: the others wait for memory
    tight = gdk.Context(0, mem_budget_bytes=3 << 20)
    pk = tight.load_pocket(w.pocket)
    res = serve.Screen(tight, pk, w.params, net, k=16, margin=margin, max_batch=100, max_inflight=4).run(w, arr)
    print(res.summary())
    assert res.budget_waits > 0
    np.testing.assert_array_equal(res.best_score, free_run.best_score)
    np.testing.assert_array_equal(res.best_orient, free_run.best_orient)
    pk.free()
    tight.close()


def test_selected_ligands_pack_like_a_sub_batch(setup):
    """gd_prepare_batch_sel packs ligands straight from the library: the same results as
    a sub-batch of those ligands (out of order and repeated indices included)."""
    ctx, pk, w, _, _ = setup
    rng = np.random.default_rng(11)
    ids = rng.choice(w.batch.n_ligands, 37, replace=False)
    ids = np.concatenate([ids, ids[:3]])  # a ligand may be listed twice
    outs = []
    for kw in (dict(batch=w.batch.subset(ids)), dict(batch=w.batch, sel=ids)):
        job = ctx.prepare_batch(pk, kw["batch"], w.params, sel=kw.get("sel"))
        job.launch()
        job.download()
        outs.append(job.fetch())
        job.free()
    for key in ("best_score", "best_orient", "best_angle", "best_xyz", "evals", "pair_tests", "atom_moves"):
        np.testing.assert_array_equal(outs[0][key], outs[1][key], err_msg=key)
    for bad in ([w.batch.n_ligands], [-1]):
        with pytest.raises(gdk.GeoDockError, match="outside"):
            ctx.prepare_batch(pk, w.batch, w.params, sel=np.array(bad))
    empty = ctx.prepare_batch(pk, w.batch, w.params, sel=np.zeros(0, np.int64))
    assert empty.L == 0
    empty.free()


def test_concurrent_jobs_on_one_context(setup):
    """Host threads docking on one context at once (ctypes releases the GIL): packing on
    the shared host pool, cached memory and per-job graphs give every job the result it
    gets alone."""
    import threading
    import torch
    ctx, pk, w, _, _ = setup
    parts = [np.arange(i, w.batch.n_ligands, 4) for i in range(4)]
    alone = []
    for ids in parts:
        job = ctx.prepare_batch(pk, w.batch, w.params, sel=ids)
        job.launch()
        job.download()
        alone.append(job.fetch())
        job.free()
    got, errors = [None] * 4, []

    def worker(t):
        try:
            s = torch.cuda.Stream()
            for _ in range(3):  # prepare, launch, relaunch (graph), fetch
                job = ctx.prepare_batch(pk, w.batch, w.params, sel=parts[t], stream=s)
                job.launch(s)
                job.launch(s)
                job.download(s)
                got[t] = job.fetch()
                job.free()
        except Exception as e:  # reported below
            errors.append(repr(e))

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors
    for t in range(4):
        for key in ("best_score", "best_orient", "best_angle", "best_xyz"):
            np.testing.assert_array_equal(got[t][key], alone[t][key], err_msg=f"{key} of part {t}")


def test_device_queue_screen_searches_the_proposed_restarts(setup):
    """The learned screen on the device queue (QueueScreen: proposer on SMs the server
    leaves free, each ligand joining the running launch with its restart list): every
    result is the maximum over exactly the restarts its proposal chose (ties to the
    smaller restart), against the exhaustive per-restart scores, with the fallback rule
    giving k or k_fallback restarts."""
    ctx, pk, w, net, margin = setup
    L = 160
    sub = synth.Workload("sub", w.pocket, w.batch.subset(np.arange(L)), w.params)
    full = ctx.dock_batch(pk, sub.batch, sub.params, debug=True)
    scores = full.fetch()["orient_score"].reshape(L, -1).astype(np.int64)
    full.free()
    scr = serve.QueueScreen(ctx, pk, w.params, net, k=16, margin=margin, k_fallback=128, max_batch=48,
                            free_sms=16, max_rotamers=int(np.diff(w.batch.rot_off).max()))
    arr = serve.poisson_arrivals(L, 20000.0, seed=4)
    res = scr.run(sub, arr)
    print(res.summary(), scr.srv.stats())
    lists, cnt = scr.propose(sub.batch, np.arange(L))
    scr.close()
    np.testing.assert_array_equal(res.restarts, cnt)
    assert set(np.unique(cnt)) <= {16, 128} and 0 < np.mean(cnt == 128) < 1
    for i in range(L):
        chosen = lists[i, :cnt[i]].astype(np.int64)
        s = scores[i, chosen]
        best = s.max()
        assert res.best_score[i] == best, i
        assert res.best_orient[i] == chosen[s == best].min(), i
