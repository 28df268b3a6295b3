"""The learned proposer on the GPU: features against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_1901_06229_b300 import geodock as gdk
from paper_1901_06229_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = gdk.Context(0)
    yield c
    c.close()


def gpu_features(ctx, w):
    import torch
    pk = ctx.load_pocket(w.pocket)
    job = ctx.prepare_batch(pk, w.batch, w.params)
    L, O = w.batch.n_ligands, w.params.n_orient
    xf = torch.zeros((L * O, 48), device="cuda")
    xb = torch.zeros((L * O, 48), dtype=torch.bfloat16, device="cuda")
    job.features(x_bf16=xb, x_f32=xf)
    torch.cuda.synchronize()
    job.free()
    pk.free()
    return xf.cpu().numpy(), xb.float().cpu().numpy()


def _slot_boundary_workload():
    """Ligands on both sides of the feature kernel's atom-slot variants (1, 2, 4 or 8 atoms
    per lane: at most 32, 64, 128 or 256 atoms), and the largest the generator builds."""
    ligs = []
    for i, n in enumerate((25, 32, 33, 64, 65, 128, 129, 250)):
        rng = synth.SplitMix64(synth.ligand_seed(synth.BASE_SEED + 77, i))
        ligs.append(synth.gen_ligand(rng, n, max(1, n // 6)))
    return synth.Workload("slot-boundaries", synth.pocket_64(), synth.pack(ligs), synth.SearchParams(2, 2, 2, 64))


@pytest.mark.parametrize("which", ["batched", "single", "large", "slot_boundaries"])
def test_features_match_oracle(ctx, which):
    w = {"batched": lambda: synth.workload_batched(12), "single": synth.workload_single,
         "large": lambda: synth.workload_large(2), "slot_boundaries": _slot_boundary_workload}[which]()
    xf, xb = gpu_features(ctx, w)
    O = w.params.n_orient
    rng = np.random.default_rng(3)
    compared = {"samples": 0, "skipped": 0}
    for i in range(w.batch.n_ligands):
        lig = w.batch.ligand(i)
        for o in sorted(set(rng.integers(0, O, size=6).tolist()) | {0, O - 1}):
            ref = oracle.features(lig.xyz, len(lig.rot_bond), o, w.params, w.pocket)
            g = xf[i * O + o]
            q, qr = g[:4].astype(np.float64), ref["feat"][:4]
            if abs(qr[0]) < 1e-6:  # q and -q are the same rotation
                q = q if np.dot(q, qr) >= 0 else -q
            np.testing.assert_allclose(q, qr, atol=2e-6)
            np.testing.assert_allclose(g[4:7], ref["feat"][4:7], rtol=2e-6, atol=1e-7)
            if ref["hist_edge"] > 1e-5:
                np.testing.assert_allclose(g[7:23], ref["feat"][7:23], atol=1e-7)
            if ref["fps_gap"] > 1e-5:
                ok = ~ref["sample_fragile"]
                np.testing.assert_array_equal(g[23:][ok], ref["feat"][23:][ok].astype(np.float32))
                compared["samples"] += int(ok.sum())
            else:
                compared["skipped"] += 1
    print(compared)
    assert compared["samples"] > 100
    # the BF16 copy is the FP32 features rounded to nearest
    np.testing.assert_array_equal(xb, _bf16(xf))


def _bf16(x):
    import torch
    return torch.tensor(x).to(torch.bfloat16).float().numpy()


def _topk_host(pred, k):
    """Top-k restarts per row, ties to the smaller restart id."""
    L, O = pred.shape
    out = []
    for i in range(L):
        order = np.lexsort((np.arange(O), -pred[i].astype(np.float64)))
        out.append(order[:k])
    return np.array(out)


def test_bounded_fallback_searches_the_best_predicted_restarts(ctx):
    """gd_job_launch_proposed_fb: ligands whose top-k spread exceeds the margin search
    their k_fallback best-predicted restarts (ties to the smaller id), the others their k
    best; each best pose is the best over exactly those restarts."""
    import torch
    w = synth.workload_batched(32)
    L, O, k, kf = w.batch.n_ligands, w.params.n_orient, 16, 64
    pk = ctx.load_pocket(w.pocket)
    job = ctx.prepare_batch(pk, w.batch, w.params, debug=True)
    job.launch()
    job.download()
    ex = job.fetch()
    pred = np.random.default_rng(7).normal(size=(L, O)).astype(np.float32)
    pred[:, 3] = pred[:, 200] = 9.0  # a planted tie: restart 3 ranks before 200
    top_k = _topk_host(pred, k)
    spread = pred[np.arange(L), top_k[:, 0]] - pred[np.arange(L), top_k[:, -1]]
    margin = float(np.median(spread))  # about half of the ligands fall back
    job.launch_proposed(torch.tensor(pred.ravel()).cuda(), k, margin, rule=1, k_fallback=kf)
    job.download()
    pr = job.fetch()
    cnt, _ = job.selection()
    fb = spread > margin
    assert 0 < fb.sum() < L
    np.testing.assert_array_equal(cnt, np.where(fb, kf, k))
    top_f = _topk_host(pred, kf)
    R = np.diff(w.batch.rot_off)
    for i in range(L):
        chosen = top_f[i] if fb[i] else top_k[i]
        sc = ex["orient_score"][i, chosen].astype(np.int64)
        assert pr["best_score"][i] == sc.max()
        assert pr["best_orient"][i] == chosen[sc == sc.max()].min()
        np.testing.assert_array_equal(pr["orient_score"][i, chosen], ex["orient_score"][i, chosen])
        assert pr["evals"][i] == len(chosen) * R[i] * w.params.n_angles
    with pytest.raises(gdk.GeoDockError, match="k_fallback"):
        job.launch_proposed(torch.tensor(pred.ravel()).cuda(), k, margin, rule=1, k_fallback=k - 1)
    job.free()
    pk.free()


def test_subset_search_is_the_best_of_the_chosen_restarts(ctx):
    import torch
    w = synth.workload_batched(24)
    L, O, k = w.batch.n_ligands, w.params.n_orient, 16
    pk = ctx.load_pocket(w.pocket)
    job = ctx.prepare_batch(pk, w.batch, w.params, debug=True)
    job.launch()
    job.download()
    ex = job.fetch()
    pred = np.random.default_rng(2).normal(size=(L, O)).astype(np.float32)
    pred[:, 5] = pred[:, 9] = 10.0  # a planted tie: restart 5 ranks before 9
    job.launch_proposed(torch.tensor(pred.ravel()).cuda(), k, 1e30, rule=1)
    job.download()
    pr = job.fetch()
    cnt, spread = job.selection()
    assert np.all(cnt == k)
    top = _topk_host(pred, k)
    R = np.diff(w.batch.rot_off)
    for i in range(L):
        sc = ex["orient_score"][i, top[i]].astype(np.int64)
        best = sc.max()
        assert pr["best_score"][i] == best
        assert pr["best_orient"][i] == top[i][sc == best].min()
        np.testing.assert_array_equal(pr["orient_score"][i, top[i]], ex["orient_score"][i, top[i]])
        assert pr["evals"][i] == k * R[i] * w.params.n_angles
        np.testing.assert_allclose(spread[i], np.sort(pred[i])[::-1][0] - np.sort(pred[i])[::-1][k - 1], rtol=1e-6)
    # rule 0 with an infinite margin: every ligand falls back to the full search
    job.launch_proposed(torch.tensor(pred.ravel()).cuda(), k, 1e30, rule=0)
    job.download()
    full = job.fetch()
    assert np.all(job.selection()[0] == O)
    for key in ("best_score", "best_orient", "best_angle", "best_xyz", "evals"):
        np.testing.assert_array_equal(full[key], ex[key], err_msg=key)
    job.free()
    pk.free()
