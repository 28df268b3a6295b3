"""Learned orientation proposer: data, training and evaluation driven through the C ABI.

The network (include/geodock_mlp.h) predicts each restart's final score
S_final / (255 n) from 48 features; at inference only the top-k restarts of every ligand
get the full fragment search, unless the spread of its top-k predictions is below a
margin, in which case every restart is searched.  Every computation -- features,
exhaustive search for the targets, forward / backward / Adam, selection, pruned search --
runs in libgeodock's kernels; this module sequences the calls.
"""
from __future__ import annotations

import time

import numpy as np

from . import geodock as gdk
from . import mlp as _mlp


def dataset(ctx, pk, w, stream=None):
    """Features (BF16 [L*O, 48]) and targets S_final / (255 n) (FP32 [L*O]) on the GPU."""
    import torch
    L, O = w.batch.n_ligands, w.params.n_orient
    job = ctx.prepare_batch(pk, w.batch, w.params, stream=stream, debug=True)
    X = torch.empty((L * O, 48), dtype=torch.bfloat16, device="cuda")
    job.features(x_bf16=X, stream=stream)
    job.launch(stream)
    job.download(stream)
    out = job.fetch()
    job.free()
    n = np.diff(w.batch.atom_off).astype(np.float32)
    t = (out["orient_score"].astype(np.float32) / (255.0 * n[:, None])).reshape(-1)
    return X, torch.tensor(t, device="cuda"), out


def standardise(t):
    """Targets as (t - mean) / std (the ranking, all the selection uses, is unchanged)."""
    mu, sd = float(t.mean()), float(t.std())
    return (t - mu) / max(sd, 1e-12), mu, sd


def train(net, X, t, epochs=12, batch=4096, lr=2e-3, seed=0, lr_decay=0.85):
    """Adam over shuffled minibatches; returns the mean loss of every epoch."""
    import torch
    N = X.shape[0] // batch * batch
    loss = torch.zeros(1, device="cuda")
    hist = []
    g = torch.Generator().manual_seed(seed)
    for ep in range(epochs):
        perm = torch.randperm(X.shape[0], generator=g)[:N].to(torch.int32).cuda()
        acc = torch.zeros(1, device="cuda")
        for b in range(N // batch):
            net.train_step(X, t, lr, loss=loss, idx=perm[b * batch:(b + 1) * batch], B=batch)
            acc += loss
        hist.append(acc.item() / (N // batch))
        lr *= lr_decay
    return hist


def predict(ctx, net, pk, w, stream=None):
    """(prepared job, predictions [L*O] on the GPU)."""
    import torch
    L, O = w.batch.n_ligands, w.params.n_orient
    job = ctx.prepare_batch(pk, w.batch, w.params, stream=stream)
    X = torch.empty((L * O, 48), dtype=torch.bfloat16, device="cuda")
    job.features(x_bf16=X, stream=stream)
    y = torch.empty(L * O, device="cuda")
    net.predict(X, y)
    return job, y


def evaluate(ctx, net, pk, w, k=16, margin=1e30, rule=1, exhaustive=None, k_fallback=None):
    """Recall / regret of the pruned search against the exhaustive one on workload w
    (ligands that fall back search their k_fallback best restarts, all when None)."""
    job, y = predict(ctx, net, pk, w)
    job.launch_proposed(y, k, margin, rule, k_fallback=k_fallback)
    job.download()
    pruned = job.fetch()
    cnt, spread = job.selection()
    if exhaustive is None:
        job.launch()
        job.download()
        exhaustive = job.fetch()
    job.free()
    be, bp = exhaustive["best_score"].astype(np.int64), pruned["best_score"].astype(np.int64)
    recall = float(np.mean(bp == be))
    regret = float(np.mean((be - bp) / np.maximum(be, 1)))
    return dict(recall=recall, regret=regret, fallback=float(np.mean(cnt > k)), restarts=float(cnt.mean()),
                pruned=pruned, exhaustive=exhaustive, spread=spread)


def tune_margin(ctx, net, pk, w, k=16, target=0.99, rule=1, margins=None, k_fallback=None):
    """The margin that reaches `target` best-pose recall on workload w with the fewest
    fallbacks: for rule 1 (fall back above the margin) the largest such margin, scanned
    downwards; for rule 0 the smallest, scanned upwards."""
    if margins is None:
        grid = list(np.geomspace(1e-3, 10.0, 41))
        margins = grid[::-1] if rule == 1 else [-1e30] + grid
    ex, r = None, None
    for m in margins:
        r = evaluate(ctx, net, pk, w, k, m, rule, exhaustive=ex, k_fallback=k_fallback)
        ex = r["exhaustive"]
        if r["recall"] >= target:
            return float(m), r
    return float(margins[-1]), r


def fit(ctx, pk, n_train=12000, n_val=4000, k=16, target=0.99, seed=1, k_fallback=None):
    """Train on streaming-screen ligands and tune the fallback margin for `target` recall
    on a held-out split.  Returns (network, margin, training info)."""
    import torch
    from . import synth
    wt = synth.workload_stream(n_train, seed_offset=50)
    wv = synth.workload_stream(n_val, seed_offset=51)
    X, t, _ = dataset(ctx, pk, wt)
    ts, mu, sd = standardise(t)
    net = _mlp.MLP(torch.cuda.current_device(), seed=seed, max_batch=4096)
    t0 = time.perf_counter()
    hist = train(net, X, ts)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    margin, r = tune_margin(ctx, net, pk, wv, k=k, target=target, rule=1, k_fallback=k_fallback)
    del X, t, ts
    return net, margin, dict(rows=n_train * wt.params.n_orient, epochs=len(hist), seconds=secs,
                             final_loss=hist[-1], val_recall=r["recall"], val_fallback=r["fallback"])
