"""Streaming screen: continuous batching of arriving ligands onto the resident pocket.

Ligands arrive over time (a Poisson process in the benchmark).  Whenever an in-flight
slot is free and the context's device-memory budget admits it, every ligand that has
arrived and is still waiting is packed into one batch (up to max_batch) and submitted on
its own CUDA stream: features -> proposer network -> restart selection with fallback ->
pruned search -> copy back.  Several batches are in flight at once, so packing and
copies of one overlap the kernels of others, and a ligand arriving while others run
waits only for the next free slot, not for a fixed batch to fill.  Completions are
polled without blocking; each ligand's latency is its completion time minus its
arrival time.  Every computation runs in libgeodock's kernels; this module schedules.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import geodock as gdk
from . import synth


@dataclass(eq=False)  # batches are compared by identity
class _Batch:
    ids: np.ndarray
    job: object
    X: object
    y: object
    stream: object
    submitted: float


@dataclass
class ScreenResult:
    best_score: np.ndarray
    best_orient: np.ndarray
    arrival: np.ndarray
    done: np.ndarray
    batches: int = 0
    budget_waits: int = 0
    batch_sizes: list = field(default_factory=list)
    restarts: np.ndarray = None

    @property
    def latency(self):
        return self.done - self.arrival

    def summary(self):
        lat = self.latency
        span = float(self.done.max() - self.arrival.min())
        return dict(ligands=int(len(lat)), ligands_per_s=len(lat) / span, p50_ms=1e3 * float(np.percentile(lat, 50)),
                    p99_ms=1e3 * float(np.percentile(lat, 99)), mean_batch=float(np.mean(self.batch_sizes)),
                    batches=self.batches, budget_waits=self.budget_waits,
                    restarts_per_ligand=float(np.mean(self.restarts)))


def slot_bytes(max_batch, n_orient):
    """Device bytes of one in-flight slot's proposer buffers: a BF16 feature row (48 x 2
    bytes) and an FP32 prediction per (ligand, restart) of a full batch."""
    return max_batch * n_orient * (48 * 2 + 4)


class Screen:
    """Continuous-batching screen of one pocket with a trained proposer (k restarts per
    ligand, k_fallback -- all when None -- where the proposer's top-k spread falls back).

    Memory: every in-flight slot owns its proposer buffers (features and predictions of a
    full batch, slot_bytes), allocated once here; the search's own memory comes from the
    context and counts against its budget, so a screen under a total budget B runs on a
    context created with B - max_inflight * slot_bytes (Screen.context_budget).
    Admission: a batch is admitted when a slot is free and gd_prepare_batch fits the
    context's budget; otherwise it waits for an in-flight batch to finish, and if nothing
    is in flight the batch size is halved.  Each completed batch lets the size grow back
    (doubling, up to max_batch)."""

    def __init__(self, ctx, pocket, params, net, k=16, margin=1e30, rule=1, max_batch=512, max_inflight=4,
                 k_fallback=None,
                 debug=False):
        import torch
        self.ctx, self.pk, self.params, self.net = ctx, pocket, params, net
        self.k, self.margin, self.rule, self.k_fallback = k, margin, rule, k_fallback
        self.max_batch, self.debug = max_batch, debug
        self.streams = [torch.cuda.Stream() for _ in range(max_inflight)]
        rows = max_batch * params.n_orient
        self.X = [torch.empty((rows, 48), dtype=torch.bfloat16, device="cuda") for _ in range(max_inflight)]
        self.y = [torch.empty(rows, device="cuda") for _ in range(max_inflight)]

    @staticmethod
    def context_budget(total_bytes, max_batch, n_orient, max_inflight=4):
        """Budget of the context of a screen that may hold total_bytes of device memory."""
        return total_bytes - max_inflight * slot_bytes(max_batch, n_orient)

    def _submit(self, batch, ids, slot):
        """Queue ligands ids of the library batch (packed straight from it, no sub-batch)."""
        import torch
        stream = self.streams[slot]
        job = self.ctx.prepare_batch(self.pk, batch, self.params, stream=stream, debug=self.debug, sel=ids)
        rows = len(ids) * self.params.n_orient
        with torch.cuda.stream(stream):
            X, y = self.X[slot][:rows], self.y[slot][:rows]
            job.features(x_bf16=X, stream=stream)
            self.net.predict(X, y)
            job.launch_proposed(y, self.k, self.margin, self.rule, stream, k_fallback=self.k_fallback)
            job.download(stream)
        return job, X, y

    def run(self, workload, arrival_times, clock=time.perf_counter, ligand_of=None):
        """Serve one request per arrival time: request i asks for ligand ligand_of[i] of
        `workload`'s library (default: ligand i) and becomes available arrival_times[i]
        seconds after the start.  Returns per-request results and timings."""
        N = len(arrival_times)
        ligand_of = np.arange(N) if ligand_of is None else np.asarray(ligand_of, np.int64)
        order = np.argsort(arrival_times, kind="stable")
        res = ScreenResult(best_score=np.zeros(N, np.uint32), best_orient=np.zeros(N, np.int32),
                           arrival=np.asarray(arrival_times, np.float64).copy(), done=np.zeros(N),
                           restarts=np.zeros(N, np.int32))
        pending, inflight = deque(), []
        free = list(range(len(self.streams)))
        cap = self.max_batch  # shrinks if a batch cannot fit the budget even alone
        nxt, finished = 0, 0
        t0 = clock()
        while finished < N:
            now = clock() - t0
            while nxt < N and arrival_times[order[nxt]] <= now:
                pending.append(order[nxt])
                nxt += 1
            progressed = False
            for b in list(inflight):
                out = b.job.fetch(blocking=False)
                if out is None:
                    continue
                t_done = clock() - t0
                cnt, _ = b.job.selection()
                res.best_score[b.ids] = out["best_score"]
                res.best_orient[b.ids] = out["best_orient"]
                res.restarts[b.ids] = cnt
                res.done[b.ids] = t_done
                b.job.free()
                free.append(self.streams.index(b.stream))
                inflight.remove(b)
                finished += len(b.ids)
                cap = min(self.max_batch, 2 * cap)  # memory came back: let the batch size recover
                progressed = True
            if pending and free:
                take = [pending.popleft() for _ in range(min(cap, len(pending)))]
                ids = np.array(take, np.int64)
                slot = free[-1]
                stream = self.streams[slot]
                try:
                    job, X, y = self._submit(workload.batch, ligand_of[ids], slot)
                except gdk.GeoDockError as e:
                    if e.status != gdk.GD_EBUDGET:
                        raise
                    pending.extendleft(reversed(take))
                    res.budget_waits += 1
                    if not inflight:  # nothing will free memory: admit a smaller batch
                        if len(take) == 1:
                            raise
                        cap = max(1, len(take) // 2)
                    time.sleep(1e-4)  # else wait for a batch to finish and return its memory
                    continue
                free.pop()
                inflight.append(_Batch(ids, job, X, y, stream, clock() - t0))
                res.batches += 1
                res.batch_sizes.append(len(ids))
                progressed = True
            if not progressed:
                wait = 2e-4
                if nxt < N and not inflight:
                    wait = max(0.0, min(wait, arrival_times[order[nxt]] - (clock() - t0)))
                time.sleep(wait)
        return res


def poisson_arrivals(n, rate, seed=0):
    """Arrival times (s) of n events of a Poisson process with `rate` per second."""
    rng = synth.SplitMix64(synth.ligand_seed(seed, 0))
    t, out = 0.0, np.empty(n)
    for i in range(n):
        t += -np.log(1.0 - rng.uniform()) / rate
        out[i] = t
    return out


class QueueScreen:
    """The learned screen on the device queue: arriving ligands are proposed in batches
    (features -> proposer network -> restarts by prediction, ties to the smaller id, the k best
    unless the spread pred(1st) - pred(k-th) exceeds the margin, then the k_fallback best:
    the selection rule of the batched learned path) on SMs the server leaves free, and each
    ligand then joins the running search launch with its restart list
    (gd_server_submit_restarts); results come back per ligand as they finish.  The server
    runs a wide tile (one block of 16 warps per SM, all of its registers), so the reserved
    SMs stay free for the proposer's kernels.  Up to max_inflight proposals run at once,
    each on its own stream with its own buffers; a proposal's restart lists are copied to
    pinned host memory and submitted once its event has completed, so the host loop never
    waits for the device.

    A proposal batch is padded to one of a few sizes (powers of two from 64 up to
    max_batch, the rows past the batch discarded), each prepared once per stream before the
    server starts (warm_library: a batch holding at least one ligand), so that the
    context's memory caches and torch's allocator serve every later batch without
    allocating: an allocation waits for the running search launch to end (it ends only
    after idle_ms without work), which put 0.2 s into a batch's latency."""

    def __init__(self, ctx, pocket, params, net, k=16, margin=1e30, k_fallback=128, max_batch=1024, free_sms=16,
                 tile=8, capacity=8192, max_rotamers=64, idle_ms=200, warm_library=None, max_inflight=3):
        import torch
        self.ctx, self.pk, self.params, self.net = ctx, pocket, params, net
        self.k, self.margin, self.kf = k, margin, min(k_fallback, params.n_orient)
        self.max_batch = max_batch
        self.srv = gdk.Server(ctx, pocket, params, capacity=capacity, max_atoms=256, max_rotamers=max_rotamers,
                              idle_ms=idle_ms, tile=tile, free_sms=free_sms)
        rows = max_batch * params.n_orient
        self.streams = [torch.cuda.Stream() for _ in range(max_inflight)]
        self.X = [torch.empty((rows, 48), dtype=torch.bfloat16, device="cuda") for _ in range(max_inflight)]
        self.y = [torch.empty(rows, device="cuda") for _ in range(max_inflight)]
        self.h_lists = [torch.empty((max_batch, self.kf), dtype=torch.int32, pin_memory=True)
                        for _ in range(max_inflight)]
        self.h_cnt = [torch.empty(max_batch, dtype=torch.int32, pin_memory=True) for _ in range(max_inflight)]
        self.sizes = sorted({min(max_batch, 1 << b) for b in range(6, 16) if (1 << (b - 1)) < max_batch})
        if warm_library is not None:
            for slot in range(max_inflight):
                for n in self.sizes:
                    job, ev = self._launch(warm_library, np.zeros(n, np.int64), slot)
                    ev.synchronize()
                    job.free()

    def _padded(self, n):
        return next(s for s in self.sizes if s >= n)

    def _launch(self, batch, ids, slot):
        """Queue the proposal of ligands ids on stream `slot`: (job, completion event)."""
        import torch
        O = self.params.n_orient
        n = len(ids)
        m = self._padded(n)  # padded with copies of the first ligand
        sel = np.concatenate([np.asarray(ids, np.int64), np.full(m - n, ids[0], np.int64)])
        st = self.streams[slot]
        job = self.ctx.prepare_batch(self.pk, batch, self.params, stream=st, sel=sel)
        with torch.cuda.stream(st):
            X, y = self.X[slot][:m * O], self.y[slot][:m * O]
            job.features(x_bf16=X, stream=st)
            self.net.predict(X, y)
            # larger prediction first, ties to the smaller restart (the device selection's order)
            val, idx = torch.sort(y.view(m, O), dim=1, descending=True, stable=True)
            fall = (val[:, 0] - val[:, self.k - 1]) > self.margin
            self.h_lists[slot][:m].copy_(idx[:, :self.kf].to(torch.int32), non_blocking=True)
            self.h_cnt[slot][:m].copy_(torch.where(fall, self.kf, self.k).to(torch.int32), non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        return job, ev

    def _lists(self, slot, n):
        return self.h_lists[slot][:n].numpy().astype(np.uint16), self.h_cnt[slot][:n].numpy().copy()

    def propose(self, batch, ids):
        """Restart lists [n, k_fallback] (uint16) and their lengths [n] for ligands ids
        (synchronously, on the first stream)."""
        n = len(ids)
        if n > self.max_batch:
            parts = [self.propose(batch, ids[i:i + self.max_batch]) for i in range(0, n, self.max_batch)]
            return np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts])
        job, ev = self._launch(batch, ids, 0)
        ev.synchronize()
        job.free()
        return self._lists(0, n)

    def run(self, workload, arrival_times, clock=time.perf_counter, ligand_of=None):
        """Serve one request per arrival time (as Screen.run)."""
        N = len(arrival_times)
        ligand_of = np.arange(N) if ligand_of is None else np.asarray(ligand_of, np.int64)
        order = np.argsort(arrival_times, kind="stable")
        res = ScreenResult(best_score=np.zeros(N, np.uint32), best_orient=np.zeros(N, np.int32),
                           arrival=np.asarray(arrival_times, np.float64).copy(), done=np.zeros(N),
                           restarts=np.zeros(N, np.int32))
        pending = deque()
        inflight = []  # (slot, requests, job, event), oldest first
        free = list(range(len(self.streams)))
        ready = deque()  # (requests, restart lists, counts) proposed but not yet submitted
        req_of = {}  # server sequence number -> request
        nxt = finished = 0
        t0 = clock()
        while finished < N:
            now = clock() - t0
            while nxt < N and arrival_times[order[nxt]] <= now:
                pending.append(order[nxt])
                nxt += 1
            progressed = False
            if pending and free:
                take = np.array([pending.popleft() for _ in range(min(self.max_batch, len(pending)))], np.int64)
                slot = free.pop()
                job, ev = self._launch(workload.batch, ligand_of[take], slot)
                inflight.append((slot, take, job, ev))
                res.batches += 1
                res.batch_sizes.append(len(take))
                progressed = True
            while inflight and inflight[0][3].query():  # proposals complete in stream order per slot
                slot, take, job, ev = inflight.pop(0)
                lists, cnt = self._lists(slot, len(take))
                job.free()
                free.append(slot)
                ready.append((take, lists, cnt))
                progressed = True
            while ready:
                take, lists, cnt = ready[0]
                try:
                    first = self.srv.submit(workload.batch, ligand_of[take], restarts=lists, n_restarts=cnt)
                except gdk.GeoDockError as e:  # no free slot: return finished results first
                    if e.status != gdk.GD_EBUSY:
                        raise
                    break
                ready.popleft()
                for j, r in enumerate(take.tolist()):
                    req_of[first + j] = r
                res.restarts[take] = cnt
                progressed = True
            got = self._collect(res, req_of, clock, t0)
            finished += got
            if not progressed and not got:
                wait = 5e-5
                if nxt < N and not req_of and not inflight:
                    wait = max(0.0, min(2e-4, arrival_times[order[nxt]] - (clock() - t0)))
                time.sleep(wait)
        return res

    def _collect(self, res, req_of, clock, t0):
        seqs, sc, ob = self.srv.collect(8192)
        if not len(seqs):
            return 0
        t = clock() - t0
        for q, a, b in zip(seqs.tolist(), sc.tolist(), ob.tolist()):
            r = req_of.pop(q)
            res.best_score[r], res.best_orient[r], res.done[r] = a, b, t
        return len(seqs)

    def close(self):
        self.srv.close()
