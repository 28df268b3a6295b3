"""Benchmark of the GeoDock pose search on B300: ligands/s and pose-evals/s.

A step is one pass of the whole hot path over one batch: every ligand of the batched
workload (4,096 ligands of 20-80 atoms, 2-12 rotamers; 64^3 pocket at 0.375 A;
256 Euler restarts x 64 angles) placed, swept and reduced to its best pose by one
graph replay: a small pose-setup kernel (restart rotations, centred ligands) and the
persistent fused search kernel.

  value : ligands/s with the packed batch resident in HBM (gd_job_launch replays the
          search; the L2 is flushed between steps, outside the timed events)
  e2e   : the same metric through gd_dock_batch + gd_fetch_results with host buffers:
          validation/packing, the host->device copy, the search and the copy of the
          results back are all inside the timed region (at least 20 batches, two in
          flight)
  roofline : the bound the search kernel meets, instruction issue: warp instructions
             of one launch (ncu count, keyed by a hash of the kernel sources) over the
             launch's CUDA-event time, against 148 SMs x 4 schedulers x the maximum clock.
             Beside it, ``work_rate_vs_fp32_peak``: the method's own work, counted by the
             oracle over the whole workload (per candidate 16 FP32 operations and one grid
             byte load per fragment atom, 7 operations per pair test with the candidate
             stopping at its first bump, 32-pair tiles), per second over the FP32 pipe's
             peak -- above 1, because the exact reach filter proves most of those pair
             tests unnecessary; and ``executed``, the FP32 operations the kernel performs.
  large / learned24 : the same measurement on the large-ligand workload, and the learned
             proposer (trained on the GPU on 1M plain-method tuples, then learned-pruned
             vs plain search on 16,384 held-out ligands with best-pose recall), run after
             the headline measurement at N = 1
  cpu_baseline : the FP64 oracle on the host cores, on a bounded sample

--impl reference times the oracle itself (the paper has no code to run) on the same
workload and metric.  With torchrun (N > 1) every rank docks its own 4,096 ligands
(weak scaling, no collective on the data path; one scalar all-reduce for timing).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1901_06229_b300 import synth  # noqa: E402

METRIC = "ligands/s (pose search, 1 B300)"
# learned path: a ligand whose top-16 predictions are spread out searches its 128
# best-predicted restarts (the fewest that still reach 99 % best-pose recall on held-out
# streaming ligands; 32 or 64 cannot)
K_FALLBACK = 128
# Best-pose recall the learned path must keep, and the recall its fallback margin is
# tuned for on the 4,000-ligand validation split: the two splits' recalls differ by
# sampling alone with a spread of about 0.18 % (binomial, 4,000 and 16,384 ligands at
# 99 %), so tuning 0.3 % above the target keeps the held-out recall above it.
RECALL_TARGET = 0.99
VAL_RECALL_TARGET = 0.993
# the serving sub-record of the default line: runs x seconds of Poisson arrivals at --rate
SERVE_SUB_REPEATS = 3
SERVE_SUB_SECONDS = 2.0
# SMs the learned device-queue screen leaves to its proposer's kernels: beside a busy
# search launch on the rest, a small proposal took 33 ms with 40 left free and 0.9 ms
# with 120, and at 100k ligands/s the pruned search needs a small part of the GPU
SERVE_LEARNED_FREE_SMS = 100
# FP32 operations the kernel executes (the "executed" roofline figure)
EXEC_OPS_PER_PAIR = 3        # 2 FFMA (|x_a - x_b|^2 + (cos-1) P + sin Q) + FMNMX
EXEC_OPS_PER_ATOM_MOVE = 6   # turn about the bond axis (6 FFMA; coordinates are grid units)
FP32_LANES_PER_SM = 128
LOADS_PER_SM_CLK = 32        # one 32-lane shared/L1 load instruction per clock per SM
# algorithmic work of each benchmark workload, counted by the oracle (oracle/algorithmic_work.py)
ALGORITHMIC_WORK = os.path.join(ROOT, "oracle", "algorithmic_work.json")

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one search-kernel launch,
# from one ncu capture of the full-size workload, keyed by a hash of the kernel sources
# and by (workload, tile): reported only while the kernel is the one that was measured.
SEARCH_KERNEL_SOURCES = ("paper_1901_06229_b300/csrc/gd_search.cu", "paper_1901_06229_b300/csrc/gd_internal.h")
MEASURED_TRAFFIC = {
    "d330ce6744aaba88": {("batched-4096lig-64grid", 14): 4557056 + 1178368,
                         ("batched-4096lig-64grid", 15): 4860160 + 1211904,
                         ("large-512lig-128grid", 16): 2730240 + 9728,
                         ("large-512lig-128grid", 18): 3069696 + 9216},
    "0dd17a1cd3e68422": {("batched-4096lig-64grid", 14): 4561408 + 1121024,
                         ("batched-4096lig-64grid", 15): 4743424 + 1152512,
                         ("large-512lig-128grid", 16): 2742528 + 8960,
                         ("large-512lig-128grid", 18): 3049216 + 12800},
    "250345eb4db4aed3": {("batched-4096lig-64grid", 14): 4553472 + 1180160,
                         ("batched-4096lig-64grid", 15): 4556544 + 1187072,
                         ("large-512lig-128grid", 16): 2849536 + 9728,
                         ("large-512lig-128grid", 18): 3107840 + 10240},
    "e95d5b061be765f4": {("batched-4096lig-64grid", 14): 4684032 + 1184256,
                         ("batched-4096lig-64grid", 15): 4559104 + 1190912,
                         ("large-512lig-128grid", 16): 3100672 + 11520,
                         ("large-512lig-128grid", 18): 2902528 + 10496},
    "6f657c070d65f73e": {("batched-4096lig-64grid", 14): 4555520 + 1185024,
                         ("batched-4096lig-64grid", 15): 4555264 + 1213184,
                         ("large-512lig-128grid", 16): 3054080 + 9728,
                         ("large-512lig-128grid", 18): 2749440 + 9728},
    "c9a7dbf8340ec2f4": {("batched-4096lig-64grid", 14): 4557056 + 1204736,
                         ("batched-4096lig-64grid", 15): 4556032 + 1150464,
                         ("large-512lig-128grid", 16): 3102208 + 9216,
                         ("large-512lig-128grid", 18): 3362560 + 8960},
    "8849191a14128210": {("batched-4096lig-64grid", 14): 4568832 + 1177856,
                         ("batched-4096lig-64grid", 15): 4556544 + 1146880,
                         ("large-512lig-128grid", 16): 2858752 + 9216,
                         ("large-512lig-128grid", 18): 2807040 + 11264},
    "ad511480c64b7604": {("batched-4096lig-64grid", 14): 4564992 + 1341440,
                         ("batched-4096lig-64grid", 15): 4736256 + 1323008,
                         ("large-512lig-128grid", 9): 3233280 + 5632},
    "089efa26c3e7fd61": {("batched-4096lig-64grid", 14): 4551680 + 1316352,
                         ("batched-4096lig-64grid", 15): 4552960 + 1300992,
                         ("large-512lig-128grid", 9): 3128832 + 5120},
}


# Warp instructions (smsp__inst_executed.sum) of one search-kernel launch, from one ncu
# capture of the full-size workload (one pass), keyed like MEASURED_TRAFFIC: the kernel
# is issue-bound, so its instruction issue rate against the schedulers' peak (4 per SM
# per clock) is the roofline that binds it.
MEASURED_INSTRUCTIONS = {
    "d330ce6744aaba88": {("batched-4096lig-64grid", 14): 8462969358,
                         ("batched-4096lig-64grid", 15): 8463073248,
                         ("large-512lig-128grid", 16): 15525958491,
                         ("large-512lig-128grid", 18): 15526017451},
    "0dd17a1cd3e68422": {("batched-4096lig-64grid", 14): 8462969337,
                         ("batched-4096lig-64grid", 15): 8463073215,
                         ("large-512lig-128grid", 16): 15525958569,
                         ("large-512lig-128grid", 18): 15526017496},
    "250345eb4db4aed3": {("batched-4096lig-64grid", 14): 8462969343,
                         ("batched-4096lig-64grid", 15): 8463073238,
                         ("large-512lig-128grid", 16): 15525958491,
                         ("large-512lig-128grid", 18): 15526017496},
    "e95d5b061be765f4": {("batched-4096lig-64grid", 14): 8462969330,
                         ("batched-4096lig-64grid", 15): 8463073267,
                         ("large-512lig-128grid", 16): 15525958491,
                         ("large-512lig-128grid", 18): 15526017451},
    "6f657c070d65f73e": {("batched-4096lig-64grid", 14): 8462969359,
                         ("batched-4096lig-64grid", 15): 8463073244,
                         ("large-512lig-128grid", 16): 15525958491,
                         ("large-512lig-128grid", 18): 15526017496},
    "c9a7dbf8340ec2f4": {("batched-4096lig-64grid", 14): 8469406704,
                         ("batched-4096lig-64grid", 15): 8469510617,
                         ("large-512lig-128grid", 16): 15486849117,
                         ("large-512lig-128grid", 18): 15486908155},
    "8849191a14128210": {("batched-4096lig-64grid", 14): 8469406720,
                         ("batched-4096lig-64grid", 15): 8469510627,
                         ("large-512lig-128grid", 16): 15486849117,
                         ("large-512lig-128grid", 18): 15486908104},
    "ad511480c64b7604": {("batched-4096lig-64grid", 14): 8448360711,
                         ("batched-4096lig-64grid", 15): 8448465499,
                         ("large-512lig-128grid", 9): 14709211994},
    "089efa26c3e7fd61": {("batched-4096lig-64grid", 14): 8448360733,
                         ("batched-4096lig-64grid", 15): 8448465523,
                         ("large-512lig-128grid", 9): 14709211960},
}
ISSUE_PER_SM_CLK = 4


# DRAM bytes of one proposer-network forward (mlp_infer_kernel, 4,194,304 rows), keyed by
# a hash of its source like MEASURED_TRAFFIC.
MLP_KERNEL_SOURCES = ("paper_1901_06229_b300/csrc/gd_mlp.cu",)
MEASURED_MLP_TRAFFIC = {
    "7c1706b4e4b0e212": {4194304: 402895104 + 15636992},
    "80d6c3c81be0ce7b": {4194304: 402857216 + 15846144},
    "5869ebdabcb3ead0": {4194304: 402904064 + 15991808},
    "0b6551ae97cb3c63": {4194304: 402875904 + 16060928},
}


def pipe_peaks(pipes: dict, achieved, loads, peak_tops: float, peak_loads: float) -> dict:
    """The pipes' peaks as measured by gd_measure_peaks beside the nominal ones the
    roofline divides by (lane FFMAs and lane shared-memory byte loads per second)."""
    f, l = pipes["ffma_per_s"] / 1e12, pipes["lds_u8_per_s"] / 1e12
    return {"ffma_T_per_s": f, "lds_u8_T_per_s": l, "ffma_of_nominal": f / peak_tops, "lds_u8_of_nominal": l / peak_loads,
            "frac_fp32": achieved / f if achieved is not None else None,
            "frac_loads": loads / l if loads is not None else None,
            "how": "gd_measure_peaks: every SM full, best of 3 launches, run after the timed region"}


def search_kernel_hash(sources=SEARCH_KERNEL_SOURCES) -> str:
    """Hash of a kernel's sources without // comments and blank lines (an edit of the
    documentation does not detach the measurements)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in sources:
        with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
            for line in fh:
                code = re.sub(r"//.*", "", line).rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def algorithmic_work(name, evals, moves):
    """The oracle's work totals of workload ``name`` (plain data), if they describe the
    launch that ran (same candidate and fragment-atom counts), else None."""
    try:
        with open(ALGORITHMIC_WORK) as f:
            t = json.load(f).get(name)
    except OSError:
        return None
    if not t or t["candidates"] != int(evals) or t["frag_atom_moves"] != int(moves):
        return None
    return t


def workload_for(name, rank, ligands=None):
    if name == "batched":
        n = ligands or 4096
        return synth.workload_batched(n, start=n * rank)
    if name == "large":
        n = ligands or 512
        return synth.workload_large(n, start=n * rank)
    if name == "single":
        return synth.workload_single()
    raise SystemExit(f"unknown workload {name}")


def workload_config(w, flush):
    p = w.params
    b = w.batch
    n = np.diff(b.atom_off)
    return {"workload": w.name, "ligands": int(b.n_ligands), "atoms": [int(n.min()), int(n.max())],
            "rotamers": int(len(b.rot_bond)), "grid": list(w.pocket.grid.shape[::-1]),
            "spacing": w.pocket.spacing, "orientations": p.n_orient, "euler": [p.n_alpha, p.n_beta, p.n_gamma],
            "angles": p.n_angles, "repetitions": p.repetitions, "bump_dist": p.bump_dist,
            "l2": flush}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = [r.split(",") for r in (self.out or "").strip().splitlines() if r.count(",") >= 7]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in rows if r[0].strip().replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if "Active" in r[4 + k] and "Not" not in r[4 + k]})
        busy = [s for s in sm if s > 0.5 * max(sm)] if sm else []
        return {"sm_mhz": float(np.median(busy or sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(rows), "reasons": reasons}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def cpu_baseline(w, seconds=12.0, single_seconds=4.0):
    """Oracle throughput on the host cores over a bounded sample of the workload: one
    std::thread per core over ligands, and single-threaded on the first ligands."""
    import oracle
    cores = os.cpu_count() or 1
    done, t0, i = 0, time.perf_counter(), 0
    while time.perf_counter() - t0 < seconds and i < w.batch.n_ligands:
        idx = list(range(i, min(i + cores, w.batch.n_ligands)))
        oracle.dock_batch(w.batch.subset(idx), w.pocket, w.params, n_threads=cores)
        done += len(idx)
        i += len(idx)
    dt = time.perf_counter() - t0
    one, t1 = 0, time.perf_counter()
    while time.perf_counter() - t1 < single_seconds and one < w.batch.n_ligands:
        oracle.dock_batch(w.batch.subset([one]), w.pocket, w.params, n_threads=1)
        one += 1
    dt1 = time.perf_counter() - t1
    return {"value": done / dt, "unit": "ligands/s", "cores": cores, "kind": "oracle",
            "sample": f"first {done} ligands of {w.name}, {dt:.1f} s, one std::thread per core",
            "single_thread": {"value": one / dt1, "unit": "ligands/s", "cores": 1,
                              "sample": f"first {one} ligands, {dt1:.1f} s"}}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return world, rank, local


def reduce_max(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def run_reference(args, world, rank):
    if rank != 0:
        return
    w = workload_for(args.workload, 0, args.ligands)
    cores = os.cpu_count() or 1
    import oracle
    per_step = max(cores, 8)
    times = []
    i = 0
    for s in range(args.warmup + args.steps):
        idx = [(i + k) % w.batch.n_ligands for k in range(per_step)]
        i += per_step
        t0 = time.perf_counter()
        oracle.dock_batch(w.batch.subset(idx), w.pocket, w.params, n_threads=cores)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    dt = float(np.sum(times))
    v = per_step * args.steps / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "ligands/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(w, "n/a (CPU)"),
        "cpu_baseline": {"value": v, "unit": "ligands/s", "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} ligands per step of {w.name}"},
        "e2e": {"value": v, "unit": "ligands/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


MLP_FLOPS_PER_ROW = 2 * (48 * 256 + 256 * 256 + 256)


def run_learned(args, world, rank, local):
    rec = learned_record(args, world, rank, local, args.workload, args.steps, args.warmup,
                         cpu=not args.no_cpu_baseline)
    if rec is not None:
        print(json.dumps(rec))


def learned_record(args, world, rank, local, workload, steps, warmup, cpu=True):
    """Learned-pruned search vs the plain exhaustive search on the same held-out ligands.

    Training: 12,000 streaming-screen ligands (lognormal sizes) x 256 restarts, targets
    from the plain search; margin tuned for 99.3 % best-pose recall on 4,000 more, so that
    the 16,384 held-out ligands it is timed on keep at least 99 %.  A learned step = features + network + selection + pruned
    search; a plain step = the exhaustive search.  Both device-timed with CUDA events.
    """
    import torch
    from paper_1901_06229_b300 import geodock as gdk, mlp, proposer
    torch.cuda.set_device(local)
    dev = torch.cuda.current_device()
    n_eval = args.ligands or 16384
    if workload == "learned24":  # the proposer's own spec: 24-atom, 4-rotamer ligands
        wt = synth.workload_proposer_train(3907)
        wv = synth.workload_proposer_eval(4000, start=100000)
        we = synth.workload_proposer_eval(n_eval, start=200000 * (rank + 1))
    else:
        wt = synth.workload_stream(12000, seed_offset=50)
        wv = synth.workload_stream(4000, seed_offset=51)
        we = synth.workload_stream(n_eval, seed_offset=52 + 10 * rank)
    ctx = gdk.Context(dev)
    pk = ctx.load_pocket(we.pocket)
    X, t, _ = proposer.dataset(ctx, pk, wt)
    ts, mu, sd = proposer.standardise(t)
    net = mlp.MLP(dev, seed=1, max_batch=4096)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = proposer.train(net, X, ts)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    k = 16
    margin, _ = proposer.tune_margin(ctx, net, pk, wv, k=k, target=VAL_RECALL_TARGET, rule=1, k_fallback=K_FALLBACK)
    L, O = we.batch.n_ligands, we.params.n_orient
    stream = torch.cuda.current_stream()
    job = ctx.prepare_batch(pk, we.batch, we.params, stream=stream, tile=args.tile)
    Xe = torch.empty((L * O, 48), dtype=torch.bfloat16, device="cuda")
    ye = torch.empty(L * O, device="cuda")
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def plain():
        job.launch(stream)

    def learned():
        job.features(x_bf16=Xe, stream=stream)
        net.predict(Xe, ye)
        job.launch_proposed(ye, k, margin, 1, stream, k_fallback=K_FALLBACK)

    times = {}
    clk = ClockSampler(dev).__enter__()
    for name, fn in (("plain", plain), ("learned", learned)):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        ev = []
        for s in range(steps):
            flush.fill_(s & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            ev.append((a, b))
        torch.cuda.synchronize()
        times[name] = reduce_max(sum(a.elapsed_time(b) for a, b in ev) / 1e3, world)
        job.download(stream)
        times[name + "_res"] = job.fetch()
    clk.__exit__(None, None, None)
    cnt, _ = job.selection()
    # each stage of a learned step alone
    def stage_time(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3 / steps
    mlp_s = stage_time(lambda: net.predict(Xe, ye))
    feat_s = stage_time(lambda: job.features(x_bf16=Xe, stream=stream))
    search_s = stage_time(lambda: job.launch_proposed(ye, k, margin, 1, stream, k_fallback=K_FALLBACK))
    ex, pr = times["plain_res"], times["learned_res"]
    recall = float(np.mean(pr["best_score"] == ex["best_score"]))
    be, bp = ex["best_score"].astype(np.int64), pr["best_score"].astype(np.int64)
    regret = float(np.mean((be - bp) / np.maximum(be, 1)))
    job.free()
    pk.free()
    ctx.close()
    if rank != 0:
        return None
    peaks = measured_peaks()
    tflops = MLP_FLOPS_PER_ROW * L * O / mlp_s / 1e12
    peak = peaks.get("bf16_tflops", 1787.5)
    value = L * world * steps / times["learned"]
    plain_v = L * world * steps / times["plain"]
    return {
        "metric": "ligands/s (learned-pruned pose search, 1 B300)", "value": value, "unit": "ligands/s",
        "n_gpus": world, "steps": steps, "warmup": warmup,
        "ms_per_step": 1e3 * times["learned"] / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 search / bf16 network", "data": "synthetic (seeded generators)",
        "config": workload_config(we, "flushed between steps (256 MB write)") | {
            "k": k, "k_fallback": K_FALLBACK,
            "margin_rule": "search the 128 best-predicted restarts when pred(1st) - pred(16th) > margin",
            "margin": margin,
            "train": {"ligands": wt.batch.n_ligands, "rows": int(X.shape[0]), "epochs": len(hist), "seconds": train_s,
                      "final_loss_std_units": hist[-1]}},
        "plain_value": plain_v, "speedup_vs_plain": value / plain_v,
        "best_pose_recall": recall, "recall_target": RECALL_TARGET, "validation_recall_target": VAL_RECALL_TARGET,
        "score_regret": regret, "fallback_fraction": float(np.mean(cnt > k)),
        "restarts_searched_per_ligand": float(cnt.mean()),
        "gpu_launches": steps * 8,  # pose setup + features, MLP, 3 selection kernels, pose setup + search
        "roofline": {"bound": "tensor", "kernel": "mlp_infer_kernel (fused two-layer forward, 1 launch)",
                     "achieved": tflops, "peak": peak, "unit": "TFLOP/s", "frac": tflops / peak,
                     "traffic": MEASURED_MLP_TRAFFIC.get(search_kernel_hash(MLP_KERNEL_SOURCES), {}).get(L * O),
                     "peak_kind": "bf16_tflops of MEASURED_PEAKS.json (burst)"},
        "mlp_rows_per_s": L * O / mlp_s,
        "stage_ms": {"features": 1e3 * feat_s, "network": 1e3 * mlp_s, "select_and_search": 1e3 * search_s},
        "clocks": clk.summary(),
        # the oracle searches every restart (the exhaustive search the learned path prunes)
        "cpu_baseline": cpu_baseline(we) if cpu else None,
    }


def run_mlp(args, world, rank, local):
    """The proposer network's fused tensor-core forward alone: L x 256 rows of 48 BF16
    features (random weights and inputs), rows/s and TFLOP/s against the BF16 peak."""
    import torch
    from paper_1901_06229_b300 import mlp
    torch.cuda.set_device(local)
    rows = (args.ligands or 16384) * 256
    net = mlp.MLP(torch.cuda.current_device(), seed=1, max_batch=1024)
    g = torch.Generator(device="cuda").manual_seed(rank)
    X = torch.rand((rows, 48), device="cuda", generator=g).to(torch.bfloat16)
    y = torch.empty(rows, device="cuda")
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        net.predict(X, y)
    torch.cuda.synchronize()
    barrier(world)
    st = torch.cuda.current_stream()
    ev = []
    with ClockSampler(torch.cuda.current_device()) as clk:
        for s in range(args.steps):
            flush.fill_(s & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            net.predict(X, y)
            b.record(st)
            ev.append((a, b))
        torch.cuda.synchronize()
    t = reduce_max(sum(a.elapsed_time(b) for a, b in ev) / 1e3, world)
    assert net.error() == 0 and bool(torch.isfinite(y).all())
    P = net.get_params()
    Xs = X[:65536].float().cpu().numpy()
    net.close()
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline:  # the FP64 numpy reference of the same forward on a sample
        from oracle import mlp as om
        t0 = time.perf_counter()
        om.forward(P, Xs, rounding=True)
        dt = time.perf_counter() - t0
        cpu = {"value": len(Xs) / dt, "unit": "rows/s", "cores": os.cpu_count() or 1, "kind": "oracle",
               "sample": f"first {len(Xs)} rows, {dt:.1f} s, numpy FP64 (BLAS threads)"}
    tflops = MLP_FLOPS_PER_ROW * rows * world * args.steps / t / 1e12
    peak = measured_peaks().get("bf16_tflops", 1787.5)
    print(json.dumps({
        "metric": "rows/s (proposer network forward, 1 B300)", "value": rows * world * args.steps / t,
        "unit": "rows/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 (fp32 accumulate)", "data": "synthetic (random weights and features)",
        "config": {"workload": f"mlp-48-256-256-1-{rows}rows", "rows": rows, "l2": "flushed between steps"},
        "gpu_launches": args.steps,
        "roofline": {"bound": "tensor", "achieved": tflops, "peak": peak, "unit": "TFLOP/s", "frac": tflops / peak,
                     "traffic": MEASURED_MLP_TRAFFIC.get(search_kernel_hash(MLP_KERNEL_SOURCES), {}).get(rows),
                     "peak_kind": "bf16_tflops of MEASURED_PEAKS.json (burst)"},
        "clocks": clk.summary(), "cpu_baseline": cpu}))


def run_stream(args, world, rank, local):
    """Streaming screen: Poisson arrivals onto the resident pocket with continuous batching,
    learned pruning with fallback, an 8 GB device-memory budget (the context's search
    memory plus the screen's proposer buffers); ligands/s and p50/p99 latency over
    repeated runs of at least `--stream-seconds` each (requests cycle over the
    100,000-ligand library when a run needs more), reported as median and range."""
    import torch
    from paper_1901_06229_b300 import geodock as gdk, proposer, serve
    torch.cuda.set_device(local)
    dev = torch.cuda.current_device()
    n = args.ligands or 100000
    w = synth.workload_stream(n, seed_offset=53 + 10 * rank)
    budget = 8 << 30
    ctx = gdk.Context(dev, mem_budget_bytes=serve.Screen.context_budget(budget, args.max_batch, w.params.n_orient))
    pk = ctx.load_pocket(w.pocket)
    net, margin, info = proposer.fit(ctx, pk, target=VAL_RECALL_TARGET, k_fallback=K_FALLBACK)
    scr = serve.Screen(ctx, pk, w.params, net, k=16, margin=margin, max_batch=args.max_batch, max_inflight=4,
                       k_fallback=K_FALLBACK)
    # warm-up on the first ligands
    warm = w.batch.subset(np.arange(min(2048, n)))
    scr.run(synth.Workload("warm", w.pocket, warm, w.params), np.zeros(warm.n_ligands))
    n_req = max(n, int(np.ceil(args.rate * args.stream_seconds)))
    runs = []
    with ClockSampler(dev) as clk:
        for rep in range(args.stream_repeats):
            arr = serve.poisson_arrivals(n_req, args.rate, seed=rank + 1000 * rep)
            res = scr.run(w, arr, ligand_of=np.arange(n_req) % n)
            runs.append(res.summary())
    pk.free()
    ctx.close()
    if rank != 0:
        return
    def stat(key):
        v = np.array([r[key] for r in runs])
        return {"median": float(np.median(v)), "min": float(v.min()), "max": float(v.max())}
    thr, p50, p99 = stat("ligands_per_s"), stat("p50_ms"), stat("p99_ms")
    print(json.dumps({
        "metric": "ligands/s and per-ligand latency (streaming screen, 1 B300)", "value": thr["median"],
        "unit": "ligands/s", "n_gpus": world, "steps": args.stream_repeats, "warmup": 1, "ms_per_step": None,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 search / bf16 network",
        "data": "synthetic (seeded generators)",
        "config": workload_config(w, "resident pocket; no flush (serving)") | {
            "arrivals": f"Poisson, {args.rate:g} ligands/s", "requests_per_run": n_req,
            "runs": args.stream_repeats, "max_batch": args.max_batch, "inflight": 4, "budget_bytes": budget,
            "k": 16, "k_fallback": K_FALLBACK, "margin": margin, "proposer": info},
        "ligands_per_s": thr, "latency_ms": {"p50": p50, "p99": p99}, "runs": runs, "clocks": clk.summary()}))


def run_serve(args, world, rank, local):
    rec = serve_record(args, world, rank, local, args.stream_repeats, args.stream_seconds)
    if rec is not None:
        print(json.dumps(rec))


def serve_record(args, world, rank, local, repeats, seconds):
    """Streaming screen on the device queue: Poisson arrivals submitted to one running
    search launch (gd_server: continuous batching on the device, plain exhaustive search
    of every restart), results collected as they finish; ligands/s and per-ligand latency
    (finish seen on the host minus arrival) over `repeats` runs of at least `seconds` of
    arrivals each, median and range."""
    import torch
    from paper_1901_06229_b300 import geodock as gdk, serve
    torch.cuda.set_device(local)
    dev = torch.cuda.current_device()
    n = args.ligands or 100000
    w = synth.workload_stream(n, seed_offset=53 + 10 * rank)
    ctx = gdk.Context(dev, mem_budget_bytes=8 << 30)
    pk = ctx.load_pocket(w.pocket)
    R = np.diff(w.batch.rot_off)
    srv = gdk.Server(ctx, pk, w.params, capacity=args.max_batch * 4, max_atoms=256, max_rotamers=int(R.max()),
                     idle_ms=200, tile=max(args.tile, 0))
    # warm-up: the first ligands at once
    warm = min(2048, n)
    srv.submit(w.batch, np.arange(warm))
    got = 0
    while got < warm:
        got += len(srv.collect()[0])
    n_req = max(n, int(np.ceil(args.rate * seconds)))
    runs = []
    with ClockSampler(dev) as clk:
        for rep in range(repeats):
            arr = serve.poisson_arrivals(n_req, args.rate, seed=rank + 1000 * rep)
            lig = np.arange(n_req) % n
            done_t = np.zeros(n_req)
            seq0 = None
            nxt = finished = 0
            t0 = time.perf_counter()
            while finished < n_req:
                now = time.perf_counter() - t0
                hi = int(np.searchsorted(arr, now, side="right"))
                if hi > nxt:
                    take = min(hi, nxt + srv.capacity // 2)
                    try:
                        q = srv.submit(w.batch, lig[nxt:take])
                        seq0 = q - nxt if seq0 is None else seq0
                        nxt = take
                    except gdk.GeoDockError as e:
                        if e.status != gdk.GD_EBUSY:
                            raise
                seqs, _, _ = srv.collect(8192)
                if len(seqs):
                    done_t[seqs.astype(np.int64) - seq0] = time.perf_counter() - t0
                    finished += len(seqs)
                elif hi == nxt:
                    time.sleep(5e-5)
            lat = done_t - arr
            span = float(done_t.max() - arr.min())
            runs.append({"ligands_per_s": n_req / span, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                         "p99_ms": 1e3 * float(np.percentile(lat, 99)), "ligands": n_req})
    st = srv.stats()
    srv.close()
    pk.free()
    ctx.close()
    if rank != 0:
        return None

    def stat(key):
        v = np.array([r[key] for r in runs])
        return {"median": float(np.median(v)), "min": float(v.min()), "max": float(v.max())}
    return {
        "metric": "ligands/s and per-ligand latency (device-queue screen, 1 B300)",
        "value": stat("ligands_per_s")["median"], "unit": "ligands/s", "n_gpus": world,
        "steps": repeats, "warmup": 1, "ms_per_step": None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded generators)",
        "config": workload_config(w, "resident pocket; no flush (serving)") | {
            "arrivals": f"Poisson, {args.rate:g} ligands/s", "requests_per_run": n_req, "runs": repeats,
            "search": "every restart (plain method)", "capacity": srv.capacity, "budget_bytes": 8 << 30},
        "ligands_per_s": stat("ligands_per_s"), "latency_ms": {"p50": stat("p50_ms"), "p99": stat("p99_ms")},
        "server": st, "runs": runs, "clocks": clk.summary()}


def run_serve_learned(args, world, rank, local):
    rec = serve_learned_record(args, world, rank, local, args.stream_repeats, args.stream_seconds)
    if rec is not None:
        print(json.dumps(rec))


def serve_learned_record(args, world, rank, local, repeats, seconds):
    """The learned screen on the device queue: Poisson arrivals proposed in batches
    (features, network, top-16 with the spread fallback to the best 128) on SMs the
    server leaves free, each ligand then joining the running search launch with its
    restart list; ligands/s and per-ligand latency over `repeats` runs of at least
    `seconds` of arrivals, median and range."""
    import torch
    from paper_1901_06229_b300 import geodock as gdk, proposer, serve
    torch.cuda.set_device(local)
    dev = torch.cuda.current_device()
    n = args.ligands or 100000
    w = synth.workload_stream(n, seed_offset=53 + 10 * rank)
    ctx = gdk.Context(dev, mem_budget_bytes=8 << 30)
    pk = ctx.load_pocket(w.pocket)
    net, margin, info = proposer.fit(ctx, pk, target=VAL_RECALL_TARGET, k_fallback=K_FALLBACK)
    R = np.diff(w.batch.rot_off)
    free_sms = SERVE_LEARNED_FREE_SMS
    scr = serve.QueueScreen(ctx, pk, w.params, net, k=16, margin=margin, k_fallback=K_FALLBACK,
                            max_batch=args.max_batch, free_sms=free_sms, max_rotamers=int(R.max()),
                            warm_library=w.batch)
    warm = min(2048, n)
    scr.run(synth.Workload("warm", w.pocket, w.batch.subset(np.arange(warm)), w.params), np.zeros(warm))
    n_req = max(n, int(np.ceil(args.rate * seconds)))
    runs = []
    with ClockSampler(dev) as clk:
        for rep in range(repeats):
            arr = serve.poisson_arrivals(n_req, args.rate, seed=rank + 1000 * rep)
            runs.append(scr.run(w, arr, ligand_of=np.arange(n_req) % n).summary())
    st = scr.srv.stats()
    scr.close()
    pk.free()
    ctx.close()
    if rank != 0:
        return None

    def stat(key):
        v = np.array([r[key] for r in runs])
        return {"median": float(np.median(v)), "min": float(v.min()), "max": float(v.max())}
    return {
        "metric": "ligands/s and per-ligand latency (learned screen on the device queue, 1 B300)",
        "value": stat("ligands_per_s")["median"], "unit": "ligands/s", "n_gpus": world, "steps": repeats,
        "warmup": 1, "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 search / bf16 network", "data": "synthetic (seeded generators)",
        "config": workload_config(w, "resident pocket; no flush (serving)") | {
            "arrivals": f"Poisson, {args.rate:g} ligands/s", "requests_per_run": n_req, "runs": repeats,
            "k": 16, "k_fallback": K_FALLBACK, "margin": margin, "free_sms": free_sms, "server_tile": 8,
            "max_batch": args.max_batch, "proposer": info},
        "ligands_per_s": stat("ligands_per_s"), "latency_ms": {"p50": stat("p50_ms"), "p99": stat("p99_ms")},
        "restarts_per_ligand": stat("restarts_per_ligand"), "server": st, "runs": runs, "clocks": clk.summary()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched",
                    choices=["batched", "large", "single", "learned", "learned24", "stream", "serve", "serve_learned",
                             "mlp"])
    ap.add_argument("--rate", type=float, default=100000.0, help="stream: Poisson arrival rate (ligands/s)")
    ap.add_argument("--max-batch", type=int, default=2048, help="stream: largest admitted batch")
    ap.add_argument("--stream-seconds", type=float, default=3.0, help="stream: least offered duration of a run")
    ap.add_argument("--stream-repeats", type=int, default=5, help="stream: runs (median and range reported)")
    ap.add_argument("--tile", type=int, default=-1, help="-1 autotune, 0 default, >0 tile id")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--ligands", type=int, default=None, help="smaller batch (profiling runs only)")
    ap.add_argument("--sub", default="large,learned24,serve",
                    help="batched line: other workloads measured after it (large, learned24, learned, serve)")
    ap.add_argument("--no-sub", action="store_true", help="batched line only")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    assert args.warmup >= 3 or args.steps <= 3, "at least 3 warm-up steps"
    if args.workload in ("learned", "learned24"):
        run_learned(args, world, rank, local)
        return
    if args.workload == "stream":
        run_stream(args, world, rank, local)
        return
    if args.workload == "serve":
        run_serve(args, world, rank, local)
        return
    if args.workload == "serve_learned":
        run_serve_learned(args, world, rank, local)
        return
    if args.workload == "mlp":
        run_mlp(args, world, rank, local)
        return

    import torch
    from paper_1901_06229_b300 import geodock as gdk

    torch.cuda.set_device(local)
    dev = torch.cuda.current_device()
    w = workload_for(args.workload, rank, args.ligands)
    stream = torch.cuda.Stream()
    ctx = gdk.Context(dev)
    pk = ctx.load_pocket(w.pocket)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    # ---- value: device-resident inputs, one graph replay per step -------------------------
    tile = resolve_tile(ctx, pk, w, args.tile, stream)
    d = time_search(ctx, pk, w, tile, args.steps, args.warmup, stream, flush, world)
    first, res, dev_s, clocks = d["first"], d["res"], d["dev_s"], d["clocks"]
    L = w.batch.n_ligands
    value = L * world * args.steps / dev_s
    ms_step = 1e3 * dev_s / args.steps

    # ---- e2e: host buffers through the public API --------------------------------------------
    # at least 20 batches: the first batch's packing and copy, before any search runs, and
    # the last one's result copy are paid once per run, not per batch (the line records
    # the count it used)
    e2e_steps = args.e2e_steps or max(args.steps, 20)
    # gd_dock_batch returns once the work is queued, so a streaming caller packs and
    # submits batch k+1 while batch k runs; two jobs are in flight, on two streams, so one
    # job's copies run on the copy engines while the other's search runs
    streams = [stream, torch.cuda.Stream()]
    for _ in range(2):  # warm the context's memory caches with two jobs alive at once
        warm = [ctx.dock_batch(pk, w.batch, w.params, stream=s, tile=tile) for s in streams]
        for j in warm:
            j.fetch()
            j.free()
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    inflight = []
    for step in range(e2e_steps):
        inflight.append(ctx.dock_batch(pk, w.batch, w.params, stream=streams[step % 2], tile=tile))
        if len(inflight) == 2:
            j = inflight.pop(0)
            out = j.fetch()
            h2d, d2h = j.bytes_moved()
            j.free()
    while inflight:
        j = inflight.pop(0)
        out = j.fetch()
        h2d, d2h = j.bytes_moved()
        j.free()
    e2e_s = reduce_max(time.perf_counter() - t0, world)
    assert np.array_equal(out["best_score"], first["best_score"])
    e2e = {"value": L * world * e2e_steps / e2e_s, "unit": "ligands/s", "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(d2h), "steps": e2e_steps, "jobs_in_flight": 2, "streams": 2}

    pk.free()
    if rank != 0:
        ctx.close()
        return

    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    pipes = gdk.measure_peaks(torch.cuda.current_device())  # own microbenchmarks, after the timed region
    roof = search_roofline(w, tile, res, d["kernel_ms"], sm_count, pipes)
    line = {
        "metric": METRIC, "value": value, "unit": "ligands/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded generators; no public dataset)",
        "config": workload_config(w, "flushed between steps (256 MB write)") | {
            "tile": tile, "tile_warps_slots_regs": list(gdk.tile_info(tile)) if tile > 0 else None,
            "launch": d["info"]},
        "pose_evals_per_s": float(res["evals"].sum()) * world * args.steps / dev_s,
        "pair_tests_per_s": float(res["pair_tests"].sum()) * world * args.steps / dev_s,
        "e2e": e2e,
        "gpu_launches": 2 * args.steps,  # pose setup + search per step
        "roofline": roof,
        "clocks": clocks,
        "wall_s_timed": d["wall"],
    }
    # the other workloads of the method, measured after the headline one on the same GPU:
    # large flexible ligands (plain search) and the learned proposer (trained here on the
    # GPU, then learned-pruned against the plain search); one GPU only
    subs = [] if (args.no_sub or world > 1 or args.workload != "batched") else args.sub.split(",")
    if "large" in subs:
        line["large"] = large_record(ctx, args, world, stream, flush, sm_count, pipes)
    ctx.close()
    del flush
    for name in subs:
        if name in ("learned", "learned24"):
            rec = learned_record(args, world, rank, local, name, min(args.steps, 20), args.warmup, cpu=False)
            line[name] = learned_summary(rec)
        if name == "serve":
            # the device-queue screen at the offered rate, shorter runs than --workload serve
            rec = serve_record(args, world, rank, local, SERVE_SUB_REPEATS, SERVE_SUB_SECONDS)
            line[name] = {k: rec[k] for k in rec if k != "runs"}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    print(json.dumps(line))


def resolve_tile(ctx, pk, w, tile, stream):
    if tile == -1:
        tile, _ = ctx.autotune(pk, w.batch, w.params, max_ligands=512, stream=stream)
    return tile


def time_search(ctx, pk, w, tile, steps, warmup, stream, flush, world):
    """Device time of `steps` search launches (graph replays) on a resident batch, the L2
    flushed before each outside the timed events; clocks sampled meanwhile."""
    import torch
    job = ctx.dock_batch(pk, w.batch, w.params, stream=stream, tile=tile)
    first = job.fetch()
    info = job.info()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            flush.fill_(1)
            job.launch(stream)
    torch.cuda.synchronize()
    barrier(world)
    with ClockSampler(torch.cuda.current_device()) as clk:
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for k in range(steps):
                flush.fill_(k & 0xFF)  # evict the L2 (256 MB > 126 MB) outside the timed events
                ev[k][0].record(stream)
                job.launch(stream)
                ev[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    barrier(world)
    kernel_ms = [a.elapsed_time(b) for a, b in ev]
    dev_s = reduce_max(sum(kernel_ms) / 1e3, world)
    job.download(stream)
    res = job.fetch()
    assert np.array_equal(res["best_score"], first["best_score"]), "relaunch changed results"
    job.free()
    return dict(first=first, res=res, kernel_ms=kernel_ms, dev_s=dev_s, wall=wall, clocks=clk.summary(), info=info)


def search_roofline(w, tile, res, kernel_ms, sm_count, pipes):
    """Roofline of the search kernel.  The bound it meets is instruction issue: warp
    instructions per launch (ncu, keyed by the kernel-source hash) over the launch time,
    against 4 schedulers per SM per clock.  Beside it: the method's own work rate (the
    oracle's FP32 count over the FP32 peak, above 1 because the exact reach filter skips
    most pair tests that count charges) and the FP32 operations the kernel executes."""
    peaks = measured_peaks()
    mhz = peaks.get("sm_max_mhz", 2032.0)
    launch_s = float(np.mean(kernel_ms)) / 1e3
    evals, pairs, moves = (float(res[k].sum()) for k in ("evals", "pair_tests", "atom_moves"))
    peak_tops = sm_count * FP32_LANES_PER_SM * mhz * 1e6 / 1e12
    peak_loads = sm_count * LOADS_PER_SM_CLK * mhz * 1e6 / 1e12
    peak_issue = sm_count * ISSUE_PER_SM_CLK * mhz * 1e6 / 1e12
    exec_ops = EXEC_OPS_PER_PAIR * pairs + EXEC_OPS_PER_ATOM_MOVE * moves
    executed = {"achieved": exec_ops / launch_s / 1e12, "peak": peak_tops, "unit": "TFLOP/s",
                "frac": exec_ops / launch_s / 1e12 / peak_tops, "ops_per_launch": exec_ops,
                "note": "FP32 operations the kernel performs: 3 per pair test it runs, 6 per turned atom"}
    h = search_kernel_hash()
    inst = MEASURED_INSTRUCTIONS.get(h, {}).get((w.name, tile))
    achieved = inst / launch_s / 1e12 if inst else None
    alg = algorithmic_work(w.name, evals, moves)
    if alg:
        work_ach = alg["fp32_ops"] / launch_s / 1e12
        loads = alg["byte_loads"] / launch_s / 1e12
        work = {"achieved": work_ach, "peak": peak_tops, "unit": "TFLOP/s (method's count)",
                "frac": max(work_ach / peak_tops, loads / peak_loads),
                "note": "the oracle's count of the method's work (16 FP32 ops + 1 byte load per fragment atom, "
                        "7 ops per early-exit pair test, 32-pair tiles) per second over the FP32 pipe's peak; "
                        "above 1 because the exact reach filter proves most of those pair tests unnecessary",
                "ops_per_launch": alg["fp32_ops"], "byte_loads_per_launch": alg["byte_loads"],
                "candidates_per_launch": alg["candidates"], "pair_tests_early_per_launch": alg["pair_tests_early"],
                "pair_tests_full_per_launch": alg["pair_tests_full"],
                "loads": {"achieved": loads, "peak": peak_loads, "unit": "Tloads/s", "frac": loads / peak_loads}}
    else:
        work_ach = loads = None
        work = {"note": "no oracle work table for this workload"}
    return {
        "bound": "issue", "kernel": "search_kernel (fused a3-a10 persistent launch)",
        "achieved": achieved, "peak": peak_issue, "unit": "T warp-instructions/s",
        "frac": achieved / peak_issue if achieved else None,
        "instructions_per_launch": inst,
        "instructions_from": (f"ncu smsp__inst_executed.sum of this kernel source (hash {h}) on this workload and tile"
                              if inst else f"not measured for kernel source hash {h}: frac withheld"),
        "traffic": MEASURED_TRAFFIC.get(h, {}).get((w.name, tile)),
        "peak_kind": f"{sm_count} SMs x {ISSUE_PER_SM_CLK} schedulers x {mhz:.0f} MHz (sm_max_mhz of "
                     "MEASURED_PEAKS.json)",
        "work_rate_vs_fp32_peak": work, "executed": executed,
        "microbenchmark": pipe_peaks(pipes, work_ach, loads, peak_tops, peak_loads),
    }


def large_record(ctx, args, world, stream, flush, sm_count, pipes):
    """Large flexible ligands (512 ligands of 100-250 atoms, 20-60 rotamers, 128^3 pocket,
    256 restarts x 128 angles): the plain search, device-resident, autotuned."""
    w = synth.workload_large(512)
    pk = ctx.load_pocket(w.pocket)
    tile = resolve_tile(ctx, pk, w, -1, stream)
    steps = min(args.steps, 20)
    d = time_search(ctx, pk, w, tile, steps, args.warmup, stream, flush, world)
    pk.free()
    res = d["res"]
    return {"metric": "ligands/s (pose search, large ligands, 1 B300)",
            "value": w.batch.n_ligands * steps / d["dev_s"], "unit": "ligands/s", "steps": steps,
            "ms_per_step": 1e3 * d["dev_s"] / steps,
            "pose_evals_per_s": float(res["evals"].sum()) * steps / d["dev_s"],
            "pair_tests_per_s": float(res["pair_tests"].sum()) * steps / d["dev_s"],
            "config": workload_config(w, "flushed between steps (256 MB write)") | {"tile": tile, "launch": d["info"]},
            "roofline": search_roofline(w, tile, res, d["kernel_ms"], sm_count, pipes), "clocks": d["clocks"],
            "gpu_launches": 2 * steps}


def learned_summary(rec):
    keep = ("metric", "value", "unit", "steps", "ms_per_step", "plain_value", "speedup_vs_plain", "best_pose_recall",
            "recall_target", "score_regret", "fallback_fraction", "restarts_searched_per_ligand", "roofline",
            "stage_ms", "clocks", "gpu_launches")
    out = {k: rec[k] for k in keep if k in rec}
    cfg = rec["config"]
    out["config"] = {k: cfg[k] for k in ("workload", "ligands", "atoms", "orientations", "angles", "k", "k_fallback",
                                         "margin", "train") if k in cfg}
    out["beats_plain_at_target_recall"] = bool(rec["value"] > rec["plain_value"] and
                                               rec["best_pose_recall"] >= rec["recall_target"])
    return out


if __name__ == "__main__":
    main()
