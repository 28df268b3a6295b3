"""Algorithmic work of the benchmark workloads, counted by the oracle.

TEST INFRASTRUCTURE ONLY (like the rest of this package).  Runs the FP64 oracle over
each whole seeded benchmark workload once and writes the per-launch totals to
``algorithmic_work.json`` beside this file; the benchmark reads that table as plain data
to state the work one search launch does, independently of how the kernel does it.

Work of one candidate (one restart x rotamer x angle of the sweep, Sec. 3.1):
  * rotation: 9 FP32 operations per fragment atom (a 3 x 3 matrix-vector product with
    the angle's matrix precomputed);
  * grid gather: 7 operations per fragment atom (3 to cell coordinates, 3 float-to-int
    conversions, 1 index multiply-add) and one byte load;
  * bump check (BumpCheck, Sec. 3.2): 7 FP32 operations per pair tested, where the
    candidate tests its pairs moving atom ascending, then static atom ascending, and
    stops at the first bump, in whole 32-pair tiles (``pair_tests_early``).

Usage: python -m oracle.algorithmic_work [--threads N] [workload ...]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
from paper_1901_06229_b300 import synth  # noqa: E402

TABLE = os.path.join(HERE, "algorithmic_work.json")
WORKLOADS = {"single": synth.workload_single, "batched": synth.workload_batched, "large": synth.workload_large}
ROTATION_OPS_PER_ATOM = 9
GATHER_OPS_PER_ATOM = 7
BUMP_OPS_PER_PAIR = 7


def frag_atoms(batch, params) -> int:
    """Sum over candidates of the moving fragment's atom count."""
    total = 0
    for i in range(batch.n_ligands):
        lig = batch.ligand(i)
        n = len(lig.xyz)
        total += sum(int(oracle.fragment(n, lig.bonds, int(rb))[0].sum()) for rb in lig.rot_bond)
    return total * params.n_orient * params.n_angles * params.repetitions


def count(w, threads: int, chunk: int = 128) -> dict:
    L = w.batch.n_ligands
    early = full = cand = 0
    for s in range(0, L, chunk):
        sub = w.batch.subset(list(range(s, min(L, s + chunk))))
        out = oracle.dock_batch(sub, w.pocket, w.params, n_threads=threads)
        early += int(out["pair_tests_early"].sum())
        full += int(out["pair_tests_full"].sum())
        cand += int(out["evals"].sum())
    moves = frag_atoms(w.batch, w.params)
    fp32 = (ROTATION_OPS_PER_ATOM + GATHER_OPS_PER_ATOM) * moves + BUMP_OPS_PER_PAIR * early
    return {"ligands": L, "candidates": cand, "frag_atom_moves": moves, "pair_tests_early": early,
            "pair_tests_full": full, "fp32_ops": fp32, "byte_loads": moves}


def load() -> dict:
    with open(TABLE) as f:
        return json.load(f)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workloads", nargs="*", default=list(WORKLOADS))
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    table = load() if os.path.exists(TABLE) else {}
    for name in args.workloads:
        w = WORKLOADS[name]()
        t0 = time.perf_counter()
        table[w.name] = count(w, args.threads)
        print(f"{w.name}: {table[w.name]} ({time.perf_counter() - t0:.0f} s)", flush=True)
        with open(TABLE, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
            f.write("\n")


if __name__ == "__main__":
    main()
