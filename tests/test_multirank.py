"""The benchmark's multi-rank path on CPU: two gloo ranks on 127.0.0.1.

Under torchrun every rank docks its own batch (weak scaling, no collective on the data
path); the ranks meet only in a barrier and a max-reduction of their timings, and only
rank 0 prints (and runs the reference arm).  These run the same helpers bench.py uses.
"""
import importlib.util
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    b = _bench()
    w, r, local = b.dist_setup()
    assert (w, r, local) == (world, rank, rank)
    b.barrier(w)
    got = b.reduce_max(10.0 * (rank + 1), w)  # each rank's "elapsed time"
    b.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(repr(got))


def test_two_gloo_ranks_reduce_the_slowest_time(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for rank in range(2):
        assert float((tmp_path / f"rank{rank}.txt").read_text()) == 20.0


@pytest.mark.parametrize("name, n", [("batched", 6), ("large", 3)])
def test_ranks_dock_disjoint_equal_shards(name, n):
    b = _bench()
    w0, w1 = b.workload_for(name, 0, n), b.workload_for(name, 1, n)
    assert w0.batch.n_ligands == w1.batch.n_ligands == n  # weak scaling: the same work per rank
    assert w0.params == w1.params
    np.testing.assert_array_equal(w0.pocket.grid, w1.pocket.grid)  # the pocket is replicated
    # rank 1 takes the ligands after rank 0's: its first ligand is the global ligand n
    both = b.workload_for(name, 0, 2 * n)
    x1 = np.asarray(w1.batch.xyz)
    k = int(both.batch.atom_off[n])
    np.testing.assert_array_equal(x1, np.asarray(both.batch.xyz)[k:k + len(x1)])
    assert not np.array_equal(np.asarray(w0.batch.xyz)[:10], x1[:10])


def test_only_rank0_runs_the_reference_arm(capsys):
    b = _bench()

    class Args:
        workload, ligands, steps, warmup, gpus = "single", None, 1, 0, 2

    assert b.run_reference(Args, 2, 1) is None
    assert capsys.readouterr().out == ""
