"""gd_dock_batch_noalloc, the entry point for callers that cannot allocate.

Some callers cannot allocate device memory when they dock: their device memory is
already reserved by another framework's caching allocator, their service forbids
allocation after start-up, or they cannot afford the device-wide synchronisation of
cudaMalloc/cudaFree.  gd_dock_batch_noalloc runs the same search kernel with all of
its working memory in the library's fixed __device__ array.  These tests call it
through the C ABI twice in a row and check every result against gd_dock_batch (which
allocates per job); this file is collected last so that a failure here does not stop
the rest of the GPU suite.
"""
import numpy as np
import pytest

from paper_1901_06229_b300 import geodock as gdk
from paper_1901_06229_b300 import synth

pytestmark = pytest.mark.gpu

KEYS = ("best_score", "best_orient", "best_angle", "best_xyz", "evals", "pair_tests", "atom_moves",
        "reach_tests")


def test_noalloc_matches_dock_batch_on_two_calls_in_a_row():
    w = synth.workload_batched(96)
    ref = gdk.dock(w.batch, w.pocket, w.params)          # allocating entry point
    for call in range(2):
        out = gdk.dock_noalloc(w.batch, w.pocket, w.params)
        for k in KEYS:  # bitwise: the same kernel on the same packed inputs
            np.testing.assert_array_equal(out[k], ref[k], err_msg=f"call {call}: {k}")


def test_noalloc_second_shape_reuses_the_array():
    # a different pocket (global-memory grid path), ligand sizes and angle count after
    # the first call: nothing from the previous call may leak into this one
    w = synth.workload_large(3)
    params = synth.SearchParams(2, 2, 2, 128)
    ref = gdk.dock(w.batch, w.pocket, params)
    for call in range(2):
        out = gdk.dock_noalloc(w.batch, w.pocket, params)
        for k in KEYS:
            np.testing.assert_array_equal(out[k], ref[k], err_msg=f"call {call}: {k}")


def test_noalloc_rejects_batches_beyond_its_fixed_memory():
    w = synth.workload_batched(64)
    big = synth.SearchParams(32, 32, 32, 64)  # 32,768 restarts: per-restart scratch > 64 MiB
    with pytest.raises(gdk.GeoDockError) as e:
        gdk.dock_noalloc(w.batch, w.pocket, big)
    assert e.value.status == gdk.GD_EINVAL and "working memory" in str(e.value)
