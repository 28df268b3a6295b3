"""Failure reporting without a GPU fault: a device wait that runs out.

The search kernels that stage the pocket grid in shared memory wait on an mbarrier for
the bulk copies, with a bound of about two seconds.  GD_FLAG_TEST_STAGE_TIMEOUT makes
the barrier expect 16 bytes more than are copied, so the wait runs out (the copies all
land; nothing faults or hangs): every block records the timeout and returns, the job
reports GD_ETIMEOUT, and the same context docks correctly afterwards.
"""
import time

import numpy as np
import pytest

from paper_1901_06229_b300 import geodock as gdk
from paper_1901_06229_b300 import synth

pytestmark = pytest.mark.gpu

STAGED_TILE = 10  # 2 warps x 1 angle per lane, 128-register build: stages a grid that fits


def test_staging_timeout_is_reported_and_the_context_survives():
    assert gdk.tile_info(STAGED_TILE)[2] == 128
    ctx = gdk.Context(0)
    w = synth.workload_single()  # 32^3 pocket: the grid is staged in shared memory
    pk = ctx.load_pocket(w.pocket)
    ref = ctx.dock_batch(pk, w.batch, w.params, tile=STAGED_TILE)
    want = ref.fetch()
    ref.free()
    job = ctx.dock_batch(pk, w.batch, w.params, tile=STAGED_TILE, test_stage_timeout=True)
    t0 = time.perf_counter()
    with pytest.raises(gdk.GeoDockError, match="GD_ETIMEOUT"):
        job.fetch()
    waited = time.perf_counter() - t0
    job.free()
    assert 0.5 < waited < 30.0, waited  # the bounded wait (about 2 s), not an immediate error
    again = ctx.dock_batch(pk, w.batch, w.params, tile=STAGED_TILE)
    got = again.fetch()
    again.free()
    for key in ("best_score", "best_orient", "best_angle", "best_xyz"):
        np.testing.assert_array_equal(got[key], want[key], err_msg=key)
    pk.free()
    ctx.close()
