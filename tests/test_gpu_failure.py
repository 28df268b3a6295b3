"""Failure reporting without a GPU fault: a device wait that runs out.

The search kernels that stage the pocket grid in shared memory wait on an mbarrier for
the bulk copies, with a bound of about two seconds.  GD_FLAG_TEST_STAGE_TIMEOUT makes
the barrier expect 16 bytes more than are copied, so the wait runs out (the copies all
land; nothing faults or hangs): every block records the timeout and returns, the job
reports GD_ETIMEOUT, and the same context docks correctly afterwards.

The proposer network's tensor-core kernels wait on their MMA commits with the same
bound.  gd_mlp_test_hold makes the next launch withhold its first commit (the MMAs still
run): the wait runs out, the kernel drains its MMAs with one more commit before freeing
its tensor memory, and the model's error flag is set; once cleared, the same model
computes what an untouched one does.
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


def _mlp_case(M, seed=11):
    import torch
    from paper_1901_06229_b300 import mlp
    rng = np.random.default_rng(seed)
    from oracle import mlp as om
    P = rng.normal(scale=0.15, size=om.NPARAM).astype(np.float32)
    X = torch.tensor(rng.uniform(0, 1, size=(M, 48)).astype(np.float32)).to(torch.bfloat16).cuda()
    t = torch.tensor(rng.uniform(0, 1, size=M).astype(np.float32)).cuda()
    nets = []
    for _ in range(2):
        net = mlp.MLP(0, seed=1, max_batch=1024)
        net.set_params(P)
        nets.append(net)
    return nets, X, t


@pytest.mark.parametrize("M", [1000, 40000])  # one tile per CTA; several (the tile loop's waits)
def test_mlp_inference_wait_runs_out_and_the_model_recovers(M):
    import torch
    (net, ref), X, _ = _mlp_case(M)
    want = torch.empty(M, device="cuda")
    ref.predict(X, want)
    y = torch.empty(M, device="cuda")
    net.test_hold(True)
    t0 = time.perf_counter()
    net.predict(X, y)
    torch.cuda.synchronize()
    waited = time.perf_counter() - t0
    assert net.error() == 1
    assert 0.5 < waited < 60.0, waited  # the bounded waits, not an immediate error
    net.test_hold(False)
    assert net.error() == 0
    net.predict(X, y)
    torch.cuda.synchronize()
    assert net.error() == 0 and ref.error() == 0
    assert torch.equal(y, want)
    net.close()
    ref.close()


def test_mlp_gemm_wait_runs_out_and_the_model_recovers():
    import torch
    (net, ref), X, t = _mlp_case(1024, seed=12)
    n = ref.nparam
    g_want, g = torch.empty(n, device="cuda"), torch.empty(n, device="cuda")
    l_want, l = torch.zeros(1, device="cuda"), torch.zeros(1, device="cuda")
    ref.gradients(X, t, g_want, l_want, B=1024)
    net.test_hold(True)  # the first GEMM of the forward pass
    t0 = time.perf_counter()
    net.gradients(X, t, g, l, B=1024)
    torch.cuda.synchronize()
    waited = time.perf_counter() - t0
    assert net.error() == 1
    assert 0.5 < waited < 60.0, waited
    net.test_hold(False)
    net.gradients(X, t, g, l, B=1024)
    torch.cuda.synchronize()
    assert net.error() == 0 and ref.error() == 0
    assert torch.equal(g, g_want)  # the loss is summed with atomics: equal to rounding
    assert torch.allclose(l, l_want, rtol=1e-5, atol=0)
    net.close()
    ref.close()

