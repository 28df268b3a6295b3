"""The parity helpers themselves (CPU): the oracle compared with itself passes with every
step compared, a changed pick at a step the oracle flags fragile counts as a legitimate
parting of trajectories, and a changed pick, score, bump flag or coordinate anywhere else
fails."""
import numpy as np
import pytest

import oracle
from paper_1901_06229_b300 import synth
from parity import compare_debug
from test_oracle_pins import textured_pocket


def _as_device(orc, batch, params):
    """The oracle's results in the layout the library returns (bump bits 0/1)."""
    O, reps = params.n_orient, params.repetitions
    ro = np.asarray(batch.rot_off, np.int64)
    best_angle = np.zeros(int(ro[-1]) * reps, np.int16)
    for i in range(batch.n_ligands):
        S = int(ro[i + 1] - ro[i]) * reps
        b = int(orc["best_orient"][i])
        base = int(ro[i]) * reps * O
        best_angle[ro[i] * reps: ro[i] * reps + S] = orc["orient_pick"][base + b * S: base + (b + 1) * S]
    return dict(orient_pick=orc["orient_pick"].copy(), orient_score=orc["orient_score"].astype(np.uint32),
                bump_bits=(orc["bump"] == 1).astype(np.uint8), best_orient=orc["best_orient"].copy(),
                best_score=orc["best_score"].astype(np.uint32), evals=orc["evals"].copy(),
                pair_tests=orc["pair_tests_full"].copy(), atom_moves=np.ones(batch.n_ligands, np.uint64),
                best_xyz=orc["best_xyz"].astype(np.float32), best_angle=best_angle)


@pytest.fixture(scope="module")
def case():
    w = synth.workload_single()
    P = textured_pocket()
    orc = oracle.dock_batch(w.batch, P, w.params, n_threads=8, debug=True)
    assert orc["orient_step_fragile"].sum() > 0, "the case needs fragile steps"
    return w, orc


def test_oracle_against_itself_compares_every_step(case):
    w, orc = case
    st = compare_debug(_as_device(orc, w.batch, w.params), orc, w.batch, w.params, min_compared=1.0)
    assert st["picks_compared"] == st["steps_total"] == 64 * 4 and st.get("diverged_restarts", 0) == 0
    assert st["fragile_steps"] == int((orc["orient_step_fragile"] & 1).sum()) > 0


def test_other_pick_at_a_fragile_step_parts_the_trajectories(case):
    w, orc = case
    g = _as_device(orc, w.batch, w.params)
    s = int(np.flatnonzero(orc["orient_step_fragile"] & 1)[0])
    g["orient_pick"][s] = (g["orient_pick"][s] + 1) % w.params.n_angles
    o, step = divmod(s, 4)
    g["orient_score"][0, o] += 7  # after parting, the restart's score is not compared
    g["best_orient"][0] = int(np.argmax(g["orient_score"][0]))
    g["best_score"][0] = g["orient_score"][0].max()
    st = compare_debug(g, orc, w.batch, w.params)
    assert st["diverged_restarts"] == 1 and st["picks_compared"] == 64 * 4 - (4 - step)


@pytest.mark.parametrize("what", ["pick", "score", "bump", "coords"])
def test_planted_mistakes_fail(case, what):
    w, orc = case
    g = _as_device(orc, w.batch, w.params)
    robust = np.flatnonzero(orc["orient_fragile"][0] < 0)
    o = int(robust[len(robust) // 2])
    if what == "pick":
        g["orient_pick"][o * 4 + 1] = (g["orient_pick"][o * 4 + 1] + 1) % w.params.n_angles
    elif what == "score":
        g["orient_score"][0, o] = orc["orient_score_hi"][0, o] + 1
    elif what == "bump":
        k = int(np.flatnonzero(orc["bump"][o * 4 * 32: (o + 1) * 4 * 32] == 0)[0])
        g["bump_bits"][o * 4 * 32 + k] = 1
    else:
        g["best_xyz"][0, 0] += 2e-4
    with pytest.raises(AssertionError):
        compare_debug(g, orc, w.batch, w.params)
