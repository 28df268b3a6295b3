"""Element-by-element comparison of the CUDA library's results with the FP64 oracle.

Tolerance rules (from the method's arithmetic: FP32 on the device, FP64 in the oracle):
* picks (angle indices), best restart indices, bump flags and scores are compared
  exactly, except where the oracle marks a decision fragile -- a pick or a bump flag
  that a 1e-4 A move of any atom could flip (an atom within 1e-4 A of a face between
  cells of different value, or a pair within 1e-4 A of bump_dist).  The oracle flags
  every fragile step of its trajectory.  A restart is followed step by step: a step
  where the device made the oracle's pick keeps the two on one trajectory (the poses
  then differ by FP32 rounding only, ~1e-6 A, far below 1e-4 A), so the next step must
  match again; at a fragile step the device may legitimately pick otherwise, and from
  there on the trajectories part (counted as diverged) and nothing later compares.  A
  differing pick at a step the oracle does not flag fails the test.
* the final score of a restart that never parted from the oracle must lie inside the
  oracle's [lo, hi] interval (exact equality unless an atom sits within 1e-4 A of a
  cell face);
* coordinates of such restarts agree within 1e-4 A.
Every comparison helper counts the steps it compared against the steps in all, so a
test can require that fragility left only a small share of the search uncompared.
"""
import numpy as np

COORD_TOL = 1e-4  # A


class Stats(dict):
    def add(self, k, v=1):
        self[k] = self.get(k, 0) + v

    def compared_fraction(self):
        return self.get("picks_compared", 0) / max(1, self.get("steps_total", 0))


def follow(gp, op, sf, fs, g_rig=None, o_rig=None, where=""):
    """Walk one restart's steps: device picks gp against oracle picks op with the oracle's
    per-step fragility sf (bit 1: the pick; bit 2 of step 0: the rigid choice) and its
    first fragile step fs.  Returns (steps compared, index of the step where the two
    parted or -1).  A differing pick or rigid choice the oracle does not flag raises."""
    S = len(op)
    if g_rig is not None and o_rig is not None:
        rigid_fragile = fs == 0 and (S == 0 or (int(sf[0]) & 2))
        if g_rig != o_rig:
            assert rigid_fragile, f"{where}: rigid choice {g_rig} vs oracle {o_rig}"
            return 0, 0
    for s in range(S):
        if int(gp[s]) == int(op[s]):
            continue
        assert int(sf[s]) & 1, f"{where}: step {s} pick {int(gp[s])} vs oracle {int(op[s])} (not fragile)"
        return s, s
    return S, -1


def compare_debug(gpu, orc, batch, params, bumps=True, coord_tol=COORD_TOL, min_compared=None):
    """Full comparison (GPU run with debug=True[, bumps=True] vs oracle.dock_batch(debug=True)).
    min_compared: the least share of all steps that must be compared (fragility and
    legitimate divergence excluded only up to that)."""
    st = Stats()
    L = batch.n_ligands
    O, reps, A = params.n_orient, params.repetitions, params.n_angles
    rot_off = np.asarray(batch.rot_off, np.int64)
    for i in range(L):
        R = int(rot_off[i + 1] - rot_off[i])
        S = reps * R
        base = int(rot_off[i]) * reps * O
        same = np.zeros(O, bool)
        for o in range(O):
            gp = gpu["orient_pick"][base + o * S: base + (o + 1) * S]
            op = orc["orient_pick"][base + o * S: base + (o + 1) * S]
            sf = orc["orient_step_fragile"][base + o * S: base + (o + 1) * S]
            fs = int(orc["orient_fragile"][i, o])
            rig = ("orient_rigid" in gpu and "orient_rigid" in orc)
            upto, parted = follow(gp, op, sf, fs, int(gpu["orient_rigid"][i, o]) if rig else None,
                                  int(orc["orient_rigid"][i, o]) if rig else None, f"ligand {i} restart {o}")
            st.add("restarts")
            st.add("steps_total", S)
            st.add("picks_compared", upto)
            st.add("fragile_steps", int((sf[:upto + (parted >= 0)] & 1).sum()))
            if rig:
                st.add("rigid_compared")
            if fs >= 0:
                st.add("fragile_restarts")
            if parted >= 0:
                st.add("diverged_restarts")
            same[o] = parted < 0
            gs = int(gpu["orient_score"][i, o])
            if same[o]:
                lo, hi = int(orc["orient_score_lo"][i, o]), int(orc["orient_score_hi"][i, o])
                assert lo <= gs <= hi, f"score ligand {i} restart {o}: gpu {gs} oracle [{lo},{hi}]"
                st.add("scores_exact" if gs == int(orc["orient_score"][i, o]) else "scores_in_interval")
            if bumps:
                last = S if parted < 0 else parted + 1  # the parting step starts from one pose
                cb = base * A + o * S * A
                ob = orc["bump"][cb: cb + last * A]
                gb = gpu["bump_bits"][cb: cb + last * A]
                sure = ob != 2
                np.testing.assert_array_equal(gb[sure], ob[sure], err_msg=f"bumps ligand {i} restart {o}")
                st.add("bumps_compared", int(sure.sum()))
                st.add("bumps_uncertain", int((~sure).sum()))
        check_ligand(gpu, orc, batch, params, i, st, coord_tol, same=same)
    if min_compared is not None:
        assert st.compared_fraction() >= min_compared, (st.compared_fraction(), dict(st))
    return st


def check_ligand(gpu, orc, batch, params, i, st, coord_tol=COORD_TOL, same=None):
    """Best restart / score / picks / coordinates of ligand i.  same[o]: restart o never
    parted from the oracle's trajectory (default: the oracle flags no fragile step)."""
    O, reps = params.n_orient, params.repetitions
    rot_off = np.asarray(batch.rot_off, np.int64)
    R = int(rot_off[i + 1] - rot_off[i])
    S = reps * R
    if same is None:
        same = orc["orient_fragile"][i] < 0
    gb, ob = int(gpu["best_orient"][i]), int(orc["best_orient"][i])
    gs = int(gpu["best_score"][i])
    assert int(gpu["evals"][i]) == int(orc["evals"][i])
    if R:
        assert 0 <= int(gpu["pair_tests"][i]) <= int(orc["pair_tests_full"][i])
        assert int(gpu["atom_moves"][i]) > 0
    if "orient_rigid" in gpu:
        assert int(gpu["best_rigid"][i]) == int(gpu["orient_rigid"][i, gb])
    if "orient_score" in gpu:  # self-consistency of the reduction over restarts
        row = gpu["orient_score"][i].astype(np.int64)
        assert gs == row.max() and gb == int(np.argmax(row)), f"ligand {i}: best restart not the first max"
        np.testing.assert_array_equal(
            gpu["best_angle"][rot_off[i] * reps: rot_off[i] * reps + S],
            gpu["orient_pick"][rot_off[i] * reps * O + gb * S: rot_off[i] * reps * O + (gb + 1) * S])
    # the best restart is decided when every restart stayed on the oracle's trajectory and
    # no other restart's score interval reaches the best one's (ties: smaller o)
    lo, hi = orc["orient_score_lo"][i].astype(np.int64), orc["orient_score_hi"][i].astype(np.int64)
    o_ids = np.arange(O)
    apart = np.where(o_ids < ob, hi < lo[ob], hi <= lo[ob])
    apart[ob] = True
    if bool(np.all(same)) and bool(np.all(apart)):
        st.add("ligands_robust")
        assert gb == ob, f"ligand {i}: best restart {gb} vs oracle {ob}"
        assert lo[ob] <= gs <= hi[ob], f"ligand {i}: best score {gs} vs oracle [{lo[ob]},{hi[ob]}]"
    else:
        st.add("ligands_fragile")
    if gb == ob and bool(same[ob]):
        a0, a1 = int(batch.atom_off[i]), int(batch.atom_off[i + 1])
        d = np.abs(gpu["best_xyz"][a0:a1].astype(np.float64) - orc["best_xyz"][a0:a1]).max()
        assert d <= coord_tol, f"ligand {i}: coordinates differ by {d:.3g} A"
        st["max_coord_err"] = max(st.get("max_coord_err", 0.0), float(d))
        np.testing.assert_array_equal(
            gpu["best_angle"][rot_off[i] * reps: rot_off[i] * reps + S],
            orc["orient_pick"][rot_off[i] * reps * O + ob * S: rot_off[i] * reps * O + (ob + 1) * S])
        st.add("coords_compared")


def check_pose_vs_oracle(gpu, batch, params, pocket, i, o, st, oracle_mod, coord_tol=COORD_TOL):
    """One (ligand, restart) of a GPU debug run against oracle.dock_pose: its picks along
    the oracle's trajectory (see follow), and its final score when the two never parted.
    Returns (oracle result, True if the restart stayed on the oracle's trajectory)."""
    O, reps = params.n_orient, params.repetitions
    rot_off = np.asarray(batch.rot_off, np.int64)
    R = int(rot_off[i + 1] - rot_off[i])
    S = reps * R
    ref = oracle_mod.dock_pose(batch.ligand(i), pocket, params, o)
    base = int(rot_off[i]) * reps * O
    gp = gpu["orient_pick"][base + o * S: base + (o + 1) * S]
    g_rig = int(gpu["orient_rigid"][i, o]) if "orient_rigid" in gpu else None
    upto, parted = follow(gp, ref["picks"], ref["step_fragile"], ref["fragile"], g_rig,
                          ref["rigid"] if g_rig is not None else None, f"ligand {i} restart {o}")
    st.add("sampled_restarts")
    st.add("steps_total", S)
    st.add("picks_compared", upto)
    st.add("fragile_steps", int((ref["step_fragile"][:upto + (parted >= 0)] & 1).sum()))
    if parted < 0:
        gs = int(gpu["orient_score"][i, o])
        assert ref["score_lo"] <= gs <= ref["score_hi"], (i, o, gs, ref["score_lo"], ref["score_hi"])
        st.add("sampled_exact" if gs == ref["score"] else "sampled_in_interval")
    else:
        st.add("sampled_diverged")
    return ref, parted < 0
