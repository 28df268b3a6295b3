"""Element-by-element comparison of the CUDA library's results with the FP64 oracle.

Tolerance rules (from the method's arithmetic: FP32 on the device, FP64 in the oracle):
* picks (angle indices), best restart indices, bump flags and scores are compared
  exactly, except where the oracle marks a decision fragile -- a pick or a bump flag
  that a 1e-4 A move of any atom could flip (an atom within 1e-4 A of a face between
  cells of different value, or a pair within 1e-4 A of bump_dist).  After the first
  fragile step of a restart the two trajectories may legitimately differ, so only the
  steps before it are compared; every such case is counted.
* a score that an atom within 1e-4 A of a cell face could change must lie inside the
  oracle's [lo, hi] interval (exact equality otherwise);
* coordinates of non-fragile restarts agree within 1e-4 A.
"""
import numpy as np

COORD_TOL = 1e-4  # A


class Stats(dict):
    def add(self, k, v=1):
        self[k] = self.get(k, 0) + v


def compare_debug(gpu, orc, batch, params, bumps=True, coord_tol=COORD_TOL):
    """Full comparison (GPU run with debug=True[, bumps=True] vs oracle.dock_batch(debug=True))."""
    st = Stats()
    L = batch.n_ligands
    O, reps, A = params.n_orient, params.repetitions, params.n_angles
    rot_off = np.asarray(batch.rot_off, np.int64)
    for i in range(L):
        R = int(rot_off[i + 1] - rot_off[i])
        S = reps * R
        base = int(rot_off[i]) * reps * O
        for o in range(O):
            gp = gpu["orient_pick"][base + o * S: base + (o + 1) * S]
            op = orc["orient_pick"][base + o * S: base + (o + 1) * S]
            fs = int(orc["orient_fragile"][i, o])
            upto = S if fs < 0 else fs
            st.add("restarts")
            if fs >= 0:
                st.add("fragile_restarts")
            np.testing.assert_array_equal(gp[:upto], op[:upto], err_msg=f"picks ligand {i} restart {o}")
            st.add("picks_compared", upto)
            if "orient_rigid" in gpu and "orient_rigid" in orc and fs != 0:
                assert int(gpu["orient_rigid"][i, o]) == int(orc["orient_rigid"][i, o]), (i, o)
                st.add("rigid_compared")
            gs = int(gpu["orient_score"][i, o])
            if fs < 0:
                lo, hi = int(orc["orient_score_lo"][i, o]), int(orc["orient_score_hi"][i, o])
                assert lo <= gs <= hi, f"score ligand {i} restart {o}: gpu {gs} oracle [{lo},{hi}]"
                st.add("scores_exact" if gs == int(orc["orient_score"][i, o]) else "scores_in_interval")
            if bumps:
                last = S if fs < 0 else fs + 1  # the fragile step starts from an identical pose
                cb = base * A + o * S * A
                ob = orc["bump"][cb: cb + last * A]
                gb = gpu["bump_bits"][cb: cb + last * A]
                sure = ob != 2
                np.testing.assert_array_equal(gb[sure], ob[sure], err_msg=f"bumps ligand {i} restart {o}")
                st.add("bumps_compared", int(sure.sum()))
                st.add("bumps_uncertain", int((~sure).sum()))
        check_ligand(gpu, orc, batch, params, i, st, coord_tol)
    return st


def check_ligand(gpu, orc, batch, params, i, st, coord_tol=COORD_TOL):
    """Best restart / score / picks / coordinates of ligand i."""
    O, reps = params.n_orient, params.repetitions
    rot_off = np.asarray(batch.rot_off, np.int64)
    R = int(rot_off[i + 1] - rot_off[i])
    S = reps * R
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
    if orc["best_robust"][i]:
        st.add("ligands_robust")
        assert gb == ob, f"ligand {i}: best restart {gb} vs oracle {ob}"
        lo, hi = int(orc["orient_score_lo"][i, ob]), int(orc["orient_score_hi"][i, ob])
        assert lo <= gs <= hi, f"ligand {i}: best score {gs} vs oracle [{lo},{hi}]"
    else:
        st.add("ligands_fragile")
    if gb == ob and int(orc["orient_fragile"][i, ob]) < 0:
        a0, a1 = int(batch.atom_off[i]), int(batch.atom_off[i + 1])
        d = np.abs(gpu["best_xyz"][a0:a1].astype(np.float64) - orc["best_xyz"][a0:a1]).max()
        assert d <= coord_tol, f"ligand {i}: coordinates differ by {d:.3g} A"
        st["max_coord_err"] = max(st.get("max_coord_err", 0.0), float(d))
        np.testing.assert_array_equal(
            gpu["best_angle"][rot_off[i] * reps: rot_off[i] * reps + S],
            orc["orient_pick"][rot_off[i] * reps * O + ob * S: rot_off[i] * reps * O + (ob + 1) * S])
        st.add("coords_compared")


def check_pose_vs_oracle(gpu, batch, params, pocket, i, o, st, oracle_mod, coord_tol=COORD_TOL):
    """One (ligand, restart) of a GPU debug run against oracle.dock_pose."""
    O, reps = params.n_orient, params.repetitions
    rot_off = np.asarray(batch.rot_off, np.int64)
    R = int(rot_off[i + 1] - rot_off[i])
    S = reps * R
    ref = oracle_mod.dock_pose(batch.ligand(i), pocket, params, o)
    base = int(rot_off[i]) * reps * O
    gp = gpu["orient_pick"][base + o * S: base + (o + 1) * S]
    upto = S if ref["fragile"] < 0 else ref["fragile"]
    np.testing.assert_array_equal(gp[:upto], ref["picks"][:upto], err_msg=f"ligand {i} restart {o}")
    st.add("sampled_restarts")
    if ref["fragile"] < 0:
        gs = int(gpu["orient_score"][i, o])
        assert ref["score_lo"] <= gs <= ref["score_hi"]
        st.add("sampled_exact" if gs == ref["score"] else "sampled_in_interval")
    else:
        st.add("sampled_fragile")
    return ref
