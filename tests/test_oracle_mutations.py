"""The oracle's pins catch plausible mistakes: each mutant of the C++ oracle (one
plausible slip in one place, planted in a copy compiled on the CPU) must fail the pins
that cover that place.  This checks the pins, not the oracle: the real oracle passes
them (tests/test_oracle_pins.py).
"""
import os
import subprocess
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

import oracle
import test_features_oracle as feats
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "geodock_oracle.cpp")

# name: (text in the oracle, its mutant, the pins that must catch it)
MUTANTS = {
    "left-handed rotation": (
        "return c * v + s * cross(u, v)", "return c * v - s * cross(u, v)",
        [pins.test_rodrigues_right_handed_closed_form, pins.test_torsion_invariants]),
    "cell by rounding": (
        "double f = std::floor(u[d]);", "double f = std::round(u[d]);",
        [pins.test_score_on_modular_grid]),
    "non-strict bump": (
        "return d < bump_dist;", "return d <= bump_dist;",
        [pins.test_bump_threshold_and_exclusions]),
    "1-4 pairs excluded": (
        ">= min_sep) r.pairs.push_back", "> min_sep) r.pairs.push_back",
        [pins.test_bump_threshold_and_exclusions]),
    "fragment tie to the side with atom 0": (
        "else frag_is_v = side_u[0] != 0;", "else frag_is_v = side_u[0] == 0;",
        [pins.test_fragment_tie_moves_side_without_atom0]),
    "larger fragment moved": (
        "if (nv != nu) frag_is_v = nv < nu;", "if (nv != nu) frag_is_v = nv > nu;",
        [pins.test_fragment_matches_networkx]),
    "angle ties to the largest k": (
        "score[k] > score[kstar]", "score[k] >= score[kstar]",
        [pins.test_ties_go_to_the_first_angle_and_restart]),
    "Euler beta at bin edges": (
        "double beta = pi * (j + 0.5) / nb;", "double beta = pi * j / nb;",
        [pins.test_euler_grid_matches_scipy_zyz]),
    "pocket centre off by half a box": (
        "return origin + (0.5 * h)", "return origin + (1.0 * h)",
        [pins.test_placement_centroid_and_rigidity]),
    "early exit charged per pair": (
        "(first / 32 + 1) * 32", "(first + 1)",
        [pins.test_early_exit_pair_count_matches_replay]),
    "restart ties to the last": (
        "out.orient_score[o] > out.orient_score[best]", "out.orient_score[o] >= out.orient_score[best]",
        [pins.test_ties_go_to_the_first_angle_and_restart]),
    "commit one angle off": (
        "double theta = 2.0 * pi * kstar / A;", "double theta = 2.0 * pi * (kstar + 1) / A;",
        [lambda: pins.test_sequential_search_equals_exhaustive_replay(16)]),
    "static atoms left out of the score": (
        "if (!rot.moving[a]) static_score += cell_value(P, x[a]);", "",
        [pins.test_score_never_decreases_and_k0_feasible]),
    "rigid sweep ties to the last": (
        "if (sc[m] > sc[best]) best = m;", "if (sc[m] >= sc[best]) best = m;",
        [pins.test_rigid_sweep_picks_the_best_rigid_candidate, pins.test_ties_go_to_the_first_angle_and_restart]),
    "Euler angles in the wrong order": (
        "return matmul(matmul(rot_z(alpha), rot_y(beta)), rot_z(gamma));",
        "return matmul(matmul(rot_z(gamma), rot_y(beta)), rot_z(alpha));",
        [pins.test_euler_grid_matches_scipy_zyz]),
    "grid strides swapped": (  # stays inside the 7 x 5 x 4 test grid
        "return P.grid[(idx[2] * P.ny + idx[1]) * P.nx + idx[0]];",
        "return P.grid[(idx[2] * P.nx + idx[1]) * P.ny + idx[0]];",
        [pins.test_score_on_modular_grid]),
    "last cell treated as outside": (
        "if (!(f >= 0.0 && f < n[d])) return 0;", "if (!(f >= 0.0 && f < n[d] - 1)) return 0;",
        [pins.test_score_on_modular_grid]),
    "histogram bins of 1 A": (
        "const int b = (int)std::floor(d / 0.75);", "const int b = (int)std::floor(d / 1.0);",
        [feats.test_size_gyration_histogram_on_hand_placed_atoms]),
    "quaternion sign not fixed": (
        "if (q[0] < 0)", "if (q[0] > 0)",
        [feats.test_quaternion_matches_scipy]),
    "farthest-point sampling keeps the largest distance": (
        "mind[a] = s == 0 ? d : std::min(mind[a], d);", "mind[a] = s == 0 ? d : std::max(mind[a], d);",
        [feats.test_farthest_point_order_on_a_line]),
    "grid samples scaled by 1/256": (
        "feat[23 + sidx] = cell_value(P, y) / 255.0;", "feat[23 + sidx] = cell_value(P, y) / 256.0;",
        [feats.test_grid_samples_read_the_placed_pose]),
    "quaternion from full angles": (
        "const double qa[4] = {std::cos(al / 2), 0, 0, std::sin(al / 2)};",
        "const double qa[4] = {std::cos(al), 0, 0, std::sin(al)};",
        [feats.test_quaternion_matches_scipy]),
    "size feature over 256 atoms": (
        "feat[4] = n / 250.0;", "feat[4] = n / 256.0;",
        [feats.test_size_gyration_histogram_on_hand_placed_atoms]),
    "gyration without the square root": (
        "feat[6] = std::sqrt(r2 / n) / 10.0;", "feat[6] = (r2 / n) / 10.0;",
        [feats.test_size_gyration_histogram_on_hand_placed_atoms]),
}


@pytest.fixture(scope="module")
def mutant_libs():
    src = open(SRC).read()
    tmp = tempfile.mkdtemp(prefix="orc_mut_")
    jobs = {}
    for i, (name, (old, new, _)) in enumerate(MUTANTS.items()):
        assert src.count(old) == 1, f"{name}: the mutated text must occur exactly once"
        path = os.path.join(tmp, f"m{i}.cpp")
        with open(path, "w") as f:
            f.write(src.replace(old, new))
        jobs[name] = path

    def compile_one(path):
        so = path[:-4] + ".so"
        subprocess.check_call(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
                               "-o", so, path])
        return so

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        libs = dict(zip(jobs, ex.map(compile_one, jobs.values())))
    yield libs


@pytest.mark.parametrize("name", list(MUTANTS))
def test_pins_catch_the_mutant(name, mutant_libs, monkeypatch):
    monkeypatch.setattr(oracle, "build", lambda force=False: mutant_libs[name])
    monkeypatch.setattr(oracle, "_lib", None)
    caught = []
    for pin in MUTANTS[name][2]:
        try:
            pin()
        except Exception:  # an assertion, or an error the mutant provokes
            caught.append(getattr(pin, "__name__", "pin"))
    oracle._lib = None
    assert caught, f"no pin caught the mutant '{name}'"
