"""Pins of the oracle's proposer features: scipy quaternions, hand-placed atoms with
known radius of gyration, histogram and farthest-point order, and grid samples read
through the separately pinned placement and scoring functions."""
import math

import numpy as np
from scipy.spatial.transform import Rotation

import oracle
from paper_1901_06229_b300 import synth
from test_oracle_pins import modular_pocket


def test_quaternion_matches_scipy():
    w = synth.workload_single()
    lig = w.batch.ligand(0)
    for na, nb, ng in [(8, 8, 4), (3, 5, 2)]:
        p = synth.SearchParams(na, nb, ng, 32)
        for o in range(na * nb * ng):
            i, j, k = o // (nb * ng), (o // ng) % nb, o % ng
            q = Rotation.from_euler("ZYZ", [2 * math.pi * i / na, math.pi * (j + 0.5) / nb,
                                            2 * math.pi * k / ng]).as_quat()  # x, y, z, w
            q = np.array([q[3], q[0], q[1], q[2]])
            q = -q if q[0] < 0 else q
            f = oracle.features(lig.xyz, 4, o, p, w.pocket)["feat"]
            np.testing.assert_allclose(f[:4], q, atol=1e-12)


def test_size_gyration_histogram_on_hand_placed_atoms():
    # centroid at the origin; distances 0.5, 0.5, 1.0, 2.0, 2.0, 11.9, 12.5 A...
    pts = np.array([[0.5, 0, 0], [-0.5, 0, 0], [0, 1.0, 0], [0, -1.0, 0], [0, 0, 2.0], [0, 0, -2.0],
                    [11.9, 0, 0], [-11.9, 0, 0], [0, 12.5, 0], [0, -12.5, 0]], np.float32)
    p = synth.SearchParams(1, 1, 1, 32)
    f = oracle.features(pts, 3, 0, p, modular_pocket())["feat"]
    assert f[4] == 10 / 250 and f[5] == 3 / 60
    d = np.linalg.norm(pts.astype(np.float64), axis=1)
    assert abs(f[6] - math.sqrt(np.mean(d ** 2)) / 10) < 1e-12
    hist = np.zeros(16)
    hist[0] = 2 / 10   # 0.5 A: bin [0, 0.75)
    hist[1] = 2 / 10   # 1.0 A: bin [0.75, 1.5)
    hist[2] = 2 / 10   # 2.0 A: bin [1.5, 2.25)
    hist[15] = 2 / 10  # 11.9 A: bin [11.25, 12); 12.5 A is beyond the last bin
    np.testing.assert_allclose(f[7:23], hist, atol=1e-15)


def test_farthest_point_order_on_a_line():
    # ten atoms at x = 0..9: centroid 4.5.  Atoms 0 and 9 tie at 4.5 A -> 0 (smaller
    # index); then 9 (9 A); then 4 and 5 tie at 4 A -> 4; then 7 (min(7, 2, 3) = 2 ...)
    pts = np.array([[float(i), 0, 0] for i in range(10)], np.float32)
    p = synth.SearchParams(1, 1, 1, 32)
    r = oracle.features(pts, 1, 0, p, modular_pocket())
    # after {0, 9, 4}: distances to the set: 1:1 2:2 3:1 5:1 6:2 7:2 8:1 -> 2 (tie 2, 6, 7)
    assert r["fps"][:4].tolist() == [0, 9, 4, 2]
    # ten atoms: every atom is chosen once, then the order repeats
    assert sorted(r["fps"][:10].tolist()) == list(range(10))
    np.testing.assert_array_equal(r["fps"][10:20], r["fps"][:10])


def test_grid_samples_read_the_placed_pose():
    w = synth.workload_single()
    lig = w.batch.ligand(0)
    P = modular_pocket(40, 40, 40, 0.5, origin=(-10.0, -10.0, -10.0))
    p = synth.SearchParams(4, 4, 4, 32)
    for o in (0, 9, 63):
        r = oracle.features(lig.xyz, 4, o, p, P)
        placed = oracle.place(lig.xyz, o, p, P)
        for s in range(25):
            want = oracle.score(P, placed[r["fps"][s]][None]) / 255.0
            assert r["feat"][23 + s] == want
