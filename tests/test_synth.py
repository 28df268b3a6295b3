"""Properties of the seeded input generators (ligand trees, pocket grids)."""
import math

import networkx as nx
import numpy as np

from paper_1901_06229_b300 import synth


def _check_ligand(lig, n, r):
    x = lig.xyz.astype(np.float64)
    assert lig.xyz.dtype == np.float32 and x.shape == (n, 3)
    assert lig.bonds.shape == (n - 1, 2)
    G = nx.Graph()
    G.add_nodes_from(range(n))
    G.add_edges_from(map(tuple, lig.bonds.tolist()))
    assert nx.is_tree(G)
    assert max(dict(G.degree).values()) <= synth.MAX_VALENCE
    bl = np.linalg.norm(x[lig.bonds[:, 0]] - x[lig.bonds[:, 1]], axis=1)
    np.testing.assert_allclose(bl, 1.5, atol=2e-6)
    # every atom after the first two sits at 109.5 deg to its parent's first neighbour
    nbrs = {a: [] for a in range(n)}
    for u, v in lig.bonds.tolist():
        nbrs[u].append(v)
        nbrs[v].append(u)
    for par, child in lig.bonds[1:].tolist():
        first = nbrs[par][0]
        a = x[first] - x[par]
        b = x[child] - x[par]
        ang = math.degrees(math.acos(np.dot(a, b) / np.linalg.norm(a) / np.linalg.norm(b)))
        assert abs(ang - 109.5) < 1e-3
    # no two non-bonded atoms closer than 2.2 A
    d = np.linalg.norm(x[:, None] - x[None, :], axis=-1)
    bonded = np.zeros((n, n), bool)
    bonded[lig.bonds[:, 0], lig.bonds[:, 1]] = bonded[lig.bonds[:, 1], lig.bonds[:, 0]] = True
    np.fill_diagonal(bonded, True)
    assert d[~bonded].min() >= 2.2 - 1e-5
    # rotamers: distinct, non-terminal edges
    assert len(lig.rot_bond) == r and len(set(lig.rot_bond.tolist())) == r
    deg = dict(G.degree)
    for rb in lig.rot_bond:
        u, v = lig.bonds[rb]
        assert deg[u] >= 2 and deg[v] >= 2


def test_single_ligand_shape():
    w = synth.workload_single()
    assert w.batch.n_ligands == 1
    _check_ligand(w.batch.ligand(0), 24, 4)
    assert w.pocket.grid.shape == (32, 32, 32) and w.pocket.spacing == 0.5
    assert w.params.n_orient == 64 and w.params.n_angles == 32


def test_batched_ligand_sizes():
    w = synth.workload_batched(40)
    for i in range(40):
        lig = w.batch.ligand(i)
        n, r = len(lig.xyz), len(lig.rot_bond)
        assert 20 <= n <= 80 and 2 <= r <= 12 and r <= n // 5
        _check_ligand(lig, n, r)
    assert w.pocket.grid.shape == (64, 64, 64) and w.params.n_orient == 256 and w.params.n_angles == 64


def test_large_ligand_sizes():
    w = synth.workload_large(2)
    for i in range(2):
        lig = w.batch.ligand(i)
        n, r = len(lig.xyz), len(lig.rot_bond)
        assert 100 <= n <= 250 and 20 <= r <= 60
        _check_ligand(lig, n, r)
    assert w.pocket.grid.shape == (128, 128, 128)


def test_ligands_are_reproducible_and_independent():
    a = synth.workload_batched(5)
    b = synth.workload_batched(3, start=2)
    for i in range(3):
        np.testing.assert_array_equal(a.batch.ligand(i + 2).xyz, b.batch.ligand(i).xyz)
        np.testing.assert_array_equal(a.batch.ligand(i + 2).rot_bond, b.batch.ligand(i).rot_bond)


def test_pocket_values_at_hand_computed_points():
    sph = np.array([[1.0, 2.0, 3.0, 4.0]])
    c = np.array([1.0, 2.0, 3.0])
    u = np.array([0.6, 0.0, 0.8])
    pts = np.array([c, c + 3.9 * u, c + 4.5 * u, c + 5.0 * u, c + 5.5 * u, c + 6.0 * u, c + 9 * u])
    # inside: 255; 0.5 A out: 255*0.75 = 191.25 -> 191; 1 A out: 127.5 -> 128 (half up);
    # 1.5 A out: 63.75 -> 64; 2 A and beyond: 0
    assert synth.pocket_values(sph, pts).tolist() == [255, 255, 191, 128, 64, 0, 0]
    two = np.array([[0.0, 0.0, 0.0, 3.0], [10.0, 0.0, 0.0, 3.0]])
    assert synth.pocket_values(two, np.array([[4.0, 0, 0], [6.0, 0, 0], [5.0, 0, 0]])).tolist() == [128, 128, 0]


def test_generated_pocket_layout():
    p = synth.workload_single().pocket
    nz, ny, nx_ = p.grid.shape
    # cell (i, j, k) holds the value at its centre; grid is indexed [k, j, i]
    for (i, j, k) in [(3, 17, 29), (16, 16, 16), (0, 31, 5)]:
        centre = p.origin.astype(np.float64) + (np.array([i, j, k]) + 0.5) * p.spacing
        assert p.grid[k, j, i] == synth.pocket_values(p.spheres, centre[None])[0]
    # the box is centred on the pocket centre and contains the sphere union
    assert p.grid.max() == 255 and p.grid[0, 0, 0] == 0


def test_splitmix64_reference_values():
    # first outputs for seed 0 of the published SplitMix64 generator
    g = synth.SplitMix64(0)
    assert [g.next_u64() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
