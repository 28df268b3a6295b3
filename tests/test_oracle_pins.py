"""Pins of the FP64 oracle against things other than itself.

Each test checks one part of the oracle against a closed form, a library routine
(scipy's rotations, networkx's graph algorithms), a hand-built grid with a known
sum, or an independent numpy brute force, so that a dropped term, a flipped sign,
a transposed axis or a wrong tie rule anywhere in the oracle fails at least one.
"""
import itertools
import math

import networkx as nx
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_1901_06229_b300 import synth


# ----------------------------------------------------------------------------- helpers

def textured_pocket(n=32, h=0.5, centre=(1.0, -2.0, 0.5)):
    """Smoothly varying test grid: many distinct cell values, so picks are not all ties."""
    centre = np.asarray(centre, dtype=np.float64)
    origin = (centre - n * h / 2).astype(np.float32)
    ax = origin.astype(np.float64)[None, :] + (np.arange(n)[:, None] + 0.5) * h
    z, y, x = np.meshgrid(ax[:, 2], ax[:, 1], ax[:, 0], indexing="ij")
    v = 127.5 + 127.5 * np.sin(0.9 * x) * np.cos(0.7 * y) * np.sin(0.8 * z + 0.3)
    return synth.Pocket(grid=np.floor(v).astype(np.uint8), spacing=h, origin=origin)


def modular_pocket(nx=7, ny=5, nz=4, h=0.75, origin=(1.0, -2.0, 3.5)):
    """grid[k, j, i] = (i + 2j + 3k) mod 256: every axis carries its own weight."""
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    g = ((i + 2 * j + 3 * k) % 256).astype(np.uint8)
    return synth.Pocket(grid=g, spacing=h, origin=np.asarray(origin, dtype=np.float32))


def small_ligands():
    out = []
    for s, (n, r) in enumerate([(16, 3), (24, 3), (20, 2), (12, 1)]):
        rng = synth.SplitMix64(synth.ligand_seed(777, s))
        out.append(synth.gen_ligand(rng, n, r))
    return out


def nx_graph(lig):
    G = nx.Graph()
    G.add_nodes_from(range(len(lig.xyz)))
    G.add_edges_from(map(tuple, lig.bonds.tolist()))
    return G


def nx_fragment(lig, rb):
    """Smaller side of the cut bond (tie: the side without atom 0), via networkx."""
    u, v = lig.bonds[rb]
    G = nx_graph(lig)
    G.remove_edge(u, v)
    su = nx.node_connected_component(G, u)
    sv = nx.node_connected_component(G, v)
    if len(sv) != len(su):
        frag = sv if len(sv) < len(su) else su
    else:
        frag = su if 0 in sv else sv
    q = v if v in frag else u
    p = u if q == v else v
    mask = np.zeros(len(lig.xyz), dtype=bool)
    mask[list(frag)] = True
    return mask, p, q


# ----------------------------------------------------------------------------- rotations

def test_euler_grid_matches_scipy_zyz():
    for na, nb, ng in [(4, 4, 4), (8, 8, 4), (3, 5, 2)]:
        for i, j, k in itertools.product(range(na), range(nb), range(ng)):
            o = (i * nb + j) * ng + k
            a, b, g = 2 * math.pi * i / na, math.pi * (j + 0.5) / nb, 2 * math.pi * k / ng
            ref = Rotation.from_euler("ZYZ", [a, b, g]).as_matrix()
            R = oracle.euler(o, na, nb, ng)
            np.testing.assert_allclose(R, ref, atol=1e-14)


def test_euler_grid_is_proper_and_distinct():
    na, nb, ng = 8, 8, 4
    mats = [oracle.euler(o, na, nb, ng) for o in range(na * nb * ng)]
    for R in mats:
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1.0) < 1e-14
    # closed form of the rotated z axis for ZYZ: (cos a sin b, sin a sin b, cos b)
    for o, R in enumerate(mats):
        i, j = o // (nb * ng), (o // ng) % nb
        a, b = 2 * math.pi * i / na, math.pi * (j + 0.5) / nb
        np.testing.assert_allclose(R[:, 2], [math.cos(a) * math.sin(b), math.sin(a) * math.sin(b), math.cos(b)],
                                   atol=1e-14)
    flat = np.array([m.ravel() for m in mats])
    d = np.linalg.norm(flat[:, None, :] - flat[None, :, :], axis=-1)
    assert np.all(d[~np.eye(len(mats), dtype=bool)] > 1e-3), "two restarts coincide"


def test_rodrigues_right_handed_closed_form():
    np.testing.assert_allclose(oracle.rodrigues([0, 0, 1], math.pi / 2, [1, 0, 0]), [0, 1, 0], atol=1e-15)
    np.testing.assert_allclose(oracle.rodrigues([1, 0, 0], math.pi / 2, [0, 1, 0]), [0, 0, 1], atol=1e-15)
    np.testing.assert_allclose(oracle.rodrigues([0, 1, 0], math.pi / 2, [0, 0, 1]), [1, 0, 0], atol=1e-15)
    rng = np.random.default_rng(5)
    for _ in range(50):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        th = rng.uniform(-7, 7)
        v = rng.normal(size=3) * 4
        ref = Rotation.from_rotvec(u * th).apply(v)
        np.testing.assert_allclose(oracle.rodrigues(u, th, v), ref, atol=1e-12)


# ----------------------------------------------------------------------------- topology

def test_fragment_matches_networkx():
    ligs = small_ligands() + [synth.workload_batched(6).batch.ligand(i) for i in range(6)]
    for lig in ligs:
        n = len(lig.xyz)
        G = nx_graph(lig)
        spl = dict(nx.all_pairs_shortest_path_length(G))
        ref_dist = np.array([[spl[a][b] for b in range(n)] for a in range(n)])
        for rb in lig.rot_bond:
            mv, p, q, dist = oracle.fragment(n, lig.bonds, int(rb))
            m_ref, p_ref, q_ref = nx_fragment(lig, int(rb))
            np.testing.assert_array_equal(mv, m_ref)
            assert (p, q) == (p_ref, q_ref)
            np.testing.assert_array_equal(dist, ref_dist)
            assert mv.sum() <= n - mv.sum()


def test_fragment_tie_moves_side_without_atom0():
    chain = np.array([[0, 1], [1, 2], [2, 3], [3, 4], [4, 5]], dtype=np.int32)
    mv, p, q, _ = oracle.fragment(6, chain, 2)  # bond 2-3 splits 3 | 3
    assert mv.tolist() == [False, False, False, True, True, True] and (p, q) == (2, 3)
    # same chain numbered from the other end: atom 0 now sits on the far side
    rev = np.array([[5, 4], [4, 3], [3, 2], [2, 1], [1, 0]], dtype=np.int32)
    mv, p, q, _ = oracle.fragment(6, rev, 2)  # bond 3-2
    assert mv.tolist() == [False, False, False, True, True, True] and (p, q) == (2, 3)


def test_rejects_non_tree_and_terminal_rotamer():
    with pytest.raises(ValueError):
        oracle.fragment(4, np.array([[0, 1], [1, 2], [2, 0]], np.int32), 0)  # cycle, 3 bonds / 4 atoms
    with pytest.raises(ValueError):
        oracle.fragment(4, np.array([[0, 1], [1, 2], [2, 3]], np.int32), 0)  # terminal bond


# ----------------------------------------------------------------------------- torsion

def test_torsion_invariants():
    for lig in small_ligands() + [synth.workload_large(1).batch.ligand(0)]:
        x0 = lig.xyz.astype(np.float64)
        n = len(x0)
        for rb in lig.rot_bond[:6]:
            mv, p, q, _ = oracle.fragment(n, lig.bonds, int(rb))
            for k, A in [(1, 32), (7, 32), (31, 64), (5, 128)]:
                x = oracle.torsion(x0, lig.bonds, int(rb), k, A)
                # static side and both axis atoms untouched (bitwise for the static side)
                assert np.array_equal(x[~mv], x0[~mv])
                np.testing.assert_allclose(x[q], x0[q], atol=1e-12)
                # bond lengths and all distances inside the fragment unchanged
                bl0 = np.linalg.norm(x0[lig.bonds[:, 0]] - x0[lig.bonds[:, 1]], axis=1)
                bl = np.linalg.norm(x[lig.bonds[:, 0]] - x[lig.bonds[:, 1]], axis=1)
                np.testing.assert_allclose(bl, bl0, atol=1e-12)
                f = np.where(mv)[0]
                d0 = np.linalg.norm(x0[f, None] - x0[None, f], axis=-1)
                d1 = np.linalg.norm(x[f, None] - x[None, f], axis=-1)
                np.testing.assert_allclose(d1, d0, atol=1e-12)
                # the signed angle about the axis is 2 pi k / A, right-handed
                u = (x0[q] - x0[p]) / np.linalg.norm(x0[q] - x0[p])
                far = f[np.argmax(np.linalg.norm(np.cross(x0[f] - x0[p], u), axis=1))]
                a0 = x0[far] - x0[p] - np.dot(x0[far] - x0[p], u) * u
                a1 = x[far] - x[p] - np.dot(x[far] - x[p], u) * u
                ang = math.atan2(np.dot(np.cross(a0, a1), u), np.dot(a0, a1))
                want = math.remainder(2 * math.pi * k / A, 2 * math.pi)
                assert abs(math.remainder(ang - want, 2 * math.pi)) < 1e-9
            # A steps of 2 pi / A return to the start; k = 0 is the identity
            x = x0.copy()
            for _ in range(32):
                x = oracle.torsion(x, lig.bonds, int(rb), 1, 32)
            np.testing.assert_allclose(x, x0, atol=1e-9)
            np.testing.assert_allclose(oracle.torsion(x0, lig.bonds, int(rb), 0, 32), x0, atol=1e-13)


# ----------------------------------------------------------------------------- score

def test_score_on_modular_grid():
    P = modular_pocket()
    h = P.spacing
    org = P.origin.astype(np.float64)
    cells = [(0, 0, 0), (6, 4, 3), (3, 1, 2), (1, 4, 0), (5, 0, 3)]
    pts = np.array([org + (np.array(c) + 0.5) * h for c in cells])
    want = sum((i + 2 * j + 3 * k) % 256 for i, j, k in cells)
    assert oracle.score(P, pts) == want
    for c in cells:  # one atom at a time, and jittered inside its cell
        p = org + (np.array(c) + 0.5) * h
        assert oracle.score(P, p[None]) == (c[0] + 2 * c[1] + 3 * c[2]) % 256
        assert oracle.score(P, (p + 0.49 * h)[None]) == (c[0] + 2 * c[1] + 3 * c[2]) % 256
        assert oracle.score(P, (p - 0.49 * h)[None]) == (c[0] + 2 * c[1] + 3 * c[2]) % 256
    # a point on a lower cell face belongs to that cell (floor)
    assert oracle.score(P, (org + np.array([0.0, h, 0.0]))[None]) == 2
    assert oracle.score(P, (org + np.array([2 * h, 0.0, h]))[None]) == 2 + 3
    # outside the box (below the origin or at/after the far face) scores 0
    for off in ([-1e-9, 0.5, 0.5], [0.5, -1e-9, 0.5], [0.5, 0.5, -1e-9],
                [7 * h, 0.5, 0.5], [0.5, 5 * h, 0.5], [0.5, 0.5, 4 * h], [-30, 40, 2]):
        assert oracle.score(P, (org + np.array(off))[None]) == 0


def test_score_on_generated_pocket_matches_sphere_values():
    P = synth.workload_single().pocket
    g = P.grid
    nz, ny, nx_ = g.shape
    rng = np.random.default_rng(3)
    cells = rng.integers(0, [nx_, ny, nz], size=(200, 3))
    pts = P.origin.astype(np.float64) + (cells + rng.uniform(0.01, 0.99, size=(200, 3))) * P.spacing
    for c, p in zip(cells, pts):
        assert oracle.score(P, p[None]) == g[c[2], c[1], c[0]]


# ----------------------------------------------------------------------------- bump

def test_bump_threshold_and_exclusions():
    chain = np.array([[0, 1], [1, 2], [2, 3], [3, 4], [4, 5]], dtype=np.int32)
    base = np.array([[10.0 * i, 0.0, 0.0] for i in range(6)])  # all pairs far apart
    rb = 2  # bond 2-3: moving {3,4,5}, static {0,1,2}
    assert not oracle.bumped(base, chain, rb)

    def with_pos(a, near, d):
        x = base.copy()
        x[a] = x[near] + np.array([0.0, d, 0.0])
        return x

    assert oracle.bumped(with_pos(4, 1, 1.99), chain, rb)          # graph distance 3
    assert not oracle.bumped(with_pos(4, 1, 2.01), chain, rb)
    assert not oracle.bumped(with_pos(4, 1, 2.0), chain, rb)       # strict <
    assert oracle.bumped(with_pos(5, 0, 1.5), chain, rb)           # graph distance 5
    assert not oracle.bumped(with_pos(4, 2, 1.0), chain, rb)       # graph distance 2: excluded
    assert not oracle.bumped(with_pos(3, 1, 0.5), chain, rb)       # graph distance 2: excluded
    assert oracle.bumped(with_pos(3, 0, 1.99), chain, rb)          # 1-4 pair counts at min_sep 3
    assert not oracle.bumped(with_pos(3, 0, 1.99), chain, rb, min_sep=4)
    assert not oracle.bumped(with_pos(4, 5, 0.1), chain, rb)       # both moving: never tested
    assert not oracle.bumped(with_pos(0, 1, 0.1), chain, rb)       # both static: never tested
    assert oracle.bumped(with_pos(4, 1, 2.4), chain, rb, bump_dist=2.5)


def test_generated_start_pose_is_bump_free():
    for lig in small_ligands():
        for rb in lig.rot_bond:
            assert not oracle.bumped(lig.xyz.astype(np.float64), lig.bonds, int(rb))


# ----------------------------------------------------------------------------- placement

def test_placement_centroid_and_rigidity():
    w = synth.workload_single()
    lig = w.batch.ligand(0)
    x0 = lig.xyz.astype(np.float64)
    c = x0.mean(axis=0)
    nz, ny, nx_ = w.pocket.grid.shape
    cp = w.pocket.origin.astype(np.float64) + 0.5 * w.pocket.spacing * np.array([nx_, ny, nz])
    for o in range(w.params.n_orient):
        x = oracle.place(lig.xyz, o, w.params, w.pocket)
        np.testing.assert_allclose(x.mean(axis=0), cp, atol=1e-12)
        R = oracle.euler(o, w.params.n_alpha, w.params.n_beta, w.params.n_gamma)
        np.testing.assert_allclose(x - cp, (x0 - c) @ R.T, atol=1e-12)


# ----------------------------------------------------------------------------- search

def brute_force(lig, pocket, params, orients):
    """Independent enumeration of every angle combination (R <= 3), FP64 numpy/scipy.

    Each conformation is rebuilt from the restart pose by applying the rotamer
    rotations in order with scipy; bumps are tested over *all* atom pairs at graph
    distance >= min_sep (not only moving x static); scores are a numpy gather.
    Returns per orientation the greedy picks replayed on the table, the final greedy
    score and the global optimum.
    """
    n = len(lig.xyz)
    R = len(lig.rot_bond)
    A = params.n_angles
    G = nx_graph(lig)
    spl = dict(nx.all_pairs_shortest_path_length(G))
    iu = [(a, b) for a in range(n) for b in range(a + 1, n) if spl[a][b] >= params.min_bond_sep]
    ia = np.array([a for a, _ in iu])
    ib = np.array([b for _, b in iu])
    frags = [nx_fragment(lig, int(rb)) for rb in lig.rot_bond]
    g = pocket.grid
    nz, ny, nx_ = g.shape
    org = pocket.origin.astype(np.float64)
    x0 = lig.xyz.astype(np.float64)
    c = x0.mean(axis=0)
    cp = org + 0.5 * pocket.spacing * np.array([nx_, ny, nz])
    combos = np.array(list(itertools.product(range(A), repeat=R)), dtype=np.int64)
    res = []
    for o in orients:
        i, j, k = o // (params.n_beta * params.n_gamma), (o // params.n_gamma) % params.n_beta, o % params.n_gamma
        Ro = Rotation.from_euler("ZYZ", [2 * math.pi * i / params.n_alpha, math.pi * (j + 0.5) / params.n_beta,
                                         2 * math.pi * k / params.n_gamma])
        start = cp + Ro.apply(x0 - c)
        X = np.broadcast_to(start, (len(combos), n, 3)).copy()
        for r, (mv, p, q) in enumerate(frags):
            u = X[:, q] - X[:, p]
            u /= np.linalg.norm(u, axis=1, keepdims=True)
            rot = Rotation.from_rotvec(u * (2 * math.pi * combos[:, r] / A)[:, None])
            M = rot.as_matrix()
            rel = X[:, mv] - X[:, p][:, None, :]
            X[:, mv] = X[:, p][:, None, :] + np.einsum("cij,caj->cai", M, rel)
        bumped = np.any(np.linalg.norm(X[:, ia] - X[:, ib], axis=-1) < params.bump_dist, axis=1)
        idx = np.floor((X - org) / pocket.spacing).astype(np.int64)
        inb = np.all((idx >= 0) & (idx < np.array([nx_, ny, nz])), axis=-1)
        idc = np.where(inb[..., None], idx, 0)
        vals = np.where(inb, g[idc[..., 2], idc[..., 1], idc[..., 0]], 0).astype(np.int64)
        score = vals.sum(axis=1)
        # greedy replay: step r picks over k_r with earlier picks fixed, later angles 0
        picks = []
        for r in range(R):
            best = -1
            for kk in range(A):
                key = tuple(picks) + (kk,) + (0,) * (R - r - 1)
                ci = int(np.ravel_multi_index(key, (A,) * R))
                if bumped[ci]:
                    continue
                if best < 0 or score[ci] > best_s:
                    best, best_s = kk, score[ci]
            picks.append(best)
        final = int(score[np.ravel_multi_index(tuple(picks), (A,) * R)])
        opt = int(score[~bumped].max())
        res.append((picks, final, opt))
    return res


@pytest.mark.parametrize("A", [16, 32])
def test_sequential_search_equals_exhaustive_replay(A):
    pocket = textured_pocket()
    params = synth.SearchParams(2, 2, 2, A)
    checked = 0
    for lig in small_ligands():
        b = synth.pack([lig])
        out = oracle.dock_batch(b, pocket, params)
        O = params.n_orient
        R = len(lig.rot_bond)
        picks = out["orient_pick"].reshape(O, R)
        bf = brute_force(lig, pocket, params, range(O))
        for o in range(O):
            if out["orient_fragile"][0, o] >= 0:
                continue
            want_picks, want_final, opt = bf[o]
            assert picks[o].tolist() == want_picks, (o, picks[o], want_picks)
            assert out["orient_score"][0, o] == want_final
            assert want_final <= opt
            checked += 1
    assert checked >= 20


def test_score_never_decreases_and_k0_feasible():
    w = synth.workload_single()
    pocket = textured_pocket()
    out = oracle.dock_batch(w.batch, pocket, w.params, debug=True)
    O, R, A = w.params.n_orient, 4, w.params.n_angles
    cs = out["cand_score"].reshape(O, R, A)
    bp = out["bump"].reshape(O, R, A)
    picks = out["orient_pick"].reshape(O, R)
    assert np.all(bp[:, :, 0] == 0), "the identity candidate must be free"
    for o in range(O):
        prev = cs[o, 0, 0]
        for r in range(R):
            assert cs[o, r, 0] == prev                  # k = 0 reproduces the current score
            k = picks[o, r]
            assert cs[o, r, k] == cs[o, r][bp[o, r] != 1].max()
            assert cs[o, r, k] >= cs[o, r, 0]
            prev = cs[o, r, k]
        assert out["orient_score"][0, o] == prev
    assert out["best_score"][0] == out["orient_score"][0].max()
    assert out["best_orient"][0] == int(np.argmax(out["orient_score"][0]))


def test_ties_go_to_the_first_angle_and_restart():
    """On an all-zero pocket every candidate and every restart scores 0: the picks are
    the smallest angle (k = 0, the identity, always free), the best restart is o = 0 and
    the rigid sweep keeps its first candidate (the identity)."""
    pocket = synth.Pocket(grid=np.zeros((16, 16, 16), np.uint8), spacing=0.5,
                          origin=np.array([-4.0, -4.0, -4.0], np.float32))
    params = synth.SearchParams(2, 2, 2, 8)
    for lig in small_ligands()[:2]:
        out = oracle.dock_batch(synth.pack([lig]), pocket, params)
        assert np.all(out["orient_score"] == 0)
        assert np.all(out["orient_pick"] == 0)
        assert out["best_orient"][0] == 0 and out["best_score"][0] == 0
    # the rigid sweep ties too: the identity (candidate 0) is kept
    rigid = synth.SearchParams(2, 2, 2, 8, rigid_span=1, rigid_step=0.1)
    out = oracle.dock_batch(synth.pack(small_ligands()[:1]), pocket, rigid)
    assert np.all(out["orient_rigid"] == 0)


def test_counters():
    w = synth.workload_batched(3)
    out = oracle.dock_batch(w.batch, w.pocket, w.params)
    for i in range(3):
        lig = w.batch.ligand(i)
        n = len(lig.xyz)
        assert out["evals"][i] == w.params.n_orient * len(lig.rot_bond) * w.params.n_angles
        pairs = 0
        for rb in lig.rot_bond:
            mv, _, _, dist = oracle.fragment(n, lig.bonds, int(rb))
            pairs += int(((dist >= 3) & mv[:, None] & ~mv[None, :]).sum())
        assert out["pair_tests_full"][i] == pairs * w.params.n_orient * w.params.n_angles


def early_exit_pairs(lig, pocket, params, o, picks):
    """Pair tests of restart o's sweep when each candidate stops at its first bump.

    Independent replay in numpy/scipy: the conformation of step r is the restart pose
    with the picks of the earlier rotamers applied; each candidate turns rotamer r's
    fragment (networkx) by 2 pi k / A; its pairs are listed moving atom ascending,
    then static atom ascending among those at graph distance >= min_sep; the count is
    the pair count if no pair is closer than bump_dist, else the first bumping pair's
    position rounded up to a whole 32-pair tile (at most the pair count).
    """
    n = len(lig.xyz)
    A = params.n_angles
    spl = dict(nx.all_pairs_shortest_path_length(nx_graph(lig)))
    nz, ny, nx_ = pocket.grid.shape
    x0 = lig.xyz.astype(np.float64)
    cp = pocket.origin.astype(np.float64) + 0.5 * pocket.spacing * np.array([nx_, ny, nz])
    i, j, k = o // (params.n_beta * params.n_gamma), (o // params.n_gamma) % params.n_beta, o % params.n_gamma
    Ro = Rotation.from_euler("ZYZ", [2 * math.pi * i / params.n_alpha, math.pi * (j + 0.5) / params.n_beta,
                                     2 * math.pi * k / params.n_gamma])
    x = cp + Ro.apply(x0 - x0.mean(axis=0))
    total = 0
    for r, rb in enumerate(lig.rot_bond):
        mv, p, q = nx_fragment(lig, int(rb))
        pairs = [(a, b) for a in range(n) if mv[a] for b in range(n) if not mv[b] and spl[a][b] >= params.min_bond_sep]
        ia = np.array([a for a, _ in pairs], dtype=np.int64)
        ib = np.array([b for _, b in pairs], dtype=np.int64)
        u = (x[q] - x[p]) / np.linalg.norm(x[q] - x[p])
        for kk in range(A):
            y = x.copy()
            y[mv] = x[p] + Rotation.from_rotvec(u * 2 * math.pi * kk / A).apply(x[mv] - x[p])
            hit = np.nonzero(np.linalg.norm(y[ia] - y[ib], axis=1) < params.bump_dist)[0]
            total += len(pairs) if len(hit) == 0 else min(len(pairs), 32 * (int(hit[0]) // 32 + 1))
        if picks[r] >= 0:
            x[mv] = x[p] + Rotation.from_rotvec(u * 2 * math.pi * picks[r] / A).apply(x[mv] - x[p])
    return total


def test_early_exit_pair_count_matches_replay():
    pocket = textured_pocket()
    params = synth.SearchParams(2, 2, 2, 16, bump_dist=3.0)
    checked = 0
    for lig in small_ligands():
        b = synth.pack([lig])
        out = oracle.dock_batch(b, pocket, params)
        if np.any(out["orient_fragile"][0] >= 0):
            continue
        O, R = params.n_orient, len(lig.rot_bond)
        # the picks (pinned by the exhaustive replay above) fix the trajectory; the count
        # along it is recomputed independently
        picks = out["orient_pick"].reshape(O, R)
        want = sum(early_exit_pairs(lig, pocket, params, o, picks[o]) for o in range(O))
        assert out["pair_tests_early"][0] == want
        assert 0 < want <= out["pair_tests_full"][0]
        checked += 1
    assert checked >= 2


def test_early_exit_pair_count_limits():
    w = synth.workload_batched(4)
    out = oracle.dock_batch(w.batch, w.pocket, w.params)
    # nothing closer than 0 A: every candidate tests all its pairs
    none = oracle.dock_batch(w.batch, w.pocket, synth.SearchParams(**{**w.params.__dict__, "bump_dist": 0.0}))
    np.testing.assert_array_equal(none["pair_tests_early"], none["pair_tests_full"])
    # everything bumps: the first pair of every candidate bumps, one 32-pair tile each
    huge = oracle.dock_batch(w.batch, w.pocket, synth.SearchParams(**{**w.params.__dict__, "bump_dist": 1e6}))
    for i in range(4):
        lig = w.batch.ligand(i)
        n = len(lig.xyz)
        want = 0
        for rb in lig.rot_bond:
            mv, _, _, dist = oracle.fragment(n, lig.bonds, int(rb))
            want += min(32, int(((dist >= 3) & mv[:, None] & ~mv[None, :]).sum()))
        assert huge["pair_tests_early"][i] == want * w.params.n_orient * w.params.n_angles
    assert np.all(out["pair_tests_early"] < out["pair_tests_full"])
    assert np.all(out["pair_tests_early"] > 0)


def test_algorithmic_work_table():
    """The stored per-launch work totals are the oracle's counts of the seeded workloads."""
    from oracle import algorithmic_work as aw
    table = aw.load()
    w = synth.workload_single()
    assert table[w.name] == aw.count(w, threads=2)
    for make in (synth.workload_batched, synth.workload_large):
        w = make()
        t = table[w.name]
        p = w.params
        assert t["ligands"] == w.batch.n_ligands
        assert t["candidates"] == p.n_orient * p.repetitions * p.n_angles * len(w.batch.rot_bond)
        assert t["fp32_ops"] == 16 * t["frag_atom_moves"] + 7 * t["pair_tests_early"]
        assert t["byte_loads"] == t["frag_atom_moves"]
        assert 0 < t["pair_tests_early"] < t["pair_tests_full"]


# ----------------------------------------------------------------------------- rigid sweep

def test_rigid_candidates_are_rotation_vectors_in_order():
    for span, step in [(1, 0.1), (2, 0.05)]:
        W = 2 * span + 1
        vecs = [(i - span, j - span, k - span) for i in range(W) for j in range(W) for k in range(W)
                if (i, j, k) != (span, span, span)]
        np.testing.assert_allclose(oracle.rigid_candidate(0, span, step), np.eye(3), atol=0)
        for m, v in enumerate(vecs, start=1):
            ref = Rotation.from_rotvec(step * np.array(v, float)).as_matrix()
            np.testing.assert_allclose(oracle.rigid_candidate(m, span, step), ref, atol=1e-14)


def test_rigid_sweep_picks_the_best_rigid_candidate():
    w = synth.workload_single()
    lig = w.batch.ligand(0)
    P = textured_pocket()
    span, step = 1, 0.15
    params = synth.SearchParams(2, 2, 2, 32, rigid_span=span, rigid_step=step)
    nz, ny, nx_ = P.grid.shape
    cp = P.origin.astype(np.float64) + 0.5 * P.spacing * np.array([nx_, ny, nz])
    W = 2 * span + 1
    vecs = [(0, 0, 0)] + [(i - span, j - span, k - span) for i in range(W) for j in range(W) for k in range(W)
                          if (i, j, k) != (span, span, span)]
    moved = 0
    for o in range(params.n_orient):
        start = oracle.place(lig.xyz, o, params, P)
        scores = []
        for v in vecs:  # numpy gather of the rigidly rotated pose
            x = cp + Rotation.from_rotvec(step * np.array(v, float)).apply(start - cp)
            idx = np.floor((x - P.origin.astype(np.float64)) / P.spacing).astype(int)
            ok = np.all((idx >= 0) & (idx < [nx_, ny, nz]), axis=1)
            scores.append(int(np.where(ok, P.grid[np.clip(idx[:, 2], 0, nz - 1), np.clip(idx[:, 1], 0, ny - 1),
                                                   np.clip(idx[:, 0], 0, nx_ - 1)], 0).sum()))
        r = oracle.dock_pose(lig, P, params, o)
        if r["fragile"] == 0:
            continue
        assert r["rigid"] == int(np.argmax(scores)), (o, r["rigid"], np.argmax(scores))
        moved += r["rigid"] != 0
    assert moved > 0
