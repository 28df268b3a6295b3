"""Seeded synthetic inputs for the GeoDock pose search: ligand trees and pocket grids.

This module only *makes inputs*.  It holds none of the search arithmetic (placement,
torsion rotation, bump test, scoring, argmax): both the CUDA path and the CPU oracle
receive the arrays produced here and derive everything else on their own.

The paper's experiments dock a library of ligands (atoms + rotamers) against one
target pocket (Sec. 3.1, Listing 1; Sec. 5) but neither the dataset nor the pocket is
published.  The generators below stand in for them with the shapes the workloads
fix: random heavy-atom trees with 1.50 A bonds, 109.5 deg bond angles and uniform
torsions; rotamers on non-terminal tree edges; a uint8 pocket score grid built as a
union of spheres valued 255 inside and decaying linearly to 0 over 2 A.

Randomness: SplitMix64 (Steele, Lea & Flood 2014), one independent stream per ligand
seeded with ``seed ^ (i * 0x9E3779B97F4A7C15)``, so any ligand of a workload can be
regenerated alone.  Geometry is built in float64 and rounded once to float32, which is
the coordinate type both implementations consume.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_M64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15
BOND_LEN = 1.50            # A
BOND_ANGLE_DEG = 109.5     # deg
CLASH_REDRAW = 2.2         # A: a new atom closer than this to a non-bonded atom is redrawn
MAX_VALENCE = 4            # heavy-atom degree cap used when picking a parent
BASE_SEED = 1901062290


class SplitMix64:
    """SplitMix64 generator; integer state, exact across platforms."""

    def __init__(self, seed: int):
        self.s = seed & _M64

    def next_u64(self) -> int:
        self.s = (self.s + GOLDEN) & _M64
        z = self.s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive)."""
        return lo + self.next_u64() % (hi - lo + 1)

    def normal(self) -> float:
        """Standard normal by Box-Muller (one of the pair)."""
        u1 = 1.0 - self.uniform()
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


def ligand_seed(config_seed: int, index: int) -> int:
    return (config_seed ^ ((index * GOLDEN) & _M64)) & _M64


# ----------------------------------------------------------------------------- ligands

def _frame(a, b, c):
    """Orthonormal frame (bc, m, n) of NeRF placement after the chain a-b-c."""
    bc = [c[k] - b[k] for k in range(3)]
    inv = 1.0 / math.sqrt(bc[0] ** 2 + bc[1] ** 2 + bc[2] ** 2)
    bc = [x * inv for x in bc]
    ab = [b[k] - a[k] for k in range(3)]
    n = [ab[1] * bc[2] - ab[2] * bc[1], ab[2] * bc[0] - ab[0] * bc[2], ab[0] * bc[1] - ab[1] * bc[0]]
    inv = 1.0 / math.sqrt(n[0] ** 2 + n[1] ** 2 + n[2] ** 2)
    n = [x * inv for x in n]
    m = [n[1] * bc[2] - n[2] * bc[1], n[2] * bc[0] - n[0] * bc[2], n[0] * bc[1] - n[1] * bc[0]]
    return bc, m, n


def _nerf(a, b, c, bond, angle, torsion):
    """Place d so that |cd| = bond, angle(b, c, d) = angle, dihedral(a, b, c, d) = torsion."""
    bc, m, n = _frame(a, b, c)
    d0 = -bond * math.cos(angle)
    d1 = bond * math.sin(angle) * math.cos(torsion)
    d2 = bond * math.sin(angle) * math.sin(torsion)
    return np.array([c[k] + d0 * bc[k] + d1 * m[k] + d2 * n[k] for k in range(3)])


@dataclass
class Ligand:
    xyz: np.ndarray          # float32 [n, 3]
    bonds: np.ndarray        # int32 [n-1, 2] (parent, child), ligand-local atom ids
    rot_bond: np.ndarray     # int32 [R] indices into bonds, in search order


def gen_ligand(rng: SplitMix64, n_atoms: int, n_rot: int, max_tree_tries: int = 200) -> Ligand:
    """Random heavy-atom tree with ``n_atoms`` atoms and ``n_rot`` rotamers.

    Atom 0 sits at the origin and atom 1 at +1.5 A on x.  Every further atom picks a
    parent uniformly among atoms of degree < 4 and is placed by NeRF at 1.50 A from
    it, at 109.5 deg to the parent's first neighbour, with a uniform torsion.  A draw
    within 2.2 A of any atom other than its parent is redrawn (new torsion; after 32
    torsions, a new parent).  Rotamers are ``n_rot`` distinct non-terminal edges (both
    endpoints of degree >= 2) drawn uniformly; the whole tree is redrawn if fewer exist.
    """
    if n_atoms < 2:
        raise ValueError("a ligand needs at least 2 atoms")
    ang = math.radians(BOND_ANGLE_DEG)
    clash2 = CLASH_REDRAW * CLASH_REDRAW
    for _ in range(max_tree_tries):
        xyz = np.zeros((n_atoms, 3), dtype=np.float64)
        nbrs: list[list[int]] = [[] for _ in range(n_atoms)]
        bonds = []
        xyz[1] = (BOND_LEN, 0.0, 0.0)
        nbrs[0].append(1)
        nbrs[1].append(0)
        bonds.append((0, 1))
        ok = True
        for i in range(2, n_atoms):
            placed = False
            cands = [a for a in range(i) if len(nbrs[a]) < MAX_VALENCE]
            for _ptry in range(64):
                par = cands[rng.randint(0, len(cands) - 1)]
                first = nbrs[par][0]
                ref = next((g for g in nbrs[first] if g != par), None)
                a = xyz[ref] if ref is not None else xyz[first] + np.array([0.0, 1.0, 0.0])
                bc, m, nn = _frame(a.tolist(), xyz[first].tolist(), xyz[par].tolist())
                cpar = xyz[par].tolist()
                d0 = -BOND_LEN * math.cos(ang)
                rs = BOND_LEN * math.sin(ang)
                for _ttry in range(32):
                    tors = 2.0 * math.pi * rng.uniform()
                    d1, d2_ = rs * math.cos(tors), rs * math.sin(tors)
                    pos = np.array([cpar[k] + d0 * bc[k] + d1 * m[k] + d2_ * nn[k] for k in range(3)])
                    d2 = np.sum((xyz[:i] - pos) ** 2, axis=1)
                    d2[par] = np.inf
                    if np.all(d2 >= clash2):
                        xyz[i] = pos
                        nbrs[par].append(i)
                        nbrs[i].append(par)
                        bonds.append((par, i))
                        placed = True
                        break
                if placed:
                    break
            if not placed:
                ok = False
                break
        if not ok:
            continue
        deg = [len(x) for x in nbrs]
        nonterm = [b for b, (u, v) in enumerate(bonds) if deg[u] >= 2 and deg[v] >= 2]
        if len(nonterm) < n_rot:
            continue
        # partial Fisher-Yates: n_rot distinct edges, in draw order
        pool = list(nonterm)
        rot = []
        for r in range(n_rot):
            j = rng.randint(r, len(pool) - 1)
            pool[r], pool[j] = pool[j], pool[r]
            rot.append(pool[r])
        return Ligand(xyz=xyz.astype(np.float32),
                      bonds=np.asarray(bonds, dtype=np.int32).reshape(-1, 2),
                      rot_bond=np.asarray(rot, dtype=np.int32))
    raise RuntimeError(f"could not build a {n_atoms}-atom tree with {n_rot} rotamers")


# ----------------------------------------------------------------------------- pockets

@dataclass
class Pocket:
    grid: np.ndarray         # uint8 [nz, ny, nx]
    spacing: float
    origin: np.ndarray       # float32 [3] (x, y, z) of the grid corner
    spheres: np.ndarray = field(default_factory=lambda: np.zeros((0, 4)))  # (cx, cy, cz, r)

    @property
    def shape_xyz(self):
        nz, ny, nx = self.grid.shape
        return nx, ny, nz


def pocket_values(spheres: np.ndarray, centres: np.ndarray) -> np.ndarray:
    """Score of points ``centres`` [..., 3] for a union of spheres (cx, cy, cz, r).

    255 inside any sphere, falling linearly to 0 over 2 A outside the surface; the
    value is the maximum over spheres and is rounded half up to an integer.
    """
    best = np.zeros(centres.shape[:-1], dtype=np.float64)
    for cx, cy, cz, r in spheres:
        d = np.sqrt((centres[..., 0] - cx) ** 2 + (centres[..., 1] - cy) ** 2
                    + (centres[..., 2] - cz) ** 2) - r
        d = np.maximum(d, 0.0)
        best = np.maximum(best, np.clip(1.0 - d / 2.0, 0.0, 1.0))
    return np.floor(255.0 * best + 0.5).astype(np.uint8)


def gen_pocket(rng: SplitMix64, n: int, spacing: float, n_spheres: int, ball_frac: float,
               centre=(12.5, -7.25, 3.0)) -> Pocket:
    """``n``^3 uint8 grid whose box is centred on ``centre``.

    Sphere centres are uniform in a ball of radius ``ball_frac * box`` about the box
    centre, radii uniform in [3, 5] A; each cell takes the value at its centre.
    """
    centre = np.asarray(centre, dtype=np.float64)
    box = n * spacing
    sph = []
    for _ in range(n_spheres):
        while True:
            v = np.array([2.0 * rng.uniform() - 1.0 for _ in range(3)])
            if v @ v <= 1.0:
                break
        r = 3.0 + 2.0 * rng.uniform()
        sph.append((*(centre + ball_frac * box * v), r))
    sph = np.asarray(sph, dtype=np.float64)
    origin = (centre - box / 2.0).astype(np.float32)
    ax = origin.astype(np.float64)[None, :] + (np.arange(n, dtype=np.float64)[:, None] + 0.5) * spacing
    zz, yy, xx = np.meshgrid(ax[:, 2], ax[:, 1], ax[:, 0], indexing="ij")
    grid = pocket_values(sph, np.stack([xx, yy, zz], axis=-1))
    return Pocket(grid=np.ascontiguousarray(grid), spacing=float(spacing), origin=origin, spheres=sph)


# ----------------------------------------------------------------------------- batches

@dataclass
class LigandBatch:
    """CSR ligand library (host arrays), the input format of ``gd_dock_batch``."""
    atom_off: np.ndarray     # int32 [L+1]
    xyz: np.ndarray          # float32 [N, 3]
    bond_off: np.ndarray     # int32 [L+1]
    bonds: np.ndarray        # int32 [B, 2], ligand-local ids
    rot_off: np.ndarray      # int32 [L+1]
    rot_bond: np.ndarray     # int32 [Rtot], indices into the ligand's own bond list

    @property
    def n_ligands(self) -> int:
        return len(self.atom_off) - 1

    def ligand(self, i: int) -> Ligand:
        a0, a1 = self.atom_off[i], self.atom_off[i + 1]
        b0, b1 = self.bond_off[i], self.bond_off[i + 1]
        r0, r1 = self.rot_off[i], self.rot_off[i + 1]
        return Ligand(xyz=self.xyz[a0:a1], bonds=self.bonds[b0:b1], rot_bond=self.rot_bond[r0:r1])

    def subset(self, idx) -> "LigandBatch":
        """The ligands idx (in that order) as a new batch: one ragged gather per array."""
        idx = np.asarray(idx, dtype=np.int64).reshape(-1)

        def ragged(off, rows):
            off = np.asarray(off, dtype=np.int64)
            starts, lens = off[idx], off[idx + 1] - off[idx]
            new_off = np.concatenate([[0], np.cumsum(lens)])
            take = np.arange(new_off[-1]) - np.repeat(new_off[:-1], lens) + np.repeat(starts, lens)
            return new_off.astype(np.int32), np.ascontiguousarray(rows[take])

        atom_off, xyz = ragged(self.atom_off, np.asarray(self.xyz, np.float32).reshape(-1, 3))
        bond_off, bonds = ragged(self.bond_off, np.asarray(self.bonds, np.int32).reshape(-1, 2))
        rot_off, rot_bond = ragged(self.rot_off, np.asarray(self.rot_bond, np.int32))
        return LigandBatch(atom_off=atom_off, xyz=xyz, bond_off=bond_off, bonds=bonds, rot_off=rot_off,
                           rot_bond=rot_bond)


def pack(ligs: list[Ligand]) -> LigandBatch:
    na = np.array([len(l.xyz) for l in ligs], dtype=np.int64)
    nb = np.array([len(l.bonds) for l in ligs], dtype=np.int64)
    nr = np.array([len(l.rot_bond) for l in ligs], dtype=np.int64)
    off = lambda c: np.concatenate([[0], np.cumsum(c)]).astype(np.int32)
    return LigandBatch(
        atom_off=off(na),
        xyz=(np.concatenate([l.xyz for l in ligs]) if ligs else np.zeros((0, 3))).astype(np.float32).reshape(-1, 3),
        bond_off=off(nb),
        bonds=(np.concatenate([l.bonds for l in ligs]) if ligs else np.zeros((0, 2))).astype(np.int32).reshape(-1, 2),
        rot_off=off(nr),
        rot_bond=(np.concatenate([l.rot_bond for l in ligs]) if ligs else np.zeros(0)).astype(np.int32),
    )


@dataclass
class SearchParams:
    """Search settings of one docking run (mirrors ``gd_search_params``)."""
    n_alpha: int = 4
    n_beta: int = 4
    n_gamma: int = 4
    n_angles: int = 32
    bump_dist: float = 2.0
    min_bond_sep: int = 3
    repetitions: int = 1
    rigid_span: int = 0        # rigid alignment sweep over (2s+1)^3 rotation vectors (0 = off)
    rigid_step: float = 0.0    # radians

    @property
    def n_orient(self) -> int:
        return self.n_alpha * self.n_beta * self.n_gamma


@dataclass
class Workload:
    name: str
    pocket: Pocket
    batch: LigandBatch
    params: SearchParams


def _ligand_range(config_seed, size_fn, lo, hi):
    out = []
    for i in range(lo, hi):
        rng = SplitMix64(ligand_seed(config_seed, i))
        n, r = size_fn(rng)
        out.append(gen_ligand(rng, n, r))
    return out


def _ligands(config_seed, count, size_fn, start=0, workers=None):
    """Ligands start .. start+count-1 of a workload.  Large requests are split over a
    'spawn' process pool (safe after CUDA has been initialised); every ligand has its
    own generator stream, so the result does not depend on the split."""
    import os
    if workers is None:
        workers = min(os.cpu_count() or 1, 16)
    if count < 256 or workers <= 1:
        return _ligand_range(config_seed, size_fn, start, start + count)
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    chunk = (count + workers * 4 - 1) // (workers * 4)
    bounds = [(lo, min(lo + chunk, start + count)) for lo in range(start, start + count, chunk)]
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        parts = ex.map(_ligand_range, [config_seed] * len(bounds), [size_fn] * len(bounds),
                       [b[0] for b in bounds], [b[1] for b in bounds])
        return [lig for part in parts for lig in part]


def workload_single(seed_offset: int = 1) -> Workload:
    """One 24-atom, 4-rotamer ligand vs a 32^3 pocket at 0.5 A (6 spheres);
    64 orientations (4x4x4 Euler grid), 32 angles."""
    seed = BASE_SEED + seed_offset
    pocket = gen_pocket(SplitMix64(seed ^ 0x5EED), 32, 0.5, 6, 0.25)
    ligs = _ligands(seed, 1, lambda rng: (24, 4))
    return Workload("single-24atom-32grid", pocket, pack(ligs), SearchParams(4, 4, 4, 32))


def c2_sizes(rng):
    n = rng.randint(20, 80)
    return n, min(rng.randint(2, 12), n // 5)


def c3_sizes(rng):
    return rng.randint(100, 250), rng.randint(20, 60)


def c1_style_sizes(rng):
    return 24, 4


def lognormal_sizes(rng):
    n = int(round(math.exp(math.log(40.0) + 0.5 * rng.normal())))
    n = max(15, min(250, n))
    return n, max(1, int(round(n / 6)))


def pocket_64(seed=BASE_SEED + 2) -> Pocket:
    return gen_pocket(SplitMix64(seed ^ 0x5EED), 64, 0.375, 12, 0.25)


def workload_batched(n_ligands: int = 4096, start: int = 0) -> Workload:
    """Batched plain search: atoms U{20..80}, rotamers min(U{2..12}, atoms//5);
    64^3 pocket at 0.375 A (12 spheres); 256 orientations (8x8x4), 64 angles."""
    seed = BASE_SEED + 2
    ligs = _ligands(seed, n_ligands, c2_sizes, start)
    return Workload(f"batched-{n_ligands}lig-64grid", pocket_64(), pack(ligs), SearchParams(8, 8, 4, 64))


def workload_large(n_ligands: int = 512, start: int = 0) -> Workload:
    """Large flexible ligands: atoms U{100..250}, rotamers U{20..60}; 128^3 pocket at
    0.375 A (20 spheres, ball 0.3 box); 256 orientations, 128 angles."""
    seed = BASE_SEED + 3
    pocket = gen_pocket(SplitMix64(seed ^ 0x5EED), 128, 0.375, 20, 0.30)
    ligs = _ligands(seed, n_ligands, c3_sizes, start)
    return Workload(f"large-{n_ligands}lig-128grid", pocket, pack(ligs), SearchParams(8, 8, 4, 128))


def workload_proposer_train(n_ligands: int = 3907) -> Workload:
    """Training tuples of the learned proposer: fresh 24-atom, 4-rotamer ligands docked
    exhaustively (256 restarts, 64 angles) on the 64^3 pocket: 3,907 x 256 ~ 1M rows."""
    ligs = _ligands(BASE_SEED + 4, n_ligands, c1_style_sizes)
    return Workload(f"proposer-train-{n_ligands}lig", pocket_64(), pack(ligs), SearchParams(8, 8, 4, 64))


def workload_proposer_eval(n_ligands: int = 16384, start: int = 0) -> Workload:
    """Held-out ligands of the same kind (other seeds) for recall / regret / throughput."""
    ligs = _ligands(BASE_SEED + 40, n_ligands, c1_style_sizes, start)
    return Workload(f"proposer-eval-{n_ligands}lig", pocket_64(), pack(ligs), SearchParams(8, 8, 4, 64))


def workload_stream(n_ligands: int = 100000, start: int = 0, seed_offset: int = 5) -> Workload:
    """Streaming-screen ligands: atoms lognormal (median 40, sigma 0.5) clamped to
    15..250, rotamers round(atoms / 6); 64^3 pocket; 256 restarts, 64 angles."""
    ligs = _ligands(BASE_SEED + seed_offset, n_ligands, lognormal_sizes, start)
    return Workload(f"stream-{n_ligands}lig", pocket_64(), pack(ligs), SearchParams(8, 8, 4, 64))
