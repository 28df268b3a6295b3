"""FP64 CPU oracle of the GeoDock pose search (test infrastructure).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg use
this package.  It wraps ``geodock_oracle.cpp`` (plain C++, compiled with g++ on first
use) through ctypes; it shares no code with the CUDA library.

Pinned by tests/test_oracle_pins.py against closed forms, scipy/networkx library
routines, hand-built grids and brute-force enumeration.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "geodock_oracle.cpp")
_LIB = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

EPS = 1e-4  # A: perturbation under which a decision counts as fragile


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (no FMA contraction, so results are plain FP64)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread",
                               "-ffp-contract=off", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.POINTER
            L.orc_last_error.restype = C.c_char_p
            L.orc_euler.argtypes = [C.c_int] * 4 + [P(C.c_double)]
            L.orc_rodrigues.argtypes = [P(C.c_double), C.c_double, P(C.c_double), P(C.c_double)]
            L.orc_score.argtypes = [P(C.c_uint8), C.c_int, C.c_int, C.c_int, C.c_double,
                                    P(C.c_double), P(C.c_double), C.c_int]
            L.orc_fragment.argtypes = [C.c_int, P(C.c_int32), C.c_int, C.c_int, P(C.c_uint8),
                                       P(C.c_int), P(C.c_int), P(C.c_int32)]
            L.orc_torsion.argtypes = [C.c_int, P(C.c_int32), C.c_int, C.c_int, C.c_int, C.c_int,
                                      P(C.c_double)]
            L.orc_bumped.argtypes = [C.c_int, P(C.c_int32), C.c_int, C.c_int, C.c_int, C.c_double,
                                     P(C.c_double)]
            L.orc_place.argtypes = [P(C.c_float), C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                    C.c_int, C.c_int, C.c_int, C.c_double, P(C.c_double), P(C.c_double)]
            _lib = L
        return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


class _Params(C.Structure):
    _fields_ = [("n_alpha", C.c_int32), ("n_beta", C.c_int32), ("n_gamma", C.c_int32),
                ("n_angles", C.c_int32), ("bump_dist", C.c_double),
                ("min_bond_sep", C.c_int32), ("repetitions", C.c_int32),
                ("rigid_span", C.c_int32), ("rigid_step", C.c_double)]


def _prm(params):
    return _Params(params.n_alpha, params.n_beta, params.n_gamma, params.n_angles, float(params.bump_dist),
                   params.min_bond_sep, params.repetitions, int(getattr(params, "rigid_span", 0)),
                   float(getattr(params, "rigid_step", 0.0)))


# ------------------------------------------------------------------ single operations

def rigid_candidate(m: int, span: int, step: float) -> np.ndarray:
    """Rotation matrix of candidate m of the rigid alignment sweep."""
    R = np.zeros(9)
    L = lib()
    L.orc_rigid_candidate.argtypes = [C.c_int, C.c_int, C.c_double, C.POINTER(C.c_double)]
    L.orc_rigid_candidate(int(m), int(span), float(step), _p(R, C.c_double))
    return R.reshape(3, 3)


def euler(o: int, na: int, nb: int, ng: int) -> np.ndarray:
    R = np.zeros(9)
    lib().orc_euler(o, na, nb, ng, _p(R, C.c_double))
    return R.reshape(3, 3)


def rodrigues(u, theta: float, v) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.zeros(3)
    lib().orc_rodrigues(_p(u, C.c_double), float(theta), _p(v, C.c_double), _p(out, C.c_double))
    return out


def score(pocket, xyz) -> int:
    g = np.ascontiguousarray(pocket.grid, dtype=np.uint8)
    nz, ny, nx = g.shape
    o = np.ascontiguousarray(pocket.origin, dtype=np.float64)
    x = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    return lib().orc_score(_p(g, C.c_uint8), nx, ny, nz, float(pocket.spacing), _p(o, C.c_double),
                           _p(x, C.c_double), len(x))


def place(xyz, o: int, params, pocket) -> np.ndarray:
    """Restart pose ``o`` of the ligand ``xyz`` placed in ``pocket``."""
    x = np.ascontiguousarray(xyz, dtype=np.float32).reshape(-1, 3)
    nz, ny, nx = pocket.grid.shape
    org = np.ascontiguousarray(pocket.origin, dtype=np.float64)
    out = np.zeros((len(x), 3))
    lib().orc_place(_p(x, C.c_float), len(x), o, params.n_alpha, params.n_beta, params.n_gamma,
                    nx, ny, nz, float(pocket.spacing), _p(org, C.c_double), _p(out, C.c_double))
    return out


def fragment(n: int, bonds, rb: int):
    """(moving mask, p, q, graph-distance matrix) of rotamer bond ``rb``."""
    b = np.ascontiguousarray(bonds, dtype=np.int32)
    mv = np.zeros(n, dtype=np.uint8)
    p, q = C.c_int(), C.c_int()
    dist = np.zeros((n, n), dtype=np.int32)
    if lib().orc_fragment(n, _p(b, C.c_int32), len(b), rb, _p(mv, C.c_uint8), C.byref(p), C.byref(q),
                          _p(dist, C.c_int32)):
        raise ValueError(lib().orc_last_error().decode())
    return mv.astype(bool), p.value, q.value, dist


def torsion(xyz, bonds, rb: int, k: int, A: int) -> np.ndarray:
    x = np.array(xyz, dtype=np.float64).reshape(-1, 3).copy()
    b = np.ascontiguousarray(bonds, dtype=np.int32)
    if lib().orc_torsion(len(x), _p(b, C.c_int32), len(b), rb, k, A, _p(x, C.c_double)):
        raise ValueError(lib().orc_last_error().decode())
    return x


def bumped(xyz, bonds, rb: int, min_sep: int = 3, bump_dist: float = 2.0) -> bool:
    x = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    b = np.ascontiguousarray(bonds, dtype=np.int32)
    r = lib().orc_bumped(len(x), _p(b, C.c_int32), len(b), rb, min_sep, float(bump_dist), _p(x, C.c_double))
    if r < 0:
        raise ValueError(lib().orc_last_error().decode())
    return bool(r)


def features(xyz, n_rot: int, o: int, params, pocket, eps: float = EPS) -> dict:
    """The proposer's 48 features of one (ligand, restart) in FP64, with near-tie flags."""
    x = np.ascontiguousarray(xyz, np.float32).reshape(-1, 3)
    g = np.ascontiguousarray(pocket.grid, dtype=np.uint8)
    nz, ny, nx_ = g.shape
    org = np.ascontiguousarray(pocket.origin, dtype=np.float64)
    feat = np.zeros(48)
    fps = np.zeros(25, np.int32)
    gap, edge = C.c_double(), C.c_double()
    frag = np.zeros(25, np.uint8)
    L = lib()
    L.orc_features.argtypes = [C.POINTER(C.c_float), C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                               C.POINTER(C.c_uint8), C.c_int, C.c_int, C.c_int, C.c_double, C.POINTER(C.c_double),
                               C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_double),
                               C.POINTER(C.c_double), C.POINTER(C.c_uint8)]
    if L.orc_features(_p(x, C.c_float), len(x), int(n_rot), int(o), params.n_alpha, params.n_beta, params.n_gamma,
                      _p(g, C.c_uint8), nx_, ny, nz, float(pocket.spacing), _p(org, C.c_double), float(eps),
                      _p(feat, C.c_double), _p(fps, C.c_int32), C.byref(gap), C.byref(edge), _p(frag, C.c_uint8)):
        raise ValueError("bad ligand")
    return dict(feat=feat, fps=fps, fps_gap=gap.value, hist_edge=edge.value, sample_fragile=frag.astype(bool))


# ------------------------------------------------------------------ whole search

def dock_pose(lig, pocket, params, o: int, debug: bool = False, eps: float = EPS) -> dict:
    """One restart ``o`` of one ligand: picks, score (+ eps interval), first fragile step, coords,
    step_fragile (1 where a step's pick is fragile; bit 2 of step 0: the rigid choice)."""
    n, R = len(lig.xyz), len(lig.rot_bond)
    reps, A = params.repetitions, params.n_angles
    x = np.ascontiguousarray(lig.xyz, np.float32)
    b = np.ascontiguousarray(lig.bonds, np.int32)
    rb = np.ascontiguousarray(lig.rot_bond, np.int32)
    g = np.ascontiguousarray(pocket.grid, dtype=np.uint8)
    nz, ny, nx_ = g.shape
    org = np.ascontiguousarray(pocket.origin, dtype=np.float64)
    prm = _prm(params)
    picks = np.zeros(reps * R, np.int16)
    slhf = np.zeros(5, np.int32)
    xyz = np.zeros((n, 3))
    sfrag = np.zeros(reps * R, np.uint8)
    bump = np.zeros(reps * R * A, np.uint8) if debug else None
    cand = np.zeros(reps * R * A, np.int32) if debug else None
    nul = lambda ct: C.cast(None, C.POINTER(ct))
    rc = lib().orc_dock_pose(n, _p(x, C.c_float), len(b), _p(b, C.c_int32), R, _p(rb, C.c_int32),
                             _p(g, C.c_uint8), nx_, ny, nz, C.c_double(pocket.spacing), _p(org, C.c_double),
                             C.byref(prm), C.c_double(eps), int(o), _p(picks, C.c_int16),
                             _p(bump, C.c_uint8) if debug else nul(C.c_uint8),
                             _p(cand, C.c_int32) if debug else nul(C.c_int32),
                             _p(slhf, C.c_int32), _p(xyz, C.c_double), _p(sfrag, C.c_uint8))
    if rc:
        raise ValueError(lib().orc_last_error().decode())
    out = dict(picks=picks, score=int(slhf[0]), score_lo=int(slhf[1]), score_hi=int(slhf[2]),
               fragile=int(slhf[3]), rigid=int(slhf[4]), xyz=xyz, step_fragile=sfrag)
    if debug:
        out["bump"], out["cand_score"] = bump, cand
    return out


def dock_batch(batch, pocket, params, n_threads: int = 1, debug: bool = False, eps: float = EPS) -> dict:
    """Run the search over a CSR ligand batch; returns per-ligand / per-orientation arrays.

    Keys: orient_score/_lo/_hi [L, O], orient_pick [sum R * O * reps] (ligand-major,
    then orientation, then rep*R + r), orient_fragile [L, O] (first fragile step, -1 none),
    orient_step_fragile (laid out as orient_pick: 1 where that step's pick is fragile, bit 2
    of a restart's step 0 when its rigid choice is), best_xyz [N, 3],
    best_orient/best_score/best_robust [L], pair_tests_full/evals [L], pair_tests_early [L]
    (pair tests when every candidate stops at its first bumping pair, moving atom
    ascending then static atom ascending, charged in whole 32-pair tiles); with ``debug``
    also bump (0 free / 1 bumped / 2 uncertain) and cand_score per candidate,
    flattened per ligand as [O, reps*R, A] at offsets cand_off.
    """
    L = batch.n_ligands
    O = params.n_alpha * params.n_beta * params.n_gamma
    reps = params.repetitions
    A = params.n_angles
    R = np.diff(batch.rot_off).astype(np.int64)
    cand_off = np.concatenate([[0], np.cumsum(O * reps * R * A)]).astype(np.int64)
    out = dict(
        orient_score=np.zeros((L, O), np.int32), orient_score_lo=np.zeros((L, O), np.int32),
        orient_score_hi=np.zeros((L, O), np.int32),
        orient_pick=np.zeros(int(R.sum()) * O * reps, np.int16),
        orient_fragile=np.zeros((L, O), np.int32), best_xyz=np.zeros((len(batch.xyz), 3)),
        best_orient=np.zeros(L, np.int32), best_score=np.zeros(L, np.int32),
        best_robust=np.zeros(L, np.int32), pair_tests_full=np.zeros(L, np.int64),
        evals=np.zeros(L, np.int64), status=np.zeros(L, np.int32), cand_off=cand_off,
        orient_rigid=np.zeros((L, O), np.int16), pair_tests_early=np.zeros(L, np.int64),
        orient_step_fragile=np.zeros(int(R.sum()) * O * reps, np.uint8))
    if debug:
        out["bump"] = np.zeros(int(cand_off[-1]), np.uint8)
        out["cand_score"] = np.zeros(int(cand_off[-1]), np.int32)
    prm = _prm(params)
    g = np.ascontiguousarray(pocket.grid, dtype=np.uint8)
    nz, ny, nx = g.shape
    org = np.ascontiguousarray(pocket.origin, dtype=np.float64)
    ao = np.ascontiguousarray(batch.atom_off, np.int32)
    xyz = np.ascontiguousarray(batch.xyz, np.float32)
    bo = np.ascontiguousarray(batch.bond_off, np.int32)
    bd = np.ascontiguousarray(batch.bonds, np.int32)
    ro = np.ascontiguousarray(batch.rot_off, np.int32)
    rb = np.ascontiguousarray(batch.rot_bond, np.int32)
    nul = lambda ct: C.cast(None, C.POINTER(ct))
    rc = lib().orc_dock_batch(
        L, _p(ao, C.c_int32), _p(xyz, C.c_float), _p(bo, C.c_int32), _p(bd, C.c_int32),
        _p(ro, C.c_int32), _p(rb, C.c_int32), _p(g, C.c_uint8), nx, ny, nz,
        C.c_double(pocket.spacing), _p(org, C.c_double), C.byref(prm), C.c_double(eps),
        int(n_threads), _p(out["orient_score"], C.c_int32), _p(out["orient_score_lo"], C.c_int32),
        _p(out["orient_score_hi"], C.c_int32), _p(out["orient_pick"], C.c_int16),
        _p(out["orient_fragile"], C.c_int32),
        _p(out["bump"], C.c_uint8) if debug else nul(C.c_uint8),
        _p(out["cand_score"], C.c_int32) if debug else nul(C.c_int32),
        _p(cand_off, C.c_int64), _p(out["best_xyz"], C.c_double), _p(out["best_orient"], C.c_int32),
        _p(out["best_score"], C.c_int32), _p(out["best_robust"], C.c_int32),
        _p(out["pair_tests_full"], C.c_int64), _p(out["evals"], C.c_int64), _p(out["status"], C.c_int32),
        _p(out["orient_rigid"], C.c_int16), _p(out["pair_tests_early"], C.c_int64),
        _p(out["orient_step_fragile"], C.c_uint8))
    if rc:
        raise ValueError("oracle rejected a ligand: " + lib().orc_last_error().decode())
    return out
