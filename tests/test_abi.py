"""The C ABI library: it loads, exports every entry point of include/geodock.h, and its
host-side validation rejects malformed batches (no device needed)."""
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1901_06229_b300 import geodock as gdk
from paper_1901_06229_b300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions(name="geodock.h"):
    src = open(os.path.join(ROOT, "include", name)).read()
    return sorted(set(re.findall(r"^(?:gd_status|int|const char\*)\s+(gd_\w+)\(", src, re.M)))


def all_header_functions():
    out = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            out |= set(header_functions(f))
    return sorted(out)


def test_library_exports_every_declared_function():
    lib = gdk.load()
    declared = header_functions()
    assert len(declared) >= 13
    for f in declared:
        assert hasattr(lib, f), f
    syms = subprocess.run(["nm", "-D", "--defined-only", gdk.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (gd_\w+)", syms))
    assert set(all_header_functions()) <= exported
    assert set(gdk.EXPORTS) == set(declared)


def test_tiles():
    assert gdk.tile_count() == 20
    seen = {gdk.tile_info(t) for t in range(1, 21)}
    assert len(seen) == 20
    assert {r for _, _, r in seen} == {80, 96, 128}
    with pytest.raises(gdk.GeoDockError):
        gdk.tile_info(0)


def _lig(bonds, rot, n=None):
    bonds = np.asarray(bonds, np.int32)
    n = n or int(bonds.max()) + 1
    xyz = np.stack([np.arange(n) * 3.0, np.zeros(n), np.zeros(n)], 1).astype(np.float32)
    return synth.Ligand(xyz=xyz, bonds=bonds.reshape(-1, 2), rot_bond=np.asarray(rot, np.int32))


CHAIN = [[0, 1], [1, 2], [2, 3], [3, 4], [4, 5]]


def test_check_batch_accepts_generated_workloads():
    for w in (synth.workload_single(), synth.workload_batched(50)):
        gdk.check_batch(w.batch, w.params)
    gdk.check_batch(synth.pack([]), synth.SearchParams())


@pytest.mark.parametrize("lig,msg", [
    (lambda: _lig([[0, 1], [1, 2], [2, 0]], [], n=4), "tree"),           # cycle
    (lambda: _lig([[0, 1], [2, 3], [1, 0]], [], n=4), "tree"),           # disconnected
    (lambda: _lig(CHAIN, [0]), "terminal"),                               # terminal rotamer
    (lambda: _lig(CHAIN, [7]), "bond"),                                   # rotamer bond out of range
    (lambda: _lig([[0, 7]], [], n=2), "bond"),                            # atom id out of range
    (lambda: _lig([[0, 0]], [], n=2), "bond"),                            # self bond
    (lambda: _lig([[i, i + 1] for i in range(256)], []), "atoms"),        # 257 atoms
])
def test_check_batch_rejects(lig, msg):
    with pytest.raises(gdk.GeoDockError) as e:
        gdk.check_batch(synth.pack([lig()]), synth.SearchParams())
    assert e.value.status == gdk.GD_EINVAL and msg in str(e.value)


def test_check_batch_rejects_nan_and_bad_params():
    l = _lig(CHAIN, [2])
    l.xyz[3, 1] = np.nan
    with pytest.raises(gdk.GeoDockError, match="finite"):
        gdk.check_batch(synth.pack([l]), synth.SearchParams())
    ok = synth.pack([_lig(CHAIN, [2])])
    for bad in (synth.SearchParams(0, 4, 4), synth.SearchParams(n_angles=0), synth.SearchParams(n_angles=2000),
                synth.SearchParams(bump_dist=-1.0), synth.SearchParams(repetitions=0),
                synth.SearchParams(min_bond_sep=0), synth.SearchParams(300, 300, 1)):
        with pytest.raises(gdk.GeoDockError) as e:
            gdk.check_batch(ok, bad)
        assert e.value.status == gdk.GD_EINVAL


def test_check_batch_excluded_pair_limit():
    # a star: every atom bonded to atom 1 -> with min_bond_sep 4 the pairs across the
    # rotamer bond 1-2 that are fewer than 4 bonds apart exceed the per-rotamer limit
    bonds = [[0, 1]] + [[1, k] for k in range(2, 5)] + [[2, k] for k in range(5, 9)] + [[3, 9]]
    l = _lig(bonds, [1])
    gdk.check_batch(synth.pack([l]), synth.SearchParams())
    gdk.check_batch(synth.pack([l]), synth.SearchParams(min_bond_sep=5))
    # a long path with many branches: pairs within 8 bonds across the bond exceed 128
    bonds = [[i, i + 1] for i in range(20)] + [[i, 21 + i] for i in range(20)] + \
            [[i, 41 + i] for i in range(20)]
    l = _lig(bonds, [9])
    with pytest.raises(gdk.GeoDockError, match="excluded"):
        gdk.check_batch(synth.pack([l]), synth.SearchParams(min_bond_sep=8))


def _reason(fn):
    with pytest.raises(gdk.GeoDockError) as e:
        fn()
    return e.value.status, str(e.value)


_BAD_LIGANDS = [lambda: _lig([[0, 1], [1, 2], [2, 0]], [], n=4), lambda: _lig([[0, 1], [2, 3], [1, 0]], [], n=4),
                lambda: _lig(CHAIN, [0]), lambda: _lig(CHAIN, [7]), lambda: _lig([[0, 7]], [], n=2),
                lambda: _lig([[0, 0]], [], n=2), lambda: _lig([[i, i + 1] for i in range(256)], [])]


def test_noalloc_rejects_what_check_batch_rejects_with_the_same_reason():
    """gd_dock_batch_noalloc validates ligands and parameters with the packer and checks
    gd_dock_batch uses, before it touches a device: the same status and message."""
    pocket = synth.workload_single().pocket
    ok = _lig(CHAIN, [2])
    cases = [(synth.pack([mk()]), synth.SearchParams()) for mk in _BAD_LIGANDS]
    nan = _lig(CHAIN, [2])
    nan.xyz[3, 1] = np.nan
    cases.append((synth.pack([ok, nan]), synth.SearchParams()))
    bonds = [[i, i + 1] for i in range(20)] + [[i, 21 + i] for i in range(20)] + [[i, 41 + i] for i in range(20)]
    cases.append((synth.pack([_lig(bonds, [9])]), synth.SearchParams(min_bond_sep=8)))  # excluded-pair limit
    for bad in (synth.SearchParams(0, 4, 4), synth.SearchParams(n_angles=0), synth.SearchParams(n_angles=2000),
                synth.SearchParams(bump_dist=-1.0), synth.SearchParams(repetitions=0),
                synth.SearchParams(min_bond_sep=0), synth.SearchParams(300, 300, 1)):
        cases.append((synth.pack([ok]), bad))
    for batch, params in cases:
        a = _reason(lambda: gdk.check_batch(batch, params))
        b = _reason(lambda: gdk.dock_noalloc(batch, pocket, params))
        assert a[0] == gdk.GD_EINVAL and a == b, (a, b)


def test_noalloc_rejects_the_autotuned_tile():
    w = synth.workload_single()
    st, msg = _reason(lambda: gdk.dock_noalloc(w.batch, w.pocket, w.params, tile=-1))
    assert st == gdk.GD_EINVAL and "context" in msg


C_PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "geodock.h"
#include "geodock_mlp.h"

int main(void) {
  /* a 6-atom chain with its middle bond rotatable, coordinates 1.5 A apart */
  int32_t atom_off[2] = {0, 6}, bond_off[2] = {0, 5}, rot_off[2] = {0, 1};
  int32_t bonds[10] = {0, 1, 1, 2, 2, 3, 3, 4, 4, 5}, rot_bond[1] = {2};
  float xyz[18];
  for (int a = 0; a < 6; ++a) { xyz[3 * a] = 1.5f * a; xyz[3 * a + 1] = 0.3f * (a & 1); xyz[3 * a + 2] = 0.f; }
  gd_ligand_batch b = {1, atom_off, xyz, bond_off, bonds, rot_off, rot_bond};
  gd_search_params p = {4, 4, 4, 32, 2.0f, 3, 1, 0, 0, 0, 0.0f};
  if (gd_check_batch(&b, &p) != GD_OK) { printf("rejected: %s\n", gd_last_error(NULL)); return 1; }
  bonds[9] = 0; /* 4-0 instead of 4-5: a cycle */
  if (gd_check_batch(&b, &p) != GD_EINVAL || strstr(gd_last_error(NULL), "tree") == NULL) return 2;
  int warps = 0, slots = 0, regs = 0;
  if (gd_tile_count() < 1 || gd_tile_info(1, &warps, &slots, &regs) != GD_OK || warps < 1) return 3;
  printf("ok %d tiles\n", gd_tile_count());
  return 0;
}
"""


def test_headers_compile_as_c_and_link(tmp_path):
    """The boundary is a C ABI: a C99 program includes both headers, links the library
    and calls its host-only entry points (no device needed)."""
    import subprocess
    from paper_1901_06229_b300 import build
    lib = build.build()
    src = tmp_path / "use.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "use"
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                           "-o", str(exe), "-L", os.path.dirname(lib), "-lgeodock",
                           f"-Wl,-rpath,{os.path.dirname(lib)}"])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, (out.returncode, out.stdout, out.stderr)
    assert out.stdout.startswith("ok ")
