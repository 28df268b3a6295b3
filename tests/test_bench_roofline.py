"""The benchmark's roofline bookkeeping on CPU: the measured-peak block, the source hash
that keys the ncu measurements, and the recall targets of the learned path."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_roof", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_pipe_peaks_divides_by_the_measured_rates(bench):
    pipes = {"ffma_per_s": 30.0e12, "lds_u8_per_s": 8.0e12}
    r = bench.pipe_peaks(pipes, achieved=45.0, loads=0.4, peak_tops=40.0, peak_loads=10.0)
    assert r["ffma_T_per_s"] == pytest.approx(30.0)
    assert r["lds_u8_T_per_s"] == pytest.approx(8.0)
    assert r["ffma_of_nominal"] == pytest.approx(0.75)
    assert r["lds_u8_of_nominal"] == pytest.approx(0.8)
    assert r["frac_fp32"] == pytest.approx(1.5)
    assert r["frac_loads"] == pytest.approx(0.05)
    none = bench.pipe_peaks(pipes, achieved=None, loads=None, peak_tops=40.0, peak_loads=10.0)
    assert none["frac_fp32"] is None and none["frac_loads"] is None


def test_kernel_hash_ignores_comments_but_not_code(bench, tmp_path):
    a, b, c = tmp_path / "a.cu", tmp_path / "b.cu", tmp_path / "c.cu"
    a.write_text("int f() { return 1; }\n")
    b.write_text("// a comment\nint f() { return 1; }  // trailing\n\n")
    c.write_text("int f() { return 2; }\n")
    h = bench.search_kernel_hash
    assert h((str(a),)) == h((str(b),))
    assert h((str(a),)) != h((str(c),))


def test_measurement_tables_are_well_formed(bench):
    # every table entry is keyed by a 16-hex-digit hash and (workload, tile)
    for table in (bench.MEASURED_TRAFFIC, bench.MEASURED_INSTRUCTIONS):
        for key, rows in table.items():
            assert len(key) == 16 and int(key, 16) >= 0
            for (name, tile), v in rows.items():
                assert isinstance(name, str) and tile > 0 and v > 0


def test_learned_path_tunes_above_its_recall_target(bench):
    assert bench.RECALL_TARGET == 0.99
    assert bench.RECALL_TARGET < bench.VAL_RECALL_TARGET < 1.0
