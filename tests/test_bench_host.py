"""Host-side pieces of the measurement script (no GPU): the recorded DRAM
traffic file and its lookup, the measurement options, the autotuner's option
grid."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_file_is_well_formed():
    n = 0
    for ln in open(bench.TRAFFIC_FILE).read().splitlines():
        if not ln.strip() or ln.startswith("#"):
            continue
        kernel, workload, nbytes, h = ln.split()
        assert workload.startswith("cube") and "_p" in workload
        assert float(nbytes) > 0
        assert len(h) == 16 and int(h, 16) >= 0
        n += 1
    assert n >= 2


def test_traffic_lookup_needs_the_current_sources(tmp_path, monkeypatch):
    f = tmp_path / "traffic.txt"
    cur = bench.kernel_source_hash()
    f.write_text("# comment\nk1 cube1048576_p8 123 %s\nk2 cube1048576_p8 456 0000000000000000\n" % cur)
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.recorded_traffic("k1", "cube1048576_p8") == 123.0
    assert bench.recorded_traffic("k2", "cube1048576_p8") is None  # taken on other sources
    assert bench.recorded_traffic("k1", "cube262144_p8") is None
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.txt"))
    assert bench.recorded_traffic("k1", "cube1048576_p8") is None


def test_measurement_options(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert (a.gpus, a.steps, a.warmup, a.impl, a.only, a.sets) == (1, 20, 5, "ours", None, 64)
    for part in ("build-cube", "build-plummer", "field", "backward", "batched"):
        monkeypatch.setattr(sys, "argv", ["bench.py", "--only", part, "--steps", "2", "--warmup", "1"])
        assert bench.parse().only == part


def test_autotuner_option_grid():
    torch = pytest.importorskip("torch")  # noqa: F841  (the package imports torch)
    from paper_2511_15269_gb300 import autotune, fmm
    combos = list(autotune.option_combos())
    sizes = [len(v) for v in autotune.OPTION_GRID.values()]
    expect = 1
    for k in sizes:
        expect *= k
    assert len(combos) == expect
    assert all(set(c) == set(autotune.OPTION_GRID) for c in combos)
    # the defaults of a new tree are among the candidates
    assert {fmm.FMM_OPT_SCHEDULE: 1, fmm.FMM_OPT_M2M_ONE_LAUNCH: 1, fmm.FMM_OPT_NEAR_SYMMETRIC: 1,
            fmm.FMM_OPT_M2L_BLOCKS_PER_SM: 0} in combos
