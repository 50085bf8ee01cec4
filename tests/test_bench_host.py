"""Host logic of bench.py (no GPU): the workloads' inputs and descriptions,
the kernel family a search runs, and the effective alphabet size used to
read the tuner's table for the skewed text."""
import types

import numpy as np
import pytest

import bench
import hc_inputs as hi


def _args(**kw):
    d = dict(workload="sweep", n=1 << 16, skew_n=1 << 16, cells="", params="tuned", eager=False,
             pos64=False, patterns=3)
    d.update(kw)
    return types.SimpleNamespace(**d)


def test_sweep_inputs_cover_every_cell():
    texts, grid, pats = bench.workload_inputs(_args(), 3)
    assert sorted(texts) == sorted(hi.SWEEP_SIGMAS)
    assert grid == [(s, m) for s in hi.SWEEP_SIGMAS for m in hi.SWEEP_MS]
    for (s, m), ps in pats.items():
        assert len(ps) == 3 and all(p.size == m for p in ps)
        assert set(np.unique(texts[s])) <= set(hi.alphabet(s))


def test_cells_option_limits_the_texts():
    texts, grid, pats = bench.workload_inputs(_args(cells="4:16,95:2"), 2)
    assert grid == [(4, 16), (95, 2)] and sorted(texts) == [4, 95]


def test_skewed_inputs_are_the_markov_text():
    a = _args(workload="skewed")
    texts, grid, pats = bench.workload_inputs(a, 2)
    assert list(texts) == [bench.SKEW_KEY]
    y = texts[bench.SKEW_KEY]
    assert y.size == a.skew_n and np.array_equal(y, hi.skew_text(a.skew_n))
    assert grid == [(bench.SKEW_KEY, m) for m in hi.SKEW_MS]
    for (_, m), ps in pats.items():
        for p in ps:                       # every pattern is copied from the text
            assert (np.lib.stride_tricks.sliding_window_view(y, m) == p).all(axis=1).any()
    cfg = bench.workload_config(a)
    assert cfg["workload"] == "plain HC, skewed text" and cfg["ms"] == list(hi.SKEW_MS)
    assert bench.metric_for(a) == bench.SKEW_METRIC and bench.metric_for(_args()) == bench.METRIC


def test_sigma_eff_closed_forms():
    # uniform over k symbols: exactly k when every symbol is equally frequent
    for k in (1, 2, 4, 20, 95):
        y = np.tile(hi.alphabet(k), 1000)
        assert bench.skew_sigma_eff(y) == pytest.approx(k)
    # two symbols with frequencies 3/4, 1/4: 1 / (9/16 + 1/16) = 1.6
    y = np.array([0, 0, 0, 1] * 1000, dtype=np.uint8)
    assert bench.skew_sigma_eff(y) == pytest.approx(1.6)
    # the skewed text is far more repetitive than its 60 symbols suggest
    assert 5.0 < bench.skew_sigma_eff(hi.skew_text(1 << 22)) < 30.0


@pytest.mark.parametrize("m,q,mode,fam", [(4, 4, 0, "scan_dense"), (16, 6, 0, "scan_staged"),
                                          (1024, 8, 0, "scan_direct"), (256, 4, 0, "scan_direct"),
                                          (199, 1, 0, "scan_staged"), (16, 6, 2, "scan_direct"),
                                          (8, 8, 1, "scan_staged")])
def test_scan_family(m, q, mode, fam):
    assert bench.scan_family(m, q, mode) == fam


def test_traffic_record_belongs_to_its_workload(tmp_path, monkeypatch):
    """A launch's DRAM bytes depend on its text, so a workload only reads its
    own record; a record taken on other kernel sources reads as None."""
    import hashlib
    import json
    import os
    root = tmp_path
    (root / "profiles").mkdir()
    for name in bench.KERNEL_SOURCES:
        os.makedirs(root / os.path.dirname(name), exist_ok=True)
        (root / name).write_bytes(b"kernel " + name.encode())
    h = hashlib.sha256()
    for name in bench.KERNEL_SOURCES:
        h.update((root / name).read_bytes())
    rec = {"source_sha": h.hexdigest()[:16],
           "scan_staged": {"dram_bytes_per_launch": 100, "case": "sweep"},
           "skewed": {"scan_staged": {"dram_bytes_per_launch": 400, "case": "skewed"}}}
    (root / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.recorded_traffic("scan_staged")[0] == 100
    assert bench.recorded_traffic("scan_staged", "skewed")[0] == 400
    assert bench.recorded_traffic("scan_dense", "skewed") == (None, None)
    assert bench.recorded_traffic("scan_dense") == (None, None)
    rec["source_sha"] = "0" * 16
    (root / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert bench.recorded_traffic("scan_staged") == (None, None)


def test_dense_single_pass_rule_matches_the_planner():
    """The bench counts a dense search's bytes as one pass (text + one write
    per position) exactly when the library's planner picks its single-pass
    kernel: single pass asked for, within the tile and shared-memory limits;
    otherwise (the automatic choice) the spill form."""
    import paper_2310_15711_gb300 as hc
    import bench
    assert not bench.dense_single_pass(None, 4)                               # automatic: spill form
    assert not bench.dense_single_pass(hc.SearchOpts(lane_bytes=8), 8)
    assert bench.dense_single_pass(hc.SearchOpts(lane_bytes=8, single_pass=1), 8)
    assert bench.dense_single_pass(hc.SearchOpts(lane_bytes=1, tile_steps=1, single_pass=1), 2)
    assert not bench.dense_single_pass(hc.SearchOpts(single_pass=-1), 4)
    assert not bench.dense_single_pass(hc.SearchOpts(lane_bytes=256, single_pass=1), 4)   # 128 steps per chunk
    assert not bench.dense_single_pass(hc.SearchOpts(lane_bytes=64, tile_steps=64, single_pass=1), 4)  # too big
    assert bench.dense_single_pass(hc.SearchOpts(lane_bytes=16, tile_steps=64, single_pass=1), 4)


def test_stored_tuner_table_only_on_gb300():
    """The committed GB300 tables are the default only on a GB300 and only
    for the workloads they were measured for; --retune calibrates afresh."""
    import bench
    p = bench.stored_tuner_table("sweep", "NVIDIA GB300", False)
    assert p is not None and p.endswith("profiles/tuner_sweep_gb300.txt")
    assert bench.stored_tuner_table("skewed", "NVIDIA GB300", False).endswith("tuner_skewed_gb300.txt")
    assert bench.stored_tuner_table("sweep", "NVIDIA B200", False) is None
    assert bench.stored_tuner_table("sweep", "NVIDIA GB300", True) is None
    assert bench.stored_tuner_table("batched", "NVIDIA GB300", False).endswith("tuner_batched_gb300.txt")
    assert bench.stored_tuner_table("served", "NVIDIA GB300", False) is None


def test_direct_cell_traffic_needs_the_same_launch(tmp_path, monkeypatch):
    """A direct-scan cell's recorded DRAM bytes are used only for the same
    q, alpha, lane_bytes and mode, on the kernel sources they were taken on."""
    import hashlib
    import json
    import os
    root = tmp_path
    (root / "profiles").mkdir()
    for name in bench.KERNEL_SOURCES:
        os.makedirs(root / os.path.dirname(name), exist_ok=True)
        (root / name).write_bytes(b"src " + name.encode())
    h = hashlib.sha256()
    for name in bench.KERNEL_SOURCES:
        h.update((root / name).read_bytes())
    rec = {"source_sha": h.hexdigest()[:16],
           "direct_cells": {"s4_m1024": {"q": 8, "alpha": 12, "lane_bytes": 2036, "mode": 2,
                                         "dram_bytes_per_launch": 37_000_000}}}
    (root / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.recorded_cell_traffic("s4_m1024", 8, 12, 2036, 2) == 37_000_000
    assert bench.recorded_cell_traffic("s4_m1024", 8, 11, 2036, 2) is None   # other alpha
    assert bench.recorded_cell_traffic("s4_m512", 8, 12, 2036, 2) is None    # no record
    assert bench.recorded_cell_traffic("s4_m1024", 8, 12, 2036, 2, "skewed") is None
    rec["source_sha"] = "1" * 16
    (root / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert bench.recorded_cell_traffic("s4_m1024", 8, 12, 2036, 2) is None
