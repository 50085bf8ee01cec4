"""Host logic of the autotuner (no GPU): the empty table gives the paper's
(q, alpha) (Tables 1-3, nearest text by alphabet size, nearest m on a log
scale, q clamped to m), lookups pick the nearest measured cell, staged launch
options that no longer fit a longer pattern fall back to automatic, and the
text format round-trips and rejects malformed lines."""
import os

import pytest

import hc_inputs as hi

pytestmark = pytest.mark.filterwarnings("ignore")


@pytest.fixture(scope="module")
def hc():
    import paper_2310_15711_gb300 as hc
    hc.build()
    hc.lib()
    return hc


def _write(path, lines):
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


@pytest.mark.parametrize("sigma", [1, 2, 4, 8, 9, 20, 40, 41, 60, 95, 255])
def test_empty_table_is_papers_choice(hc, sigma):
    t = hc.HCTuner()
    for m in [1, 2, 3, 4, 5, 7, 8, 11, 12, 16, 23, 24, 32, 45, 64, 100, 128, 181, 256, 362, 512,
              724, 1024, 1500, 4096, 100000]:
        e = t.lookup(sigma, m)
        assert (e["q"], e["alpha"]) == hi.paper_q_alpha(sigma, m), (sigma, m)
        assert e["lane_bytes"] == 0 and e["mode"] == 0
    t.free()


def test_paper_rows_at_printed_lengths(hc):
    """The printed rows themselves (Tables 1-3) at m = 8 .. 1024."""
    t = hc.HCTuner()
    for col, sigma in (("genome", 4), ("protein", 20), ("english", 95)):
        for m, qa in hi.PAPER_QALPHA[col].items():
            e = t.lookup(sigma, m)
            assert (e["q"], e["alpha"]) == qa, (col, m)
    # config one: sigma = 4, m = 16 -> (6, 12)
    e = t.lookup(4, 16)
    assert (e["q"], e["alpha"]) == (6, 12)
    t.free()


def test_nearest_cell_and_clamp(hc, tmp_path):
    p = str(tmp_path / "t.txt")
    _write(p, ["# sigma m q alpha lane_bytes mode gbps",
               "4 16 5 12 188 1 3000.5",
               "4 256 8 13 512 2 7000",
               "20 16 3 11 100 1 4000",
               "95 64 2 10 0 0 0"])
    t = hc.HCTuner()
    t.load(p)
    ent = t.entries()
    assert [(e["sigma"], e["m"]) for e in ent] == [(4, 16), (4, 256), (20, 16), (95, 64)]
    assert ent[0]["gbps"] == pytest.approx(3000.5)
    e = t.lookup(4, 20)            # nearest m of sigma 4 (log scale): 16
    assert (e["q"], e["alpha"], e["lane_bytes"], e["mode"]) == (5, 12, 188, 1)
    e = t.lookup(3.7, 200)         # sigma 4 column, m -> 256
    assert (e["q"], e["alpha"], e["lane_bytes"], e["mode"]) == (8, 13, 512, 2)
    e = t.lookup(5, 3)             # q clamped to m
    assert e["q"] == 3 and e["alpha"] == 12
    e = t.lookup(12, 16)           # log-nearest sigma of 12 is 20 (|ln 12 - ln 20| < |ln 12 - ln 4|)
    assert (e["q"], e["alpha"]) == (3, 11)
    e = t.lookup(1000, 1)          # nearest sigma 95; q clamped to m = 1
    assert (e["q"], e["alpha"]) == (1, 10)
    t.free()


def test_staged_options_fall_back_when_they_do_not_fit(hc, tmp_path):
    """A staged cell measured at m = 64 with 376 window starts per lane needs
    8 warps x 2 stages x (32 x 376 + 64) bytes of staging; for m = 20000
    (beyond the staged form's 16384) it falls back to automatic options."""
    p = str(tmp_path / "t.txt")
    _write(p, ["4 64 6 12 376 1 1"])
    t = hc.HCTuner()
    t.load(p)
    assert t.lookup(4, 64)["mode"] == 1
    e = t.lookup(4, 20000)
    assert e["mode"] == 0 and e["lane_bytes"] == 0 and e["q"] == 6
    t.free()


def test_save_load_round_trip_and_replace(hc, tmp_path):
    p = str(tmp_path / "a.txt")
    _write(p, ["4 8 4 12 0 0 1.5", "4 8 3 11 64 2 2.5", "2 1024 8 12 4096 2 9"])
    t = hc.HCTuner()
    t.load(p)                       # the later line for (4, 8) replaces the earlier
    assert len(t.entries()) == 2
    q = str(tmp_path / "b.txt")
    t.save(q)
    t2 = hc.HCTuner()
    t2.load(q)
    assert t2.entries() == t.entries()
    assert t2.lookup(4, 8)["alpha"] == 11
    t.free()
    t2.free()


def test_sentinel_column_round_trips(hc, tmp_path):
    """The optional last column marks a staged cell measured fastest in the
    sentinel form; lookups return it, files without it read 0."""
    p = str(tmp_path / "s.txt")
    _write(p, ["20 32 6 12 124 1 5.5 1", "4 16 6 12 68 1 4.5", "95 2 2 12 16 3 5 0"])
    t = hc.HCTuner()
    t.load(p)
    assert t.lookup(20, 32)["sentinel"] == 1
    assert t.lookup(4, 16)["sentinel"] == 0
    q = str(tmp_path / "s2.txt")
    t.save(q)
    t2 = hc.HCTuner()
    t2.load(q)
    assert t2.entries() == t.entries()
    assert t2.lookup(20, 32)["sentinel"] == 1
    t.free()
    t2.free()


def test_bitmap_column_round_trips(hc, tmp_path):
    """The optional ninth column marks a dense (m = q) cell measured fastest
    in the bitmap form; lookups return it at that m and drop it (with the
    dense mode) at another m; files without it read 0."""
    p = str(tmp_path / "b.txt")
    _write(p, ["2 2 2 8 16 3 2.6 0 1", "4 4 4 8 16 3 2.8 0", "20 32 6 12 124 1 5.5"])
    t = hc.HCTuner()
    t.load(p)
    assert t.lookup(2, 2)["bitmap"] == 1 and t.lookup(2, 2)["mode"] == 3
    assert t.lookup(4, 4)["bitmap"] == 0 and t.lookup(20, 32)["bitmap"] == 0
    far = t.lookup(2, 3)             # nearest cell is m = 2; q = 2 != 3, so no dense form
    assert far["bitmap"] == 0 and far["mode"] == 0
    q = str(tmp_path / "b2.txt")
    t.save(q)
    t2 = hc.HCTuner()
    t2.load(q)
    assert t2.entries() == t.entries()
    assert t2.lookup(2, 2)["bitmap"] == 1
    t.free()
    t2.free()


@pytest.mark.parametrize("bad", ["4 8 9 12 0 0 1", "4 8 4 16 0 0 1", "4 8 4 12 0 7 1", "4 8 4 12 0 3 1",
                                 "4 2 3 12 0 0 1", "0 8 4 12 0 0 1", "4 8 4 12 0 0",
                                 "4 8 4 12 5000 0 1", "garbage", "4 8 4 12 0 2 1 1", "4 8 4 12 0 1 1 2",
                                 "4 4 4 12 0 3 1 0 2", "4 8 4 12 0 1 1 0 1", "4 4 4 12 0 3 1 1 1"])
def test_malformed_lines_rejected(hc, tmp_path, bad):
    p = str(tmp_path / "bad.txt")
    _write(p, ["4 16 6 12 0 0 1", bad])
    t = hc.HCTuner()
    with pytest.raises(hc.HCError) as ei:
        t.load(p)
    assert ei.value.code == hc.HC_ERR_STATE
    assert t.entries() == []        # nothing of a rejected file is kept
    with pytest.raises(hc.HCError) as ei:
        t.load(os.path.join(str(tmp_path), "missing.txt"))
    assert ei.value.code == hc.HC_ERR_STATE
    t.free()


def test_invalid_arguments(hc):
    L = hc.lib()
    assert L.hc_tuner_lookup(None, 4.0, 0, None) == hc.HC_ERR_ARG
    t = hc.HCTuner()
    e = hc.TuneEntry()
    import ctypes
    assert L.hc_tuner_lookup(t.handle, 4.0, 0, ctypes.byref(e)) == hc.HC_ERR_ARG
    assert L.hc_tuner_entry(t.handle, 0, ctypes.byref(e)) == hc.HC_ERR_ARG
    # calibration arguments are checked before any device work
    sig = (ctypes.c_int * 1)(0)
    ms = (ctypes.c_uint64 * 1)(8)
    assert L.hc_tuner_calibrate(t.handle, sig, 1, ms, 1, 1 << 20, 1, 0, None) == hc.HC_ERR_ARG
    sig[0] = 4
    ms[0] = 0
    assert L.hc_tuner_calibrate(t.handle, sig, 1, ms, 1, 1 << 20, 1, 0, None) == hc.HC_ERR_ARG
    ms[0] = 8
    assert L.hc_tuner_calibrate(t.handle, sig, 1, ms, 1, 1 << 20, 1, 7, None) == hc.HC_ERR_ARG
    t.free()


def test_dense_cells_only_where_m_equals_q(hc, tmp_path):
    """A single-search table may hold dense cells (m = q); a lookup for
    another length falls back to automatic launch options."""
    p = str(tmp_path / "d.txt")
    _write(p, ["2 8 8 12 16 3 900"])
    t = hc.HCTuner()
    t.load(p)
    e = t.lookup(2, 8)
    assert (e["q"], e["alpha"], e["lane_bytes"], e["mode"]) == (8, 12, 16, 3)
    e = t.lookup(2, 10)            # q = 8 != m = 10: no dense form
    assert (e["q"], e["mode"], e["lane_bytes"]) == (8, 0, 0)
    e = t.lookup(2, 6)             # q clamped to 6 = m: dense is valid again but the cell's L was for m = 8
    assert e["q"] == 6
    t.free()
