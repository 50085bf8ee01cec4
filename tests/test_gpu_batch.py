"""GPU parity of the batched search (hc_batch_*): every query's positions and
count equal the oracle's, the device-built filters equal the oracle's F and
H_v word for word, repeated runs and a CUDA-graph replay give the same
results, and degenerate queries (n < m, n = m, cap below the count, no
position buffer) behave as in the single search."""
import numpy as np
import pytest

import hc_inputs as hi
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_15711_gb300 as hc
    hc.build()
    hc.lib()
    return hc


def _make_queries(rng, count, n_max=300_000):
    qs = []
    for i in range(count):
        sigma = int(rng.choice([1, 2, 4, 20, 95]))
        m = int(rng.choice([1, 2, 3, 4, 8, 13, 16, 31, 64, 150, 300, 512, 2000]))
        n = int(rng.integers(0, n_max)) if i % 5 else int(rng.integers(0, 3 * m + 2))
        q = int(rng.integers(1, min(m, 8) + 1))
        alpha = int(rng.choice([3, 8, 11, 12, 13]))
        y = (rng.integers(0, sigma, n, dtype=np.uint16) + 65).astype(np.uint8)
        x = (rng.integers(0, sigma, m, dtype=np.uint16) + 65).astype(np.uint8)
        for _ in range(int(rng.integers(0, 20))):
            if n >= m:
                off = int(rng.integers(0, n - m + 1))
                y[off:off + m] = x
        qs.append(dict(x=x, y=y, q=q, alpha=alpha, mode=int(rng.choice([0, 0, 1, 2])),
                       lane_bytes=int(rng.choice([0, 0, 0, 7, 64]))))
    return qs


def _device_queries(qs, cap_fn):
    out = []
    for d in qs:
        want = oracle.hc_search(d["x"], d["y"], d["q"], d["alpha"])
        cap = cap_fn(want.size)
        y_buf = torch.empty(d["y"].size + 16, dtype=torch.uint8, device="cuda")
        off = int(d["y"].size % 7)
        y_dev = y_buf[off:off + d["y"].size]
        if d["y"].size:
            y_dev.copy_(torch.from_numpy(d["y"]))
        e = dict(x_dev=torch.from_numpy(d["x"]).cuda(), y_dev=y_dev, q=d["q"], alpha=d["alpha"],
                 pos_dev=torch.full((cap,), -1, dtype=torch.int64, device="cuda") if cap else None,
                 count_dev=torch.full((1,), -1, dtype=torch.int64, device="cuda"),
                 mode=d["mode"], lane_bytes=d["lane_bytes"], _buf=y_buf, _want=want, _cap=cap)
        out.append(e)
    return out


def _check(dq):
    for i, e in enumerate(dq):
        want = e["_want"]
        assert int(e["count_dev"].item()) == want.size, i
        k = min(e["_cap"], want.size)
        if k:
            got = e["pos_dev"][:k].cpu().numpy().view(np.uint64)
            assert np.array_equal(got, want[:k]), i
        if e["_cap"] > want.size:
            assert int(e["pos_dev"][want.size].item()) == -1, i


def test_batch_equals_oracle_and_repeats(hc):
    rng = np.random.default_rng(2)
    qs = _make_queries(rng, 60)
    dq = _device_queries(qs, lambda c: c + 3)
    b = hc.hc_batch_create(dq)
    info = b.info()
    assert info["tiles"] >= 1
    for rep in range(2):
        for e in dq:
            e["count_dev"].fill_(-1)
        b.run()
        torch.cuda.synchronize()
        hc.hc_check_status()
        _check(dq)
    # filters built on the device equal the oracle's, word for word
    for i, d in enumerate(qs):
        if d["y"].size < d["x"].size:
            continue
        F, hv = b.filter(i, d["alpha"])
        ref = oracle.preprocess(d["x"], d["q"], d["alpha"])
        assert np.array_equal(F, ref["F"]), i
        assert hv == ref["hv"], i
    b.destroy()


def test_batch_capacity_and_count_only(hc):
    rng = np.random.default_rng(3)
    qs = _make_queries(rng, 30)
    dq = _device_queries(qs, lambda c: c // 2)   # cap below the count (0 -> no buffer)
    b = hc.hc_batch_create(dq)
    b.run()
    torch.cuda.synchronize()
    hc.hc_check_status()
    _check(dq)
    b.destroy()


def test_batch_graph_replay(hc):
    rng = np.random.default_rng(4)
    qs = _make_queries(rng, 40)
    dq = _device_queries(qs, lambda c: c + 1)
    b = hc.hc_batch_create(dq)
    s = torch.cuda.Stream()
    b.run(stream=s)                     # warm-up outside the capture
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.run(stream=s)
    for rep in range(3):
        for e in dq:
            e["count_dev"].fill_(-1)
            if e["pos_dev"] is not None:
                e["pos_dev"].fill_(-1)
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        hc.hc_check_status()
        _check(dq)
    b.destroy()


def test_batch_matches_single_search_on_workload_recipe(hc):
    """A scaled-down batched workload (the recipe's distributions with
    n up to 4 MiB): each query equals the single search and the oracle."""
    qrs = hi.batch_queries(64, seed=9, n_hi=4 << 20)
    qs = []
    for qr in qrs:
        x, y = hi.query_inputs(qr)
        qs.append(dict(x=x, y=y, q=qr.q, alpha=qr.alpha, mode=0, lane_bytes=0))
    dq = _device_queries(qs, lambda c: c + 1)
    b = hc.hc_batch_create(dq)
    b.run()
    torch.cuda.synchronize()
    hc.hc_check_status()
    _check(dq)
    b.destroy()


def test_batch_outputs_in_one_shared_buffer(hc):
    """All queries write into slices of one int64 buffer at arbitrary element
    offsets (8-byte but not 16-byte aligned), as a server packing outputs
    would: results equal the oracle and the gaps between slices stay intact."""
    rng = np.random.default_rng(5)
    qs = _make_queries(rng, 40)
    wants = [oracle.hc_search(d["x"], d["y"], d["q"], d["alpha"]) for d in qs]
    offs = [0]
    for w in wants:
        offs.append(offs[-1] + w.size + 1 + int(rng.integers(0, 3)))
    big = torch.full((offs[-1] + 2,), -5, dtype=torch.int64, device="cuda")
    counts = torch.full((2 * len(qs) + 1,), -5, dtype=torch.int64, device="cuda")
    dq = []
    for i, d in enumerate(qs):
        y_dev = torch.from_numpy(d["y"]).cuda() if d["y"].size else torch.empty(0, dtype=torch.uint8,
                                                                                  device="cuda")
        dq.append(dict(x_dev=torch.from_numpy(d["x"]).cuda(), y_dev=y_dev, q=d["q"],
                       alpha=d["alpha"], pos_dev=big[offs[i] + 1:offs[i] + 1 + wants[i].size],
                       count_dev=counts[2 * i + 1:2 * i + 2], mode=d["mode"],
                       lane_bytes=d["lane_bytes"]))
    b = hc.hc_batch_create(dq)
    b.run()
    torch.cuda.synchronize()
    hc.hc_check_status()
    got = big.cpu().numpy()
    cg = counts.cpu().numpy()
    for i, w in enumerate(wants):
        assert cg[2 * i + 1] == w.size, i
        assert np.array_equal(got[offs[i] + 1:offs[i] + 1 + w.size].view(np.uint64), w), i
        assert got[offs[i]] == -5 and cg[2 * i] == -5, i
    b.destroy()


def test_batch_rejects_bad_query(hc):
    x = torch.zeros(4, dtype=torch.uint8, device="cuda")
    y = torch.zeros(100, dtype=torch.uint8, device="cuda")
    c = torch.zeros(1, dtype=torch.int64, device="cuda")
    raw = torch.zeros(64, dtype=torch.uint8, device="cuda")
    for bad in (dict(q=5), dict(q=2, count_dev=raw[4:12]), dict(q=2, pos_dev=raw[2:34], cap=4)):
        qd = dict(x_dev=x, y_dev=y, q=2, alpha=10, pos_dev=None, count_dev=c)
        qd.update(bad)
        with pytest.raises(hc.HCError) as ei:
            hc.hc_batch_create([qd])
        assert ei.value.code == hc.HC_ERR_ARG


def test_tuner_calibration_and_tuned_batch(hc):
    """Calibrate a small table on the device, then run q = 0 queries whose
    alphabet size is measured from their texts: each query runs with the
    tuned cell of its alphabet, its filter equals the oracle's for those
    parameters, and its positions equal the oracle's."""
    t = hc.HCTuner()
    t.calibrate([4, 95], [8, 64], text_bytes=8 << 20, seed=3)
    ent = t.entries()
    assert [(e["sigma"], e["m"]) for e in ent] == [(4, 8), (4, 64), (95, 8), (95, 64)]
    for e in ent:
        assert 1 <= e["q"] <= min(8, e["m"]) and 8 <= e["alpha"] <= 13, e
        assert e["mode"] in (1, 2) and 1 <= e["lane_bytes"] <= 4096 and e["gbps"] > 0, e
    rng = np.random.default_rng(12)
    qs, dq = [], []
    for i in range(24):
        sigma = 4 if i % 2 else 95
        n = int(rng.integers(5000, 400_000))
        m = int(rng.choice([5, 8, 13, 40, 64, 100]))
        y = hi.uniform_text(n, sigma, seed=50 + i)
        x, _ = hi.extract_pattern(y, m, rng)
        want = oracle.naive_search(x, y)
        qs.append((x, y, sigma, want))
        dq.append(dict(x_dev=torch.from_numpy(x).cuda(), y_dev=torch.from_numpy(y).cuda(), q=0,
                       sigma=0 if i % 3 else sigma,
                       pos_dev=torch.full((want.size + 2,), -1, dtype=torch.int64, device="cuda"),
                       count_dev=torch.full((1,), -1, dtype=torch.int64, device="cuda")))
    b = hc.hc_batch_create_tuned(dq, t)
    b.run()
    torch.cuda.synchronize()
    hc.hc_check_status()
    for i, (x, y, sigma, want) in enumerate(qs):
        p = b.params(i)
        tuned = t.lookup(sigma, x.size)
        assert (p["q"], p["alpha"]) == (tuned["q"], tuned["alpha"]), (i, p, tuned)
        assert int(dq[i]["count_dev"].item()) == want.size, i
        got = dq[i]["pos_dev"][:want.size].cpu().numpy().view(np.uint64)
        assert np.array_equal(got, want), i
        F, hv = b.filter(i, p["alpha"])
        ref = oracle.preprocess(x, p["q"], p["alpha"])
        assert np.array_equal(F, ref["F"]) and hv == ref["hv"], i
    b.destroy()
    # without a tuner, q = 0 takes the paper's choice
    b = hc.hc_batch_create(dq)
    for i, (x, y, sigma, want) in enumerate(qs):
        assert (b.params(i)["q"], b.params(i)["alpha"]) == hi.paper_q_alpha(sigma, x.size), i
    b.destroy()
    t.free()


def test_tuner_single_search_path(hc):
    """Calibration on the single-search kernels (dense form included for
    m = q); searches run with the tuned (q, alpha, lane_bytes, mode) equal
    the oracle."""
    t = hc.HCTuner()
    t.calibrate([2, 20], [2, 8, 40], text_bytes=4 << 20, seed=5, path=hc.HC_TUNE_SINGLE)
    ent = t.entries()
    assert [(e["sigma"], e["m"]) for e in ent] == [(2, 2), (2, 8), (2, 40), (20, 2), (20, 8), (20, 40)]
    for e in ent:
        assert 1 <= e["q"] <= min(8, e["m"]) and e["gbps"] > 0, e
        assert e["mode"] in (1, 2, 3) and (e["mode"] != 3 or e["q"] == e["m"]), e
    rng = np.random.default_rng(21)
    for sigma in (2, 20):
        y = hi.uniform_text(700_001, sigma, seed=60 + sigma)
        y_dev = torch.from_numpy(y).cuda()
        for m in (2, 8, 40, 17):
            x, _ = hi.extract_pattern(y, m, rng)
            e = t.lookup(sigma, m)
            want = oracle.hc_search(x, y, e["q"], e["alpha"])
            f = hc.hc_preprocess(x, e["q"], e["alpha"])
            pos = torch.full((want.size + 1,), -1, dtype=torch.int64, device="cuda")
            cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
            hc.hc_search_ex(f, y_dev, pos, cnt, hc.SearchOpts(lane_bytes=e["lane_bytes"], mode=e["mode"]))
            torch.cuda.synchronize()
            hc.hc_check_status()
            assert int(cnt.item()) == want.size, (sigma, m, e)
            assert np.array_equal(pos[:want.size].cpu().numpy().view(np.uint64), want), (sigma, m, e)
            f.free()
    t.free()
