"""GPU tests of the served search (hc_server_*): every result equals the
oracle's occurrence list, a request's result is the same alone and inside a
mix of other requests batched with it, admission keeps the admitted device
bytes within the limit (requests wait, never fail, unless they can never
fit), capacity truncation keeps the exact count, the plain per-launch mode
gives the same results, and queued requests are cancelled cleanly."""
import math

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


TEXTS = [(4, 1000), (4, 300_000), (20, 2_000_000), (95, 700_001), (2, 50_000), (20, 5)]


def _texts(srv, on_device=True):
    ys, ids = [], []
    for i, (sigma, n) in enumerate(TEXTS):
        y = hi.uniform_text(n, sigma, seed=700 + i)
        ys.append(y)
        if on_device and i % 2 == 0:
            t = torch.from_numpy(y).cuda()
            ids.append(srv.add_text(t, sigma=sigma if i % 4 == 0 else 0))
        else:
            ids.append(srv.add_text(y))
    return ys, ids


def _requests(ys, count, rng):
    out = []
    for _ in range(count):
        ti = int(rng.integers(0, len(ys)))
        y = ys[ti]
        m = int(round(math.exp(rng.uniform(math.log(2), math.log(1024)))))
        if y.size >= m and rng.random() < 0.9:
            off = int(rng.integers(0, y.size - m + 1))
            x = y[off:off + m].copy()
        else:
            x = (rng.integers(0, 4, m) + 65).astype(np.uint8)
        out.append((ti, x))
    return out


def _check(res, ys, reqs_by_id, cap=4096):
    for r in res:
        ti, x = reqs_by_id[r["id"]]
        want = oracle.naive_search(x, ys[ti])
        assert r["count"] == want.size, (r, x.size)
        k = min(want.size, cap)
        assert r["npos"] == k
        assert np.array_equal(r["pos"], want[:k]), r["id"]
        assert r["status"] == (0 if want.size <= cap else 2), r   # HC_OK / HC_ERR_CAPACITY


def _collect(srv, n):
    got = []
    while len(got) < n:
        got += srv.poll(4096, wait_us=200_000)
    return got


@pytest.mark.parametrize("batch_only", [0, 1])
def test_alone_equals_in_the_mix(hc, batch_only):
    """Alone, the probe runs as a batch of one (single-search kernels, or the
    batched kernels with batch_only); in the mix it shares batches."""
    srv = hc.HCServer(hc.ServerConfig(batch_only=batch_only))
    ys, ids = _texts(srv)
    rng = np.random.default_rng(1)
    probe_t = 2
    probe_x = ys[probe_t][123_456:123_456 + 12].copy()
    pid = srv.submit(ids[probe_t], probe_x)
    srv.drain()
    alone = srv.poll(16)
    assert len(alone) == 1 and alone[0]["id"] == pid
    want = oracle.naive_search(probe_x, ys[probe_t])
    assert alone[0]["count"] == want.size and np.array_equal(alone[0]["pos"], want)

    reqs = _requests(ys, 600, rng)
    for k in (7, 150, 301, 450, 599):        # the probe again, inside the stream
        reqs[k] = (probe_t, probe_x)
    arrivals = np.cumsum(rng.exponential(4e-6, len(reqs)))      # ~250k req/s: batches form
    rids = srv.replay([(ids[t], x) for t, x in reqs], arrivals)
    srv.drain()
    res = _collect(srv, len(reqs))
    by_id = dict(zip(rids, reqs))
    _check(res, ys, by_id)
    probe_res = [r for r in res if by_id[r["id"]][1] is probe_x]
    assert len(probe_res) == 5
    for r in probe_res:
        assert r["count"] == alone[0]["count"] and np.array_equal(r["pos"], alone[0]["pos"])
        assert (r["q"], r["alpha"]) == (alone[0]["q"], alone[0]["alpha"])
    st = srv.stats()
    assert st["completed"] == st["submitted"] == len(reqs) + 1
    assert st["batches"] < len(reqs) and st["max_batch"] > 1
    assert max(r["batch_size"] for r in probe_res) > 1
    for r in res:
        assert r["submit_ns"] <= r["start_ns"] <= r["done_ns"]
    srv.destroy()


def test_admission_limit_and_capacity(hc):
    ys = [hi.uniform_text(200_000, 4, seed=5), hi.uniform_text(300_000, 20, seed=6),
          hi.uniform_text(2_500_000, 4, seed=7)]
    text_bytes = sum(y.size for y in ys)
    limit = text_bytes + (3 << 20)
    srv = hc.HCServer(hc.ServerConfig(mem_limit=limit, max_batch=64))
    ids = [srv.add_text(y) for y in ys]
    with pytest.raises(hc.HCError) as ei:        # texts beyond the limit
        srv.add_text(np.zeros(4 << 20, np.uint8))
    assert ei.value.code == hc.HC_ERR_ADMISSION
    rng = np.random.default_rng(2)
    reqs, cfgs = [], []
    for i in range(120):
        ti = i % 2
        m = int(rng.choice([2, 3, 8, 40]))
        off = int(rng.integers(0, ys[ti].size - m))
        reqs.append((ti, ys[ti][off:off + m].copy()))
        cfgs.append(150_000)                      # large caps: ~600 KB of spill workspace each
    rids = [srv.submit(ids[t], x, cap=c) for (t, x), c in zip(reqs, cfgs)]
    big = srv.submit(ids[2], ys[2][:5].copy(), cap=1 << 30)   # spill ~10 MB: can never fit
    small = srv.submit(ids[0], ys[0][:2].copy(), cap=3)        # truncated
    srv.drain()
    res = _collect(srv, len(reqs) + 2)
    by_id = dict(zip(rids, reqs))
    st = srv.stats()
    assert st["peak_inflight_bytes"] <= limit - text_bytes
    assert st["admission_waits"] > 0 and st["rejected"] == 1
    for r in res:
        if r["id"] == big:
            assert r["status"] == hc.HC_ERR_ADMISSION
        elif r["id"] == small:
            want = oracle.naive_search(ys[0][:2], ys[0])
            assert r["status"] == hc.HC_ERR_CAPACITY and r["count"] == want.size
            assert np.array_equal(r["pos"], want[:3])
        else:
            t, x = by_id[r["id"]]
            want = oracle.naive_search(x, ys[t])
            assert r["status"] == 0 and r["count"] == want.size
            assert np.array_equal(r["pos"], want)
    srv.destroy()


def test_plain_mode_gives_the_same_results(hc):
    rng = np.random.default_rng(3)
    out = {}
    for plain in (0, 1):
        srv = hc.HCServer(hc.ServerConfig(plain=plain, max_inflight=2))
        ys, ids = _texts(srv, on_device=bool(plain))
        reqs = _requests(ys, 200, np.random.default_rng(4))
        rids = srv.replay([(ids[t], x) for t, x in reqs], np.arange(len(reqs)) * 2e-6)
        srv.drain()
        res = _collect(srv, len(reqs))
        by_id = dict(zip(rids, reqs))
        _check(res, ys, by_id)
        out[plain] = {rids.index(r["id"]): (r["count"], r["pos"].tobytes()) for r in res}
        srv.destroy()
    assert out[0] == out[1]
    del rng


def test_tuned_and_explicit_parameters(hc, tmp_path):
    p = str(tmp_path / "table.txt")
    with open(p, "w") as f:
        f.write("4 16 5 10 0 0 0\n4 256 3 9 0 2 0\n95 16 2 11 0 0 0\n")
    t = hc.HCTuner()
    t.load(p)
    srv = hc.HCServer(tuner=t)
    y4 = hi.uniform_text(500_000, 4, seed=8)
    y95 = hi.uniform_text(500_000, 95, seed=9)
    a, b = srv.add_text(y4), srv.add_text(y95)
    assert abs(srv.text_info(a)["sigma"] - 4) < 0.5 and abs(srv.text_info(b)["sigma"] - 95) < 8
    x16, x300 = y4[1000:1016].copy(), y4[2000:2300].copy()
    ids = [srv.submit(a, x16), srv.submit(a, x300), srv.submit(b, y95[7:23].copy()),
           srv.submit(a, x16, q=4, alpha=12)]
    srv.drain()
    res = {r["id"]: r for r in _collect(srv, 4)}
    assert (res[ids[0]]["q"], res[ids[0]]["alpha"]) == (5, 10)
    assert (res[ids[1]]["q"], res[ids[1]]["alpha"]) == (3, 9)
    assert (res[ids[2]]["q"], res[ids[2]]["alpha"]) == (2, 11)
    assert (res[ids[3]]["q"], res[ids[3]]["alpha"]) == (4, 12)
    for i, (y, x) in enumerate([(y4, x16), (y4, x300), (y95, y95[7:23]), (y4, x16)]):
        want = oracle.naive_search(x, y)
        assert res[ids[i]]["count"] == want.size and np.array_equal(res[ids[i]]["pos"], want)
    srv.destroy()
    t.free()


def test_destroy_with_queued_requests(hc):
    srv = hc.HCServer(hc.ServerConfig(max_inflight=1, max_batch=8))
    y = hi.uniform_text(4_000_000, 4, seed=10)
    tid = srv.add_text(y)
    for i in range(400):
        srv.submit(tid, y[i * 1000:i * 1000 + 3].copy())
    srv.destroy()      # running batches finish, the rest are cancelled; returns


def test_bad_requests_rejected(hc):
    srv = hc.HCServer()
    tid = srv.add_text(hi.uniform_text(1000, 4, seed=11))
    for kw in (dict(text_id=tid + 5, x=b"ACGT"), dict(text_id=tid, x=b""),
               dict(text_id=tid, x=b"ACGT", q=5, alpha=10), dict(text_id=tid, x=b"ACGT", q=2, alpha=16)):
        with pytest.raises(hc.HCError) as ei:
            srv.submit(**kw)
        assert ei.value.code == hc.HC_ERR_ARG
    assert srv.stats()["submitted"] == 0
    srv.destroy()


def _batch_text(res, ys, rids, reqs):
    text_of = dict(zip(rids, (ti for ti, _ in reqs)))
    per_batch, size_of = {}, {}
    for r in res:
        per_batch[r["batch"]] = per_batch.get(r["batch"], 0) + ys[text_of[r["id"]]].size
        size_of[r["batch"]] = r["batch_size"]
    return per_batch, size_of


def test_batches_bounded_by_text_bytes(hc):
    """Requests that arrive one by one form batches of at most max_batch_bytes
    of text (a single larger request runs alone); a backlog submitted at once
    is cut into batches of at most max(max_batch_bytes, queued text /
    max_inflight) -- several batches, on several streams.  Every result still
    equals the oracle's."""
    bound, streams = 2_000_000, 3
    srv = hc.HCServer(hc.ServerConfig(max_batch_bytes=bound, max_batch=64, max_inflight=streams))
    ys, ids = _texts(srv)
    rng = np.random.default_rng(77)
    reqs = _requests(ys, 120, rng)
    rq = [(ids[ti], x) for ti, x in reqs]
    rids = srv.replay(rq, [0.0] * len(rq))
    srv.drain()
    res = _collect(srv, len(reqs))
    _check(res, ys, dict(zip(rids, reqs)))
    per_batch, size_of = _batch_text(res, ys, rids, reqs)
    total = sum(ys[ti].size for ti, _ in reqs)
    assert all(v <= max(bound, total // streams) or size_of[b] == 1 for b, v in per_batch.items())
    assert len(per_batch) >= streams
    # arrivals spaced so that the queue stays short: the plain bound holds
    reqs2 = _requests(ys, 40, rng)
    rq2 = [(ids[ti], x) for ti, x in reqs2]
    rids2 = srv.replay(rq2, [i * 2e-3 for i in range(len(rq2))])
    srv.drain()
    res2 = _collect(srv, len(reqs2))
    _check(res2, ys, dict(zip(rids2, reqs2)))
    per_batch, size_of = _batch_text(res2, ys, rids2, reqs2)
    assert all(v <= bound or size_of[b] == 1 for b, v in per_batch.items())
    srv.destroy()
