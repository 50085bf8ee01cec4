"""GPU parity: the CUDA search (through the C ABI) against the oracle.

Positions must agree bit for bit (sorted occurrence lists, uint64).  Cases
span several chunks with ragged tails, every q, alpha from 1 to 15, unaligned
text pointers, degenerate inputs (n < m, n == m, sigma = 1, m = q, m = 1,
alpha < q), more occurrences than the per-thread slots hold, the unstaged
kernel for very long patterns, the capacity error, and the full-size
workloads (256 MiB sweep texts, the 1 GiB order-2 Markov text) compared in
full against the oracle's HC.
"""
import numpy as np
import pytest

import hc_inputs as hi
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_15711_gb300 as hc
    hc.build()
    hc.lib()
    return hc


def _hc():
    import paper_2310_15711_gb300 as hc
    return hc


def _upload(y: np.ndarray, offset: int = 0):
    n = y.size
    buf = torch.empty(n + offset + 32, dtype=torch.uint8, device="cuda")
    if n:
        buf[offset:offset + n].copy_(torch.from_numpy(np.require(y, requirements=["C", "W"])))
    return buf[offset:offset + n], buf


def gpu_positions(x, y, q, alpha, offset=0):
    hc = _hc()
    y_dev, keep = _upload(np.asarray(y, dtype=np.uint8), offset)
    f = hc.hc_preprocess(x, q, alpha)
    pos = hc.search_positions(f, x, y_dev)
    out = pos.cpu().numpy().view(np.uint64).copy()
    f.free()
    del keep
    return out


def _case(rng, sigma, n, m, plant):
    y = (rng.integers(0, sigma, n, dtype=np.uint16) + 65).astype(np.uint8)
    x = (rng.integers(0, sigma, m, dtype=np.uint16) + 65).astype(np.uint8)
    if n >= m:
        for _ in range(plant):
            off = int(rng.integers(0, n - m + 1))
            y[off:off + m] = x
    return x, y


def test_config_one_exact():
    c = hi.config_one()
    got = gpu_positions(c["x"], c["y"], c["q"], c["alpha"])
    want = oracle.hc_search(c["x"], c["y"], c["q"], c["alpha"])
    assert np.array_equal(got, want)
    assert np.array_equal(want, oracle.naive_search(c["x"], c["y"]))
    assert c["offset"] in set(got.tolist())


@pytest.mark.parametrize("sigma", [1, 2, 4, 20, 95])
def test_random_cases_all_q(sigma):
    rng = np.random.default_rng(1000 + sigma)
    ms = [1, 2, 3, 4, 5, 7, 8, 9, 15, 16, 17, 31, 32, 33, 64, 100, 255, 256, 1000, 1024, 2047]
    for trial in range(70):
        m = int(rng.choice(ms))
        q = int(rng.integers(1, min(m, 8) + 1))
        alpha = int(rng.choice([1, 3, 4, 8, 11, 12, 13, 15]))
        n = int(rng.integers(0, 200_000)) if trial % 3 else int(rng.integers(0, 3000))
        x, y = _case(rng, sigma, n, m, plant=int(rng.integers(0, 40)))
        offset = int(rng.integers(0, 16))
        got = gpu_positions(x, y, q, alpha, offset)
        want = oracle.hc_search(x, y, q, alpha)
        assert np.array_equal(got, want), (sigma, m, q, alpha, n, offset)


def test_degenerate_inputs():
    cases = [
        (b"A", b""), (b"ABC", b"AB"), (b"ABC", b"ABC"), (b"ABC", b"ABD"),
        (b"A", b"A" * 100_000),                  # m = 1, every position
        (b"AAAA", b"A" * 300_001),               # overlapping, slot overflow
        (b"AB" * 8, b"AB" * 100_000),            # periodic
        (b"GATTACA", b"GATTACA" + b"C" * 70_000 + b"GATTACA"),
    ]
    for x, y in cases:
        x = np.frombuffer(x, np.uint8)
        y = np.frombuffer(y, np.uint8)
        want = oracle.naive_search(x, y)
        for q in sorted({1, min(2, x.size), min(4, x.size), min(8, x.size)}):
            for alpha in (2, 8, 12):
                for off in (0, 5):
                    got = gpu_positions(x, y, q, alpha, off)
                    assert np.array_equal(got, want), (bytes(x[:8]), y.size, q, alpha, off)


def test_every_q_alpha_pair():
    """All 8 x 15 (q, alpha) pairs: s = floor(alpha/q) covers every byte
    grouping of the hash, including s = 0 and s >= 8."""
    rng = np.random.default_rng(88)
    for sigma in (4, 95):
        x, y = _case(rng, sigma, 60_000, 9, plant=20)
        for q in range(1, 9):
            for alpha in range(1, 16):
                got = gpu_positions(x, y, q, alpha)
                assert np.array_equal(got, oracle.hc_search(x, y, q, alpha)), (sigma, q, alpha)
        xq = x[:4]
        for alpha in range(1, 16):          # m = q = 4: the dense kernel
            assert np.array_equal(gpu_positions(xq, y, 4, alpha), oracle.naive_search(xq, y))


def test_alpha_below_q_and_large_alpha():
    rng = np.random.default_rng(77)
    x, y = _case(rng, 4, 500_000, 24, plant=30)
    for q, alpha in [(8, 3), (7, 1), (6, 15), (1, 15), (3, 14)]:
        assert np.array_equal(gpu_positions(x, y, q, alpha), oracle.hc_search(x, y, q, alpha))


def test_very_long_pattern_unstaged_kernel():
    rng = np.random.default_rng(5)
    x, y = _case(rng, 4, 2_000_000, 20_000, plant=7)
    for q in (4, 8):
        got = gpu_positions(x, y, q, 12, offset=3)
        assert np.array_equal(got, oracle.naive_search(x, y))
        assert got.size >= 1


def test_capacity_error_writes_prefix():
    hc = _hc()
    x = np.frombuffer(b"AA", np.uint8)
    y = np.frombuffer(b"A" * 10_000, np.uint8)
    y_dev, keep = _upload(y)
    f = hc.hc_preprocess(x, 2, 10)
    pos = torch.zeros(100, dtype=torch.int64, device="cuda")
    with pytest.raises(hc.HCError) as ei:
        hc.hc_search(f, x, y_dev, pos, 100)
    assert ei.value.code == hc.HC_ERR_CAPACITY
    assert pos.cpu().numpy().tolist() == list(range(100))
    assert hc.hc_search(f, x, y_dev, None, 0, allow_truncated=True) == 9_999
    with pytest.raises(hc.HCError) as ei:
        hc.hc_search(f, b"AB", y_dev, None, 0)     # not the filter's pattern
    assert ei.value.code == hc.HC_ERR_ARG


def test_async_entry_point_and_count():
    hc = _hc()
    rng = np.random.default_rng(9)
    x, y = _case(rng, 20, 3_000_000, 12, plant=100)
    y_dev, keep = _upload(y)
    f = hc.hc_preprocess(x, 3, 11)
    want = oracle.hc_search(x, y, 3, 11)
    pos = torch.full((want.size + 10,), -1, dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        hc.hc_search_async(f, y_dev, pos, cnt, stream=s)
    s.synchronize()
    hc.hc_check_status(s)
    assert int(cnt.item()) == want.size
    assert np.array_equal(pos[:want.size].cpu().numpy().view(np.uint64), want)
    assert int(pos[want.size].item()) == -1     # nothing written past the count


@pytest.mark.parametrize("opts", [
    dict(spill_entries=1), dict(spill_entries=100), dict(lane_bytes=4, stages=2),
    dict(lane_bytes=37, stages=4), dict(lane_bytes=1000, stages=2, ctas_per_sm=1),
    dict(lane_bytes=260, spill_entries=5000), dict(mode=1, lane_bytes=68),
    dict(mode=2), dict(mode=2, lane_bytes=3001, spill_entries=77), dict(mode=2, lane_bytes=8),
    dict(speculate=1), dict(speculate=1, mode=2), dict(speculate=-1),
    dict(speculate=1, spill_entries=3), dict(speculate=1, lane_bytes=5, stages=4)])
def test_launch_options_and_spill_overflow(opts):
    """Every launch shape gives the same positions, including spill regions
    too small for the occurrences (the emit kernel re-scans those chunks)."""
    hc = _hc()
    rng = np.random.default_rng(31)
    for sigma, m, n in [(2, 3, 700_001), (4, 8, 1_500_000), (20, 2, 333_333), (1, 5, 100_000)]:
        x, y = _case(rng, sigma, n, m, plant=50)
        q, alpha = min(m, 3), 11
        want = oracle.hc_search(x, y, q, alpha)
        y_dev, keep = _upload(y, offset=int(rng.integers(0, 16)))
        f = hc.hc_preprocess(x, q, alpha)
        for cap in (want.size + 3, max(want.size // 3, 1)):
            pos = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
            cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
            hc.hc_search_ex(f, y_dev, pos, cnt, hc.SearchOpts(**opts))
            torch.cuda.synchronize()
            hc.hc_check_status()
            assert int(cnt.item()) == want.size, (sigma, m, opts)
            k = min(cap, want.size)
            got = pos[:k].cpu().numpy().view(np.uint64)
            assert np.array_equal(got, want[:k]), (sigma, m, opts, cap)
        f.free()


@pytest.mark.parametrize("opts", [
    dict(mode=3), dict(mode=3, lane_bytes=1), dict(mode=3, lane_bytes=24, stages=2),
    dict(mode=3, lane_bytes=33, spill_entries=10), dict(mode=3, spill_entries=1),
    dict(mode=3, lane_bytes=5, ctas_per_sm=1, stages=3),
    dict(mode=3, single_pass=-1), dict(mode=3, single_pass=-1, lane_bytes=1),
    dict(mode=3, single_pass=-1, lane_bytes=33, spill_entries=10),
    dict(mode=3, single_pass=-1, spill_entries=1, stages=3)])
def test_dense_mode_m_equals_q(opts):
    """m = q: the warp-cooperative kernels against the oracle, for every q:
    the single-pass form (the default) and the spill-and-emit form."""
    hc = _hc()
    rng = np.random.default_rng(41)
    for sigma, m, n in [(2, 2, 1_000_003), (4, 4, 600_000), (20, 3, 250_001), (1, 5, 70_000),
                        (95, 8, 400_000), (2, 1, 100_000), (3, 6, 500_000), (4, 7, 123_457)]:
        x, y = _case(rng, sigma, n, m, plant=40)
        want = oracle.hc_search(x, y, m, 12)
        y_dev, keep = _upload(y, offset=int(rng.integers(0, 16)))
        f = hc.hc_preprocess(x, m, 12)
        for cap in (want.size + 1, max(want.size // 2, 1)):
            pos = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
            cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
            hc.hc_search_ex(f, y_dev, pos, cnt, hc.SearchOpts(**opts))
            torch.cuda.synchronize()
            hc.hc_check_status()
            assert int(cnt.item()) == want.size, (sigma, m, opts)
            k = min(cap, want.size)
            assert np.array_equal(pos[:k].cpu().numpy().view(np.uint64), want[:k]), (sigma, m, opts)
        f.free()


@pytest.mark.parametrize("opts", [
    dict(single_pass=1), dict(single_pass=1, tile_steps=1, lane_bytes=2),
    dict(single_pass=1, tile_steps=3, lane_bytes=2, stages=4),
    dict(single_pass=1, tile_steps=64, lane_bytes=4), dict(single_pass=1, lane_bytes=7, stages=3),
    dict(single_pass=1, ctas_per_sm=1, tile_steps=2), dict(single_pass=1, pos32=1, tile_steps=1, lane_bytes=2),
    dict(single_pass=1, lane_bytes=16, tile_steps=64)])
def test_dense_single_pass_tiles_and_edges(opts):
    """The single-pass dense scan: tiles of 1 to 64 steps (many tiles, so
    the look-back crosses many descriptors and several rounds of 32), texts
    from one window to a few MB at every 16-byte offset, every window a
    match (sigma = 1), capacities from 0 to above the count; the count is
    exact and the first min(count, cap) positions equal the oracle's, with
    nothing written past them."""
    hc = _hc()
    rng = np.random.default_rng(4242)
    opts = dict(opts, mode=3)
    pos32 = opts.get("pos32", 0) == 1
    cases = [(1, 1, 1), (1, 3, 3), (2, 2, 2), (4, 4, 5), (1, 2, 511), (2, 1, 513), (4, 3, 4096),
             (1, 4, 70_001), (2, 2, 1_000_003), (4, 5, 777_777), (20, 6, 300_000), (95, 8, 2_500_001),
             (4, 7, 123_457), (3, 8, 600_000), (2, 1, 3_000_001)]
    for i, (sigma, m, n) in enumerate(cases):
        x, y = _case(rng, sigma, n, m, plant=int(rng.integers(0, 60)))
        want = oracle.hc_search(x, y, m, 12)
        offset = i % 16
        y_dev, keep = _upload(y, offset=offset)
        f = hc.hc_preprocess(x, m, 12)
        for cap in sorted({0, 1, want.size // 2, want.size, want.size + 2}):
            dt = torch.int32 if pos32 else torch.int64
            buf = torch.full((cap + 2,), -7, dtype=dt, device="cuda")
            pos = buf[1:1 + cap] if cap else None
            cnt = torch.full((1,), -5, dtype=torch.int64, device="cuda")
            hc.hc_search_ex(f, y_dev, pos, cnt, hc.SearchOpts(**opts), cap=cap)
            torch.cuda.synchronize()
            hc.hc_check_status()
            assert int(cnt.item()) == want.size, (sigma, m, n, offset, opts, cap)
            k = min(cap, want.size)
            got = buf.cpu().numpy()
            vals = got[1:1 + k].view(np.uint32).astype(np.uint64) if pos32 else got[1:1 + k].view(np.uint64)
            assert np.array_equal(vals, want[:k]), (sigma, m, n, offset, opts, cap)
            assert got[0] == -7 and (got[1 + k:] == -7).all(), (sigma, m, n, offset, opts, cap)
        f.free()


@pytest.mark.parametrize("opts", [
    dict(bitmap=1), dict(bitmap=1, lane_bytes=2), dict(bitmap=1, lane_bytes=16),
    dict(bitmap=1, lane_bytes=32, pos32=1), dict(bitmap=1, lane_bytes=40), dict(bitmap=1, lane_bytes=7),
    dict(bitmap=1, pos32=1, stages=3),
])
def test_dense_bitmap_form(opts):
    """The dense scan's bitmap form (one bit per window start, expanded by
    its emit kernel): texts from one window to a few MB at every 16-byte
    offset (the lanes' windows then straddle the bitmap's 16-window groups by
    that many), every window a match (sigma = 1) and random texts, ragged
    ends, capacities from 0 to above the count; the count is exact and the
    first min(count, cap) positions equal the oracle's, nothing written past
    them."""
    hc = _hc()
    rng = np.random.default_rng(977)
    opts = dict(opts, mode=3)
    pos32 = opts.get("pos32", 0) == 1
    cases = [(1, 1, 1), (1, 3, 3), (2, 2, 2), (4, 4, 5), (1, 2, 511), (2, 1, 513), (4, 3, 4096),
             (1, 4, 70_001), (2, 2, 1_000_003), (4, 5, 777_777), (20, 6, 300_000), (95, 8, 2_500_001),
             (4, 7, 123_457), (3, 8, 600_000), (2, 1, 3_000_001), (1, 1, 1_048_577), (2, 3, 16_385),
             (2, 2, 40_000_003)]
    for i, (sigma, m, n) in enumerate(cases):
        x, y = _case(rng, sigma, n, m, plant=int(rng.integers(0, 60)))
        want = oracle.hc_search(x, y, m, 12)
        offset = (i * 7) % 16
        y_dev, keep = _upload(y, offset=offset)
        f = hc.hc_preprocess(x, m, 12)
        for cap in sorted({0, 1, want.size // 3, want.size, want.size + 2}):
            dt = torch.int32 if pos32 else torch.int64
            buf = torch.full((cap + 2,), -7, dtype=dt, device="cuda")
            pos = buf[1:1 + cap] if cap else None
            cnt = torch.full((1,), -5, dtype=torch.int64, device="cuda")
            hc.hc_search_ex(f, y_dev, pos, cnt, hc.SearchOpts(**opts), cap=cap)
            torch.cuda.synchronize()
            hc.hc_check_status()
            assert int(cnt.item()) == want.size, (sigma, m, n, offset, opts, cap)
            k = min(cap, want.size)
            got = buf.cpu().numpy()
            vals = got[1:1 + k].view(np.uint32).astype(np.uint64) if pos32 else got[1:1 + k].view(np.uint64)
            assert np.array_equal(vals, want[:k]), (sigma, m, n, offset, opts, cap)
            assert got[0] == -7 and (got[1 + k:] == -7).all(), (sigma, m, n, offset, opts, cap)
        f.free()


def test_dense_bitmap_form_full_size():
    """The bitmap form on the 256 MiB sigma = 2 sweep text, m = q = 2 (a
    quarter of all windows are occurrences: 67 M positions, every emit round
    full) and sigma = 4, m = q = 4, with u32 positions, against the oracle;
    the capacity once the whole count and once about a third of it (the cut
    then falls inside some record's chunks)."""
    hc = _hc()
    for sigma, m in ((2, 2), (4, 4)):
        y = hi.sweep_text(sigma)
        x = hi.sweep_patterns(y, sigma, m, count=1)[0]
        want = oracle.hc_search(x, y, m, 8)
        y_dev = torch.from_numpy(y).cuda()
        f = hc.hc_preprocess(x, m, 8)
        for cap in (want.size, want.size // 3 + 5):
            pos = torch.full((cap + 1,), -7, dtype=torch.int32, device="cuda")
            cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
            hc.hc_search_ex(f, y_dev, pos[:cap], cnt, hc.SearchOpts(mode=3, bitmap=1, lane_bytes=16, pos32=1),
                            cap=cap)
            torch.cuda.synchronize()
            hc.hc_check_status()
            assert int(cnt.item()) == want.size
            got = pos.cpu().numpy()
            assert np.array_equal(got[:cap].view(np.uint32).astype(np.uint64), want[:cap])
            assert got[cap] == -7
        f.free()
        del y_dev


@pytest.mark.parametrize("speculate", [1, -1])
def test_speculative_and_per_lane_forms(speculate):
    """Both forms of the staged/direct scan against the oracle, for every q,
    long patterns with full-window matches and periodic texts."""
    hc = _hc()
    rng = np.random.default_rng(500 + speculate)
    for trial in range(40):
        sigma = int(rng.choice([1, 2, 4, 20, 95]))
        m = int(rng.choice([3, 5, 9, 16, 33, 100, 300, 1024]))
        q = int(rng.integers(1, min(m, 8) + 1))
        if q == m:
            q = max(1, m - 1)
        alpha = int(rng.choice([4, 8, 11, 12, 15]))
        x, y = _case(rng, sigma, int(rng.integers(1000, 400_000)), m, plant=int(rng.integers(0, 30)))
        want = oracle.hc_search(x, y, q, alpha)
        y_dev, keep = _upload(y, offset=int(rng.integers(0, 16)))
        f = hc.hc_preprocess(x, q, alpha)
        for mode in (1, 2):
            pos = torch.full((want.size + 4,), -1, dtype=torch.int64, device="cuda")
            cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
            try:
                hc.hc_search_ex(f, y_dev, pos, cnt, hc.SearchOpts(mode=mode, speculate=speculate))
            except hc.HCError as ex:      # staging buffers too large for this m, alpha
                assert mode == 1 and ex.code == hc.HC_ERR_ARG
                continue
            torch.cuda.synchronize()
            hc.hc_check_status()
            assert int(cnt.item()) == want.size, (sigma, m, q, alpha, mode)
            assert np.array_equal(pos[:want.size].cpu().numpy().view(np.uint64), want)
        f.free()


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_positions_at_8_byte_aligned_offset(mode):
    """Output buffers that are slices of a larger int64 buffer start on an
    8-byte (not 16-byte) boundary: every kernel kind writes the same
    positions there, and nothing before or after the slice is touched."""
    hc = _hc()
    rng = np.random.default_rng(61 + mode)
    m = 4 if mode == 3 else 6
    q = 4 if mode == 3 else 3
    x, y = _case(rng, 2, 900_001, m, plant=30)
    want = oracle.hc_search(x, y, q, 12)
    assert want.size > 10_000
    y_dev, keep = _upload(y, offset=3)
    f = hc.hc_preprocess(x, q, 12)
    for lead in (1, 2, 3):
        big = torch.full((want.size + 8,), -7, dtype=torch.int64, device="cuda")
        cnt_big = torch.full((3,), -7, dtype=torch.int64, device="cuda")
        pos, cnt = big[lead:lead + want.size + 1], cnt_big[1:2]
        hc.hc_search_ex(f, y_dev, pos, cnt, hc.SearchOpts(mode=mode))
        torch.cuda.synchronize()
        hc.hc_check_status()
        assert int(cnt.item()) == want.size
        got = big.cpu().numpy()
        assert np.array_equal(got[lead:lead + want.size].view(np.uint64), want), lead
        assert (got[:lead] == -7).all() and (got[lead + want.size:] == -7).all()
        assert cnt_big[0].item() == -7 and cnt_big[2].item() == -7
    f.free()


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_outputs_in_mapped_host_memory(mode):
    """Positions and counts written by the kernels straight into mapped host
    memory (hc_mapped_alloc) equal the oracle's, for every kernel kind, at an
    offset inside the buffer; slots outside the written range keep their
    values."""
    hc = _hc()
    rng = np.random.default_rng(71 + mode)
    m, q = (3, 3) if mode == 3 else (9, 4)
    x, y = _case(rng, 4, 2_000_003, m, plant=50)
    want = oracle.hc_search(x, y, q, 11)
    y_dev, keep = _upload(y, offset=5)
    f = hc.hc_preprocess(x, q, 11)
    buf = hc.MappedBuffer(want.size + 9)
    cnt = hc.MappedBuffer(3)
    buf.array()[:] = -3
    cnt.array()[:] = -3
    hc.hc_search_ex(f, y_dev, buf.view(3, want.size + 2), cnt.view(1, 1), hc.SearchOpts(mode=mode))
    torch.cuda.synchronize()
    hc.hc_check_status()
    assert int(cnt.array()[1]) == want.size and cnt.array()[0] == -3 and cnt.array()[2] == -3
    got = buf.array()
    assert np.array_equal(got[3:3 + want.size].view(np.uint64), want)
    assert (got[:3] == -3).all() and (got[3 + want.size:] == -3).all()
    buf.free()
    cnt.free()
    f.free()


def test_graph_captured_host_copies_and_searches():
    """The end-to-end usage: per text a copy from pinned host memory into one
    device buffer, then searches of every kernel kind (the dense bitmap form
    too) writing positions and counts into mapped host memory, all captured
    once in a CUDA graph and replayed twice with new host texts of the same
    sizes; every replay's counts and last positions equal the oracle's."""
    hc = _hc()
    rng = np.random.default_rng(515)
    specs = [(4, 9, 4, dict(mode=1)), (20, 700, 5, dict(mode=2)), (2, 3, 3, dict(mode=3)),
             (4, 2, 2, dict(mode=3, bitmap=1))]
    n = 3_000_017
    pinned = torch.empty(n, dtype=torch.uint8).pin_memory()
    y_dev = torch.empty(n + 16, dtype=torch.uint8, device="cuda")[3:3 + n]
    cap = 1 << 21
    pos = hc.MappedBuffer(cap)
    cnt = hc.MappedBuffer(len(specs))
    stream = torch.cuda.Stream()
    filters = []
    for sigma, m, q, opts in specs:
        x = (rng.integers(0, sigma, m, dtype=np.uint16) + 65).astype(np.uint8)
        f = hc.hc_preprocess(x, q, 11)
        f.to_device()
        filters.append((x, q, f, opts))

    def step():
        y_dev.copy_(pinned, non_blocking=True)
        for i, (x, q, f, opts) in enumerate(filters):
            hc.hc_search_ex(f, y_dev, pos.view(), cnt.view(i, 1), hc.SearchOpts(**opts), cap=cap, stream=stream)

    with torch.cuda.stream(stream):
        step()                                   # eager once (filters on the device, pool warm)
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        step()
    for rep in range(2):
        y = (rng.integers(0, 4, n, dtype=np.uint16) + 65).astype(np.uint8)
        for x, q, f, opts in filters:            # plant every pattern a few times
            for _ in range(7):
                off = int(rng.integers(0, n - x.size + 1))
                y[off:off + x.size] = x
        pinned.copy_(torch.from_numpy(y))
        cnt.array()[:] = -1
        with torch.cuda.stream(stream):
            g.replay()
        stream.synchronize()
        hc.hc_check_status(stream)
        for i, (x, q, f, opts) in enumerate(filters):
            want = oracle.hc_search(x, y, q, 11)
            assert int(cnt.array()[i]) == want.size, (rep, i)
        x, q, f, opts = filters[-1]              # the positions buffer holds the last search's
        want = oracle.hc_search(x, y, q, 11)
        k = min(want.size, cap)
        assert np.array_equal(pos.array()[:k].view(np.uint64), want[:k]), rep
    del g
    for _, _, f, _ in filters:
        f.free()
    pos.free()
    cnt.free()


@pytest.mark.parametrize("opts", [dict(pos32=1), dict(pos32=1, mode=1), dict(pos32=1, mode=2),
                                  dict(pos32=1, spill_entries=1), dict(pos32=1, mode=2, spill_entries=3)])
def test_uint32_positions(opts):
    """pos32: the same positions as uint32 values, at a 4-byte (not 8-byte)
    aligned output, through every kernel kind, re-scans of overflowed spill
    regions and capacity truncation; nothing outside the output is written."""
    hc = _hc()
    rng = np.random.default_rng(81)
    for sigma, m, q, n in [(2, 3, 3, 700_001), (4, 8, 4, 1_500_000), (20, 2, 2, 333_333), (4, 4, 4, 600_000)]:
        if opts.get("mode") in (1, 2) and m == q and m < 3:
            continue
        x, y = _case(rng, sigma, n, m, plant=50)
        want = oracle.hc_search(x, y, q, 11)
        y_dev, keep = _upload(y, offset=int(rng.integers(0, 16)))
        f = hc.hc_preprocess(x, q, 11)
        for cap in (want.size + 3, max(want.size // 3, 1)):
            buf = torch.full((cap + 6,), -7, dtype=torch.int32, device="cuda")
            pos = buf[1:1 + cap]
            cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
            hc.hc_search_ex(f, y_dev, pos, cnt, hc.SearchOpts(**opts))
            torch.cuda.synchronize()
            hc.hc_check_status()
            assert int(cnt.item()) == want.size, (sigma, m, opts)
            k = min(cap, want.size)
            got = buf.cpu().numpy()
            assert np.array_equal(got[1:1 + k].view(np.uint32).astype(np.uint64), want[:k]), (sigma, m, opts, cap)
            assert got[0] == -7 and (got[1 + k:] == -7).all()
        f.free()


def test_uint32_positions_rejected_when_misaligned_or_invalid():
    hc = _hc()
    y_dev, keep = _upload(np.frombuffer(b"ACGT" * 1000, np.uint8))
    f = hc.hc_preprocess(b"ACGTACGT", 4, 12)
    raw = torch.zeros(256, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(hc.HCError) as ei:                      # 2-byte aligned
        hc.hc_search_ex(f, y_dev, raw[2:66], cnt, hc.SearchOpts(pos32=1), cap=16)
    assert ei.value.code == hc.HC_ERR_ARG
    with pytest.raises(hc.HCError) as ei:
        hc.hc_search_ex(f, y_dev, raw[4:68], cnt, hc.SearchOpts(pos32=2), cap=16)
    assert ei.value.code == hc.HC_ERR_ARG
    hc.hc_search_ex(f, y_dev, raw[4:68], cnt, hc.SearchOpts(pos32=1), cap=16)   # 4-byte aligned: fine
    torch.cuda.synchronize()
    hc.hc_check_status()
    assert int(cnt.item()) == 999
    f.free()


def test_misaligned_output_pointers_rejected():
    """A positions or count pointer that is not 8-byte aligned is an argument
    error, reported before anything is launched."""
    hc = _hc()
    y_dev, keep = _upload(np.frombuffer(b"ACGT" * 1000, np.uint8))
    f = hc.hc_preprocess(b"ACGTACGT", 4, 12)
    raw = torch.zeros(256, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    for pos, c in ((raw[4:132], cnt), (None, raw[4:12]), (raw[1:129], cnt)):
        with pytest.raises(hc.HCError) as ei:
            hc.hc_search_async(f, y_dev, pos, c, cap=16 if pos is not None else 0)
        assert ei.value.code == hc.HC_ERR_ARG
    torch.cuda.synchronize()
    assert (raw == 0).all()
    f.free()


def test_search_opts_rejected_when_out_of_range():
    hc = _hc()
    y_dev, keep = _upload(np.frombuffer(b"ACGT" * 1000, np.uint8))
    f = hc.hc_preprocess(b"ACGTACGT", 4, 12)
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    for bad in (dict(lane_bytes=5000), dict(stages=5), dict(stages=1), dict(mode=3),
                dict(mode=7), dict(single_pass=2), dict(single_pass=-2), dict(tile_steps=65),
                dict(tile_steps=-1), dict(mode=1, single_pass=1), dict(sentinel=2),
                dict(mode=2, sentinel=1), dict(mode=3, sentinel=1), dict(bitmap=2), dict(bitmap=-1),
                dict(bitmap=1), dict(mode=1, bitmap=1), dict(mode=2, bitmap=1)):
        with pytest.raises(hc.HCError) as ei:
            hc.hc_search_ex(f, y_dev, None, cnt, hc.SearchOpts(**bad))
        assert ei.value.code == hc.HC_ERR_ARG
    # m = q: the bitmap form excludes the single pass and needs the dense mode
    f4 = hc.hc_preprocess(b"ACGT", 4, 12)
    for bad in (dict(bitmap=1, single_pass=1), dict(mode=1, bitmap=1), dict(bitmap=1, lane_bytes=300)):
        with pytest.raises(hc.HCError) as ei:
            hc.hc_search_ex(f4, y_dev, None, cnt, hc.SearchOpts(**bad))
        assert ei.value.code == hc.HC_ERR_ARG


def test_full_size_sweep_texts():
    """256 MiB sweep texts (i.i.d. uniform), patterns copied from the text,
    full comparison with the oracle's HC for a cell of each alphabet."""
    for sigma, m in [(2, 2), (4, 16), (20, 32), (95, 1024)]:
        y = hi.sweep_text(sigma)
        x = hi.sweep_patterns(y, sigma, m, count=1)[0]
        q, alpha = hi.paper_q_alpha(sigma, m)
        got = gpu_positions(x, y, q, alpha)
        want = oracle.hc_search(x, y, q, alpha)
        assert np.array_equal(got, want), (sigma, m)
        assert got.size >= 1
        del y


def test_full_size_skewed_markov_text():
    y = hi.skew_text()
    rng = np.random.default_rng(123)
    for m in (4, 16, 128):
        x, _ = hi.extract_pattern(y, m, rng)
        q, alpha = hi.paper_q_alpha(60, m)
        got = gpu_positions(x, y, q, alpha)
        want = oracle.hc_search(x, y, q, alpha)
        assert np.array_equal(got, want), m


# (sigma, m, q, alpha, lane_bytes, mode): cells of the two full-size
# workloads with the parameters and launch options the autotuner picks for
# them on GB300 (dense, staged and direct scans)
BENCH_CELLS = [(2, 2, 2, 12, 8, 3), (4, 16, 6, 12, 68, 1), (20, 32, 2, 9, 124, 1),
               (95, 1024, 3, 11, 1022, 2), (60, 8, 8, 11, 16, 3), (60, 64, 4, 10, 376, 1),
               (60, 512, 5, 12, 1016, 2)]


def test_full_size_in_the_timed_launch_configuration():
    """The full-size texts searched as the benchmark times them: the filter
    resident on the device, uint32 positions, explicit launch options, the
    search captured in a CUDA graph on a side stream and replayed twice; the
    positions equal the oracle's in full and nothing around the output is
    written."""
    hc = _hc()
    stream = torch.cuda.Stream()
    texts = {}
    for sigma, m, q, alpha, lane_bytes, mode in BENCH_CELLS:
        if sigma not in texts:
            texts.clear()
            y = hi.skew_text() if sigma == 60 else hi.sweep_text(sigma)
            texts[sigma] = (y, torch.from_numpy(y).cuda())
        y, y_dev = texts[sigma]
        x = hi.sweep_patterns(y, sigma, m, count=1)[0]
        want = oracle.hc_search(x, y, q, alpha)
        assert want.size >= 1
        f = hc.hc_preprocess(x, q, alpha)
        f.to_device()
        opts = hc.SearchOpts(lane_bytes=lane_bytes, mode=mode, pos32=1)
        buf = torch.full((want.size + 8,), -7, dtype=torch.int32, device="cuda")
        pos = buf[1:1 + want.size + 3]
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            hc.hc_search_ex(f, y_dev, pos, cnt, opts, stream=stream)   # warm-up, outside the graph
        stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            hc.hc_search_ex(f, y_dev, pos, cnt, opts, stream=stream)
        for _ in range(2):
            buf.fill_(-7)
            cnt.zero_()
            torch.cuda.synchronize()
            with torch.cuda.stream(stream):
                g.replay()
            stream.synchronize()
            hc.hc_check_status(stream)
            assert int(cnt.item()) == want.size, (sigma, m)
            got = buf.cpu().numpy()
            assert np.array_equal(got[1:1 + want.size].view(np.uint32).astype(np.uint64), want), (sigma, m)
            assert got[0] == -7 and (got[1 + want.size:] == -7).all(), (sigma, m)
        del g
        f.free()


@pytest.mark.parametrize("lane_bytes", [0, 4, 37, 188])
def test_sentinel_form_of_the_staged_scan(lane_bytes):
    """The sentinel form (SHC's idea on the GPU: the staging buffers are
    padded so that a lane's first tests run past its window starts with no
    position test per window) gives exactly the oracle's HC and SHC results
    for every q, patterns long and short, periodic and random texts, every
    16-byte offset of the text."""
    hc = _hc()
    rng = np.random.default_rng(900 + lane_bytes)
    for trial in range(36):
        sigma = int(rng.choice([1, 2, 4, 20, 95]))
        m = int(rng.choice([2, 3, 5, 9, 16, 33, 100, 180]))
        q = int(rng.integers(1, min(m, 8) + 1))
        alpha = int(rng.choice([4, 8, 11, 12, 15]))
        x, y = _case(rng, sigma, int(rng.integers(1, 300_000)), m, plant=int(rng.integers(0, 40)))
        want = oracle.hc_search(x, y, q, alpha)
        assert np.array_equal(want, oracle.shc_search(x, y, q, alpha))
        y_dev, keep = _upload(y, offset=trial % 16)
        f = hc.hc_preprocess(x, q, alpha)
        for cap in (want.size + 2, max(want.size // 2, 1)):
            pos = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
            cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
            try:
                hc.hc_search_ex(f, y_dev, pos, cnt, hc.SearchOpts(mode=1, sentinel=1, lane_bytes=lane_bytes))
            except hc.HCError as ex:      # staging buffers too large for this m, alpha
                assert ex.code == hc.HC_ERR_ARG
                break
            torch.cuda.synchronize()
            hc.hc_check_status()
            assert int(cnt.item()) == want.size, (sigma, m, q, alpha)
            k = min(cap, want.size)
            assert np.array_equal(pos[:k].cpu().numpy().view(np.uint64), want[:k]), (sigma, m, q, alpha, cap)
        f.free()
