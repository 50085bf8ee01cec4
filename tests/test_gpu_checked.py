"""The checked build (libhc_checked.so, device-side bounds checks that count
violations and skip the access): tiny and ragged cases through every kernel
kind -- staged, direct and dense scans, emit with tiny spill regions and
re-scans, capacity truncation, a mixed batch -- give the oracle's positions,
leave canary zones around every output untouched, and count no bounds
violation."""
import ctypes

import numpy as np
import pytest

import hc_inputs as hi
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CANARY = 0x5A5A5A5A5A5A5A5A   # fits in int64
GUARD = 64


@pytest.fixture(scope="module")
def hc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_15711_gb300 as hc
    from paper_2310_15711_gb300 import _build
    hc.build()
    lib_regular = hc.lib()
    L = ctypes.CDLL(_build.build(checked=True))
    for name, (res, args) in hc.SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    hc._lib = L
    yield hc
    hc._lib = lib_regular


def _violations(hc):
    v = ctypes.c_uint64()
    hc._check(hc.lib().hc_check_bounds(ctypes.byref(v)), "hc_check_bounds")
    return v.value


def _guarded(n):
    buf = torch.full((n + 2 * GUARD,), CANARY, dtype=torch.int64, device="cuda")
    return buf, buf[GUARD:GUARD + n]


def _intact(buf, n):
    h = buf.cpu().numpy()
    return (h[:GUARD] == CANARY).all() and (h[GUARD + n:] == CANARY).all()


def test_single_search_kinds_checked(hc):
    assert _violations(hc) == 0
    rng = np.random.default_rng(77)
    cases = 0
    for trial in range(60):
        sigma = int(rng.choice([1, 2, 4, 20, 95]))
        m = int(rng.choice([1, 2, 3, 4, 7, 8, 13, 16, 33, 100, 250, 700]))
        n = int(rng.integers(0, 40_000)) if trial % 3 else int(rng.integers(m, m + 70))
        q = int(rng.integers(1, min(m, 8) + 1))
        alpha = int(rng.choice([3, 8, 11, 12, 13]))
        y = (rng.integers(0, sigma, n, dtype=np.uint16) + 65).astype(np.uint8)
        x = (rng.integers(0, sigma, m, dtype=np.uint16) + 65).astype(np.uint8)
        for _ in range(int(rng.integers(0, 12))):
            if n >= m:
                o = int(rng.integers(0, n - m + 1))
                y[o:o + m] = x
        want = oracle.naive_search(x, y)
        off = int(rng.integers(0, 16))
        ybuf = torch.empty(n + off + 64, dtype=torch.uint8, device="cuda")
        if n:
            ybuf[off:off + n].copy_(torch.from_numpy(y))
        y_dev = ybuf[off:off + n]
        f = hc.hc_preprocess(x, q, alpha)
        modes = [0, 1, 2] + ([3] if m == q else [])
        forms = [dict(mode=mode, spill_entries=spill) for mode in modes for spill in (0, 1)]
        if m == q:
            forms.append(dict(mode=3, bitmap=1, lane_bytes=int(rng.choice([2, 8, 16]))))
        for form in forms:
            mode = form["mode"]
            for cap in (want.size + 2, max(1, want.size // 2)):
                pbuf, pos = _guarded(cap)
                cbuf, cnt = _guarded(1)
                try:
                    hc.hc_search_ex(f, y_dev, pos, cnt, hc.SearchOpts(**form))
                except hc.HCError as e:       # staged buffers too large for this m
                    assert e.code == hc.HC_ERR_ARG and mode == 1
                    continue
                torch.cuda.synchronize()
                hc.hc_check_status()
                k = min(cap, want.size)
                assert int(cnt.item()) == want.size, (sigma, m, q, alpha, form)
                assert np.array_equal(pos[:k].cpu().numpy().view(np.uint64), want[:k])
                assert _intact(pbuf, cap) and _intact(cbuf, 1), (sigma, m, form, cap)
                cases += 1
        f.free()
    assert cases > 200
    assert _violations(hc) == 0


def test_batch_checked(hc):
    rng = np.random.default_rng(78)
    dq, wants, bufs = [], [], []
    for i in range(40):
        sigma = int(rng.choice([2, 4, 20, 95]))
        m = int(rng.choice([2, 3, 5, 8, 16, 40, 200, 900]))
        n = int(rng.integers(0, 60_000))
        y = hi.uniform_text(n, sigma, seed=900 + i)
        x = (rng.integers(0, sigma, m, dtype=np.uint16) + 65).astype(np.uint8) if n < m else \
            hi.extract_pattern(y, m, rng)[0]
        want = oracle.naive_search(x, y)
        cap = want.size + 1 if i % 3 else max(1, want.size // 3)
        pbuf, pos = _guarded(cap)
        cbuf, cnt = _guarded(1)
        q = int(rng.integers(1, min(m, 8) + 1))
        dq.append(dict(x_dev=torch.from_numpy(x).cuda(), y_dev=torch.from_numpy(y).cuda() if n else
                       torch.empty(0, dtype=torch.uint8, device="cuda"),
                       q=q, alpha=int(rng.choice([8, 11, 13])), pos_dev=pos, count_dev=cnt,
                       mode=int(rng.choice([0, 1, 2])) if m - q + 1 < 200 else 2))
        wants.append((want, cap))
        bufs.append((pbuf, cbuf))
    b = hc.hc_batch_create(dq)
    b.run()
    torch.cuda.synchronize()
    hc.hc_check_status()
    for i, (want, cap) in enumerate(wants):
        k = min(cap, want.size)
        assert int(dq[i]["count_dev"].item()) == want.size, i
        assert np.array_equal(dq[i]["pos_dev"][:k].cpu().numpy().view(np.uint64), want[:k]), i
        assert _intact(bufs[i][0], cap) and _intact(bufs[i][1], 1), i
    b.destroy()
    assert _violations(hc) == 0
