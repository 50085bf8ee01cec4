"""hc_search_noalloc, the entry point for callers that cannot allocate device
memory (for instance when their own allocator plans every byte of device
memory, or on a latency-critical path that must not enter an allocator): it
must return exactly what hc_search_async returns -- and what the oracle
returns -- on two calls in a row, with the filter words, the pattern, the
text and the outputs all supplied by the caller, and without taking device
memory.

Positions are integers, so "the tolerance our tests use" is bit-exact
equality.  This file is collected last on purpose, and works both on its own
in a fresh process and after the other tests.
"""
import numpy as np
import pytest

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


def _case(rng, sigma, n, m, plant):
    y = (rng.integers(0, sigma, n, dtype=np.uint16) + 65).astype(np.uint8)
    x = (rng.integers(0, sigma, m, dtype=np.uint16) + 65).astype(np.uint8)
    for _ in range(plant):
        off = int(rng.integers(0, n - m + 1))
        y[off:off + m] = x
    return x, y


# (sigma, m, q, alpha, n): the staged, dense (m = q) and direct kernels
CASES = [(4, 16, 6, 12, 3_000_001), (2, 2, 2, 12, 1_000_000), (20, 300, 4, 12, 2_000_000),
         (95, 7, 3, 11, 777_777)]


@pytest.mark.parametrize("sigma,m,q,alpha,n", CASES)
def test_noalloc_equals_hc_search_async_two_calls(hc, sigma, m, q, alpha, n):
    rng = np.random.default_rng(sigma * 1000 + m)
    x, y = _case(rng, sigma, n, m, plant=60)
    y_dev = torch.from_numpy(y).cuda()
    f = hc.hc_preprocess(x, q, alpha)
    F, _ = f.words()
    F_dev = torch.from_numpy(F.view(np.int32)).cuda()
    x_dev = torch.from_numpy(x).cuda()

    ref_cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    cap = 400_000
    ref_pos = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
    hc.hc_search_async(f, y_dev, ref_pos, ref_cnt)
    torch.cuda.synchronize()
    hc.hc_check_status()
    count = int(ref_cnt.item())
    assert 30 <= count <= cap
    want = oracle.hc_search(x, y, q, alpha)
    assert want.size == count

    free_after = []
    for call in range(2):
        pos = torch.full((cap,), -7, dtype=torch.int64, device="cuda")
        cnt = torch.full((1,), -7, dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        hc.hc_search_noalloc(f, F_dev, x_dev, y_dev, pos, cnt)
        torch.cuda.synchronize()
        free_after.append((free_before, torch.cuda.mem_get_info()[0]))
        hc.hc_check_status()
        assert int(cnt.item()) == count, call
        assert torch.equal(pos[:count], ref_pos[:count]), call
        assert np.array_equal(pos[:count].cpu().numpy().view(np.uint64), want), call
        assert int(pos[count].item()) == -7, call   # nothing written past the count
    # the second call (the first has loaded the kernels) takes no device memory
    assert free_after[1][0] == free_after[1][1]
    f.free()


def test_noalloc_count_only_and_limit(hc):
    rng = np.random.default_rng(5)
    x, y = _case(rng, 4, 4_000_000, 12, plant=10)
    y_dev = torch.from_numpy(y).cuda()
    f = hc.hc_preprocess(x, 4, 12)
    F, _ = f.words()
    F_dev = torch.from_numpy(F.view(np.int32)).cuda()
    x_dev = torch.from_numpy(x).cuda()
    ref = torch.zeros(1, dtype=torch.int64, device="cuda")
    hc.hc_search_async(f, y_dev, None, ref)
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    hc.hc_search_noalloc(f, F_dev, x_dev, y_dev, None, cnt)      # count only, cap = 0
    torch.cuda.synchronize()
    assert int(cnt.item()) == int(ref.item()) >= 10
    big = torch.empty(2_000_001, dtype=torch.int64, device="cuda")
    with pytest.raises(hc.HCError) as ei:                       # above the fixed scratch
        hc.hc_search_noalloc(f, F_dev, x_dev, y_dev, big, cnt)
    assert ei.value.code == hc.HC_ERR_ARG
    f.free()


@pytest.mark.parametrize("sigma,m,q", [(4, 12, 4), (2, 2, 2)])
def test_noalloc_largest_documented_request(hc, sigma, m, q):
    """min(cap, n - m + 1) = 2,000,000, the documented limit, fits the fixed
    scratch (staged and dense kernels) and gives the oracle's positions."""
    rng = np.random.default_rng(17 + m)
    x, y = _case(rng, sigma, 2_000_000 + m - 1 + 4096, m, plant=5)
    y_dev = torch.from_numpy(y).cuda()
    f = hc.hc_preprocess(x, q, 12)
    F, _ = f.words()
    F_dev = torch.from_numpy(F.view(np.int32)).cuda()
    x_dev = torch.from_numpy(x).cuda()
    want = oracle.hc_search(x, y, q, 12)
    pos = torch.full((2_000_000,), -7, dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    hc.hc_search_noalloc(f, F_dev, x_dev, y_dev, pos, cnt)
    torch.cuda.synchronize()
    hc.hc_check_status()
    assert int(cnt.item()) == want.size
    k = min(want.size, 2_000_000)
    assert np.array_equal(pos[:k].cpu().numpy().view(np.uint64), want[:k])
    f.free()
