"""Checks of the seeded synthetic input generators (no method arithmetic)."""
import numpy as np

import hc_inputs as hi


def test_uniform_text_is_seeded_and_on_alphabet():
    a = hi.uniform_text(100_000, 4, seed=1)
    b = hi.uniform_text(100_000, 4, seed=1)
    c = hi.uniform_text(100_000, 4, seed=2)
    assert a.dtype == np.uint8 and np.array_equal(a, b) and not np.array_equal(a, c)
    assert set(np.unique(a).tolist()) == set(b"ACGT")
    counts = np.bincount(a)[list(b"ACGT")]
    assert np.all(np.abs(counts / a.size - 0.25) < 0.01)


def test_alphabet_sizes():
    for sigma in (1, 2, 4, 20, 60, 95):
        al = hi.alphabet(sigma)
        assert al.size == sigma == np.unique(al).size


def test_markov_text_seeded_skewed_and_order2():
    t1 = hi.markov2_text(1 << 21, seed=3, block=1 << 18)
    t2 = hi.markov2_text(1 << 21, seed=3, block=1 << 18)
    assert np.array_equal(t1, t2)
    assert set(np.unique(t1).tolist()) <= set(range(65, 125))
    freq = np.bincount(t1, minlength=256)[65:125] / t1.size
    # Zipf(1.1)-like: rank-1 symbol far more frequent than rank-30
    assert freq[0] > 5 * freq[29]
    # order-2 dependence: the next-symbol distribution differs by context
    a, b = t1[:-2].astype(np.int64), t1[1:-1].astype(np.int64)
    c = t1[2:]
    ctx = (a == 65) & (b == 65)
    ctx2 = (a == 66) & (b == 65)
    p1 = np.bincount(c[ctx], minlength=256)[65:125] / max(ctx.sum(), 1)
    p2 = np.bincount(c[ctx2], minlength=256)[65:125] / max(ctx2.sum(), 1)
    assert np.abs(p1 - p2).sum() > 0.1


def test_pattern_is_copied_from_text():
    y = hi.uniform_text(10_000, 20, seed=4)
    x, off = hi.extract_pattern(y, 33, np.random.default_rng(0))
    assert np.array_equal(y[off:off + 33], x)


def test_config_one_recipe():
    c = hi.config_one()
    assert c["y"].size == 1 << 20 and c["x"].size == 16
    assert (c["q"], c["alpha"]) == (6, 12)       # Table 1, m = 16, genome
    assert np.array_equal(c["y"][c["offset"]:c["offset"] + 16], c["x"])


def test_paper_q_alpha_table():
    assert hi.paper_q_alpha(4, 1024) == (8, 12)
    assert hi.paper_q_alpha(20, 512) == (4, 12)
    assert hi.paper_q_alpha(95, 32) == (6, 12)
    assert hi.paper_q_alpha(4, 2) == (2, 12)     # clamped to m
    assert hi.paper_q_alpha(95, 4) == (3, 11)


def test_batch_and_served_recipes():
    qs = hi.batch_queries(256)
    assert all(4 << 10 <= q.n <= 64 << 20 and 4 <= q.m <= 512 for q in qs)
    assert {q.sigma for q in qs} == {4, 20}
    texts = hi.served_texts()
    assert len(texts) == 64 and all(1 << 10 <= n <= 16 << 20 for n, _, _ in texts)
    reqs = hi.served_requests(texts, 500, 1000.0)
    t = [r[0] for r in reqs]
    assert t == sorted(t) and 0.2 < t[-1] < 1.0
