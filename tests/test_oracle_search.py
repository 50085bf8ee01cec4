"""Pins of the oracle's search functions.

The naive matcher is pinned to Python's own substring search (bytes.find and a
look-ahead regular expression, both library routines).  HC and SHC are pinned
to the problem statement (Sec. 1): every occurrence, ascending.  That is
checked exhaustively on all inputs over a three-letter alphabet with m <= 4 and
n <= 8 (tests/brute_force.c), and on seeded random, periodic and degenerate
inputs.  The chunk-split invariant that the GPU decomposition relies on is
checked here too: HC started at any window reports exactly the occurrences
that start at or after it.
"""
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _find_all(x: bytes, y: bytes):
    out, p = [], y.find(x)
    while p != -1:
        out.append(p)
        p = y.find(x, p + 1)
    return out


def _rand_case(rng, sigma, n, m, plant=3):
    y = rng.integers(0, sigma, n, dtype=np.uint8) + 65
    x = rng.integers(0, sigma, m, dtype=np.uint8) + 65
    if n >= m:
        for _ in range(plant):
            off = int(rng.integers(0, n - m + 1))
            y[off:off + m] = x
    return bytes(x), bytes(y)


# ---------------------------------------------------------------- naive ---
def test_naive_matches_bytes_find_and_regex():
    rng = np.random.default_rng(1)
    for _ in range(500):
        sigma = int(rng.choice([1, 2, 3, 4, 26]))
        n = int(rng.integers(0, 300))
        m = int(rng.integers(1, 12))
        x, y = _rand_case(rng, sigma, n, m)
        want = _find_all(x, y)
        got = oracle.naive_search(x, y).tolist()
        assert got == want
        assert got == [mt.start() for mt in re.finditer(b"(?=" + re.escape(x) + b")", y)]


def test_naive_edge_cases():
    assert oracle.naive_search(b"abc", b"ab").tolist() == []          # n < m
    assert oracle.naive_search(b"ab", b"ab").tolist() == [0]          # n == m
    assert oracle.naive_search(b"aa", b"aaaa").tolist() == [0, 1, 2]  # overlaps
    assert oracle.naive_search(b"a", b"").tolist() == []
    with pytest.raises(ValueError):
        oracle.naive_search(b"", b"abc")


# ------------------------------------------------------- exhaustive HC ---
def _run_brute_force(oracle_src: str) -> dict:
    with tempfile.TemporaryDirectory() as td:
        exe = os.path.join(td, "bf")
        subprocess.run(["gcc", "-O2", "-std=c99", "-o", exe,
                        os.path.join(ROOT, "tests", "brute_force.c"), oracle_src],
                       check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return {k: int(v) for k, v in (t.split("=") for t in out.split())}


def test_brute_force_all_small_inputs():
    r = _run_brute_force(os.path.join(ROOT, "oracle", "hc_oracle.c"))
    assert r["cases"] > 20_000_000
    assert r["hc_mismatch"] == 0
    assert r["shc_mismatch"] == 0


# ----------------------------------------------------------- random HC ---
@pytest.mark.parametrize("sigma", [1, 2, 4, 20, 95])
def test_hc_and_shc_equal_naive_random(sigma):
    rng = np.random.default_rng(100 + sigma)
    for _ in range(150):
        m = int(rng.choice([1, 2, 3, 4, 5, 7, 8, 9, 13, 16, 17, 31, 32, 64, 100]))
        n = int(rng.integers(0, 4000))
        q = int(rng.integers(1, min(m, 8) + 1))
        alpha = int(rng.integers(1, 16))
        x, y = _rand_case(rng, sigma, n, m, plant=int(rng.integers(0, 6)))
        want = oracle.naive_search(x, y)
        assert np.array_equal(oracle.hc_search(x, y, q, alpha), want), (m, n, q, alpha)
        assert np.array_equal(oracle.shc_search(x, y, q, alpha), want), (m, n, q, alpha)


def test_hc_periodic_and_degenerate_texts():
    cases = [
        (b"a" * 5, b"a" * 100),                 # sigma = 1, all overlapping
        (b"ab" * 4, b"ab" * 200),               # periodic
        (b"abaab", b"abaababaabaab" * 30),      # Fibonacci-like
        (b"x", b"xyxxyx"),                      # m = 1
        (b"abcdefgh", b"zzabcdefghzz"),         # m = q possible
        (b"abc", b"abc"),                       # n == m
        (b"abcd", b"abc"),                      # n < m
    ]
    for x, y in cases:
        want = _find_all(x, y)
        for q in range(1, min(len(x), 8) + 1):
            for alpha in (1, 2, 5, 8, 12, 15):
                assert oracle.hc_search(x, y, q, alpha).tolist() == want
                assert oracle.shc_search(x, y, q, alpha).tolist() == want


def test_alpha_below_q_gives_s_zero_and_stays_exact():
    # Eq. 4 with alpha < q gives s = 0: h degenerates to a byte sum mod 2^alpha
    rng = np.random.default_rng(5)
    for _ in range(100):
        x, y = _rand_case(rng, 3, 2000, 8, plant=4)
        assert np.array_equal(oracle.hc_search(x, y, 8, 3), oracle.naive_search(x, y))


def test_occurrences_at_both_ends():
    x = b"GATTACA"
    y = x + b"CCCCCCCCCC" + x
    for q in range(1, 8):
        assert oracle.hc_search(x, y, q, 11).tolist() == [0, len(y) - len(x)]


def test_hc_rejects_invalid():
    for q, alpha in [(0, 10), (5, 10), (2, 0), (2, 16)]:
        with pytest.raises(ValueError):
            oracle.hc_search(b"abcd", b"abcdabcd", q, alpha)


# ------------------------------------------------ chunk-split invariant ---
def test_chunk_split_invariant():
    """HC over window-start ranges [a, b) (text y[a : b+m-1]) concatenated in
    order equals HC over the whole text, for random splits."""
    rng = np.random.default_rng(9)
    for _ in range(300):
        sigma = int(rng.choice([2, 4, 20]))
        m = int(rng.choice([1, 2, 4, 8, 16, 33]))
        n = int(rng.integers(m, 3000))
        q = int(rng.integers(1, min(m, 8) + 1))
        alpha = int(rng.integers(4, 13))
        x, y = _rand_case(rng, sigma, n, m, plant=5)
        full = oracle.hc_search(x, y, q, alpha)
        nwin = n - m + 1
        cuts = sorted(set([0, nwin] + rng.integers(0, nwin + 1, 6).tolist()))
        parts = []
        for a, b in zip(cuts[:-1], cuts[1:]):
            parts.append(oracle.hc_search(x, y[a:b + m - 1], q, alpha) + np.uint64(a))
        assert np.array_equal(np.concatenate(parts), full)


def test_threaded_oracle_equals_single_thread():
    rng = np.random.default_rng(11)
    for m in (2, 8, 16, 100):
        x, y = _rand_case(rng, 4, 200_000, m, plant=50)
        a = oracle.hc_search(x, y, min(m, 6), 12)
        for t in (2, 3, 8):
            assert np.array_equal(oracle.hc_search_threaded(x, y, min(m, 6), 12, t), a)
