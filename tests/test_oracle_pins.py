"""Pins of the oracle's hash functions and preprocessing to the paper.

Each check compares the oracle with something other than itself: values worked
by hand from Eq. 3 / Eq. 4 (tests/golden/hash_eq3.txt), the recursive form of
Eq. 3, the chains the paper prints for its worked examples (Fig. 1, Fig. 2;
tests/golden/fig*_chains.txt), the set-builder definition of a q-gram chain
(Sec. 3.1), the chain-count statement (Sec. 3.1), and F rebuilt pair by pair
from Eq. 1 and Eq. 2 in text order rather than chain by chain.
"""
import os
import random

import numpy as np
import pytest

import oracle


def _read_golden(path):
    rows = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------- hash h ---
def test_hash_hand_worked_values(golden_dir):
    rows = _read_golden(os.path.join(golden_dir, "hash_eq3.txt"))
    assert len(rows) >= 5
    for hexbytes, q, alpha, want in rows:
        qg = bytes.fromhex(hexbytes)
        q, alpha, want = int(q), int(alpha), int(want)
        assert len(qg) == q
        # place the q-gram inside a longer string so the end position matters
        x = b"\x07\x09" + qg + b"\x05"
        assert oracle.hash_qgram(x, 2 + q - 1, q, alpha) == want


def _h_eq3(u: bytes, s: int, alpha: int) -> int:
    """Eq. 3 as printed: h(u) = (h(u[1..]) * 2^s + u[0]) mod 2^alpha."""
    if len(u) == 0:
        return 0
    return (_h_eq3(u[1:], s, alpha) * (1 << s) + u[0]) % (1 << alpha)


def test_hash_equals_recursive_eq3():
    rng = random.Random(7)
    for _ in range(3000):
        q = rng.randint(1, 8)
        alpha = rng.randint(1, 15)
        u = bytes(rng.randrange(256) for _ in range(q))
        x = bytes(rng.randrange(256) for _ in range(3)) + u
        got = oracle.hash_qgram(x, len(x) - 1, q, alpha)
        assert got == _h_eq3(u, alpha // q, alpha), (u, q, alpha)


def test_hash_shift_is_floor_alpha_over_q():
    # Eq. 4: with u = (1, 0, .., 0, 1) the last character's weight 2^(s(q-1))
    # exposes s directly (before the mod), for every q and alpha with
    # s(q-1) < alpha.
    for q in range(2, 9):
        for alpha in range(1, 16):
            s = alpha // q
            if s * (q - 1) >= alpha:
                continue
            u = bytes([1] + [0] * (q - 2) + [1])
            want = (1 + (1 << (s * (q - 1)))) % (1 << alpha)
            assert oracle.hash_qgram(u, q - 1, q, alpha) == want


def test_link_hash_is_one_bit_at_v_mod_w():
    for v in range(1 << 15):
        lh = oracle.link_hash(v)
        assert lh != 0 and lh & (lh - 1) == 0        # exactly one bit (Eq. 5)
        assert lh.bit_length() - 1 == v % 32         # w = 32


# -------------------------------------------------------- worked examples --
def _chains_from_trace(tr, chain_calls):
    """Split the chain-phase hash positions into chains: within a chain the
    end position decreases by q; a new chain starts when it goes up."""
    chains, cur = [], []
    for p in tr[:chain_calls]:
        if cur and p > cur[-1]:
            chains.append(cur)
            cur = []
        cur.append(p)
    if cur:
        chains.append(cur)
    return chains


def test_fig1_three_chains_eleven_hashes(golden_dir):
    g = dict((r[0], int(r[1])) for r in _read_golden(
        os.path.join(golden_dir, "fig1_chains.txt")))
    m, q = g["m"], g["q"]
    x = bytes(np.random.default_rng(13).integers(0, 256, m, dtype=np.uint8))
    pre = oracle.preprocess(x, q, 12, trace=True)
    chains = _chains_from_trace(pre["trace"], pre["chain_calls"])
    assert len(chains) == g["chains"]
    assert pre["chain_calls"] == g["chain_hashes"] == m - q + 1
    assert pre["calls"] - pre["chain_calls"] == g["marking_hashes"]
    # H_v is the hash labelled H11: the last chain-phase hash ...
    hv_pos = pre["trace"][g["hv_label"] - 1]
    assert pre["hv"] == oracle.hash_qgram(x, hv_pos, q, 12)
    # ... and that q-gram is the first one of the chain ending at m-1.
    last_chain = chains[-1]
    assert last_chain[0] == m - 1 and hv_pos == last_chain[-1]
    assert hv_pos - q + 1 < q


def test_fig2_chains(golden_dir):
    rows = _read_golden(os.path.join(golden_dir, "fig2_chains.txt"))
    pat = [r[1] for r in rows if r[0] == "pattern"][0].encode()
    q = int([r[1] for r in rows if r[0] == "q"][0])
    want = {int(r[1]): r[2:] for r in rows if r[0] == "chain"}
    pre = oracle.preprocess(pat, q, 12, trace=True)
    chains = _chains_from_trace(pre["trace"], pre["chain_calls"])
    got = {}
    for ch in chains:
        starts = sorted(p - q + 1 for p in ch)
        got[starts[0]] = [pat[s:s + q].decode() for s in starts]
    assert got == want


# ----------------------------------------------- chain structure (Sec. 3.1) --
@pytest.mark.parametrize("m", list(range(1, 40)) + [64, 100, 257])
def test_chains_match_set_builder_definition(m):
    x = bytes(np.random.default_rng(m).integers(0, 256, m, dtype=np.uint8))
    for q in range(1, min(m, 9) + 1):
        pre = oracle.preprocess(x, q, 10, trace=True)
        chains = _chains_from_trace(pre["trace"], pre["chain_calls"])
        # Sec. 3.1: each pattern position j, m-q <= j < m, defines the chain
        # {x[i..i+q-1] : i >= 0, i = j-q+1, j-2q+1, ...} of floor((j+1)/q)
        # q-grams (listed here by end position, right to left).
        want = []
        for j in range(m - q, m):
            ends = list(range(j, q - 2, -q))
            assert len(ends) == (j + 1) // q
            if ends:
                want.append(ends)
        assert sorted(map(tuple, chains)) == sorted(map(tuple, want))
        # Sec. 3.1: m-q+1 distinct chains if m < 2q-1, else q
        assert len(chains) == (m - q + 1 if m < 2 * q - 1 else q)
        # every q-gram of x is hashed exactly once in the chain phase
        assert sorted(pre["trace"][:pre["chain_calls"]]) == list(range(q - 1, m))
        # the marking phase re-hashes the first min(q, m-q+1) q-grams
        assert pre["trace"][pre["chain_calls"]:] == \
            list(range(q - 1, min(2 * q - 1, m)))


# ------------------------------------------------- F from Eq. 1 and Eq. 2 --
def _filter_from_equations(x: bytes, q: int, alpha: int):
    """F built directly from Eq. 1 (every adjacent non-overlapping pair, in
    text order) and then Eq. 2 with the first optimisation of Sec. 3.4 (value
    1 only into words still empty), hashing with the recursive Eq. 3."""
    m, s = len(x), alpha // q
    F = [0] * (1 << alpha)
    h = lambda i: _h_eq3(x[i:i + q], s, alpha)   # q-gram starting at i
    for i in range(0, m - 2 * q + 1):
        F[h(i + q)] |= 1 << (h(i) % 32)
    for i in range(0, min(q, m - q + 1)):
        if F[h(i)] == 0:
            F[h(i)] = 1
    hv = h(m % q)   # first q-gram of the chain that ends at m-1 (Sec. 3.4)
    return np.array(F, dtype=np.uint32), hv


def test_filter_equals_pairwise_equations():
    rng = np.random.default_rng(21)
    for trial in range(400):
        m = int(rng.integers(1, 80))
        q = int(rng.integers(1, min(m, 8) + 1))
        alpha = int(rng.integers(1, 13))
        sigma = int(rng.choice([1, 2, 4, 20, 256]))
        x = bytes(rng.integers(0, sigma, m, dtype=np.uint8) + (0 if sigma == 256 else 60))
        pre = oracle.preprocess(x, q, alpha)
        F, hv = _filter_from_equations(x, q, alpha)
        assert np.array_equal(pre["F"], F), (x, q, alpha)
        assert pre["hv"] == hv
        assert pre["s"] == alpha // q and pre["mask"] == (1 << alpha) - 1


def test_filter_invariants_every_qgram_present_and_pairs_linked():
    rng = np.random.default_rng(22)
    for _ in range(200):
        m = int(rng.integers(1, 300))
        q = int(rng.integers(1, min(m, 8) + 1))
        alpha = int(rng.integers(8, 16))
        x = bytes(rng.integers(0, 4, m, dtype=np.uint8) + 65)
        pre = oracle.preprocess(x, q, alpha)
        F = pre["F"]
        hs = [oracle.hash_qgram(x, i + q - 1, q, alpha) for i in range(m - q + 1)]
        assert all(F[v] != 0 for v in hs)                       # Sec. 3.3 first test
        for i in range(0, m - 2 * q + 1):                       # Eq. 1
            assert F[hs[i + q]] & (1 << (hs[i] % 32))


def test_preprocess_rejects_invalid():
    with pytest.raises(ValueError):
        oracle.preprocess(b"abc", 4, 10)       # q > m
    with pytest.raises(ValueError):
        oracle.preprocess(b"abc", 0, 10)       # q < 1
    with pytest.raises(ValueError):
        oracle.preprocess(b"abc", 2, 0)        # alpha < 1
    with pytest.raises(ValueError):
        oracle.preprocess(b"abc", 2, 16)       # alpha > 15
    with pytest.raises(ValueError):
        oracle.preprocess(b"", 1, 10)          # m = 0
