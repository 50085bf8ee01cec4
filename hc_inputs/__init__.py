"""Seeded synthetic inputs for the Hash Chain matcher: texts, patterns and the
workload recipes.

This module is shared by the tests, the benchmark and the smoke check; it
holds none of the string-matching arithmetic (no hashing, no filter, no
matching) and imports neither the CUDA library nor the oracle.

The paper measures on 100 MB genome, protein and English texts from the
Pizza&Chili corpus (Sec. 4).  Those files are not used: seeded synthetic
texts with the same alphabet sizes stand in for them (sigma = 4, 20, 95), plus
sigma = 2 and an order-2 Markov source over sigma = 60 with Zipf-distributed
symbol frequencies for English-like skew.  Patterns are copied from the text
at seeded offsets, as the paper extracts its patterns from the text at random.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

# Byte alphabet used for each synthetic alphabet size.  The byte values only
# affect hash collisions (speed), never the result set.
ALPHABETS = {
    1: b"A",
    2: b"01",
    3: b"012",
    4: b"ACGT",
    20: b"ACDEFGHIKLMNPQRSTVWY",
    60: bytes(range(65, 125)),
    95: bytes(range(32, 127)),
}


def alphabet(sigma: int) -> np.ndarray:
    if sigma in ALPHABETS:
        return np.frombuffer(ALPHABETS[sigma], dtype=np.uint8)
    if not 1 <= sigma <= 256:
        raise ValueError("sigma must be in [1, 256]")
    return np.arange(256 - sigma, 256, dtype=np.uint8) if sigma > 95 else \
        np.arange(32, 32 + sigma, dtype=np.uint8)


def uniform_text(n: int, sigma: int, seed: int) -> np.ndarray:
    """n bytes drawn i.i.d. uniform over the sigma-symbol alphabet (PCG64)."""
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, sigma, size=n, dtype=np.uint8)
    return np.take(alphabet(sigma), idx)


# ---------------------------------------------------------------------------
# order-2 Markov source (compiled helper, SplitMix64 streams per block)
_HERE = os.path.dirname(os.path.abspath(__file__))
_GEN_SRC = os.path.join(_HERE, "markov.c")
_GEN_LIB = os.path.join(_HERE, "_build", "libhcgen.so")
_gen_lock = threading.Lock()
_gen = None


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_GEN_LIB), exist_ok=True)
    if force or not os.path.exists(_GEN_LIB) or \
            os.path.getmtime(_GEN_LIB) < os.path.getmtime(_GEN_SRC):
        tmp = _GEN_LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp,
                        _GEN_SRC], check=True)
        os.replace(tmp, _GEN_LIB)
    return _GEN_LIB


def _genlib():
    global _gen
    with _gen_lock:
        if _gen is None:
            lib = ctypes.CDLL(build())
            lib.hcgen_markov2_block.restype = None
            lib.hcgen_markov2_block.argtypes = [
                ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p,
                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64]
            _gen = lib
        return _gen


def _cum_u32(p: np.ndarray) -> np.ndarray:
    c = np.cumsum(p / p.sum(axis=-1, keepdims=True), axis=-1)
    c = np.minimum(np.floor(c * 4294967295.0), 4294967295.0).astype(np.uint32)
    c[..., -1] = 0xFFFFFFFF
    return np.ascontiguousarray(c)


def markov2_tables(sigma: int = 60, zipf_s: float = 1.1, seed: int = 3):
    """Unigram and transition tables of the order-2 Markov source.

    Unigram frequencies are Zipf(s): p_k proportional to 1/k^s for rank k.
    Row (a, b) of the transition table is a Dirichlet draw with concentration
    sigma * zipf, so every row is a seeded random distribution whose mean is
    the Zipf unigram."""
    rng = np.random.default_rng(seed)
    ranks = np.arange(1, sigma + 1, dtype=np.float64)
    zipf = ranks ** (-zipf_s)
    zipf /= zipf.sum()
    rows = rng.dirichlet(sigma * zipf, size=sigma * sigma)
    rows = np.maximum(rows, 1e-12)
    return zipf, rows


def markov2_text(n: int, sigma: int = 60, zipf_s: float = 1.1, seed: int = 3,
                 block: int = 1 << 20, threads: int | None = None) -> np.ndarray:
    """n bytes of the order-2 Markov source.  The text is generated in
    independent blocks of ``block`` bytes (each restarts from two unigram
    draws) so that it can be produced in parallel and reproducibly."""
    from concurrent.futures import ThreadPoolExecutor
    zipf, rows = markov2_tables(sigma, zipf_s, seed)
    uni_cum, row_cum = _cum_u32(zipf), _cum_u32(rows)
    lut = np.ascontiguousarray(alphabet(sigma))
    out = np.empty(n, dtype=np.uint8)
    lib = _genlib()
    nblocks = (n + block - 1) // block

    def gen(b):
        lo = b * block
        ln = min(block, n - lo)
        lib.hcgen_markov2_block(out.ctypes.data + lo, ln, sigma,
                                uni_cum.ctypes.data, row_cum.ctypes.data,
                                lut.ctypes.data, seed, b)

    threads = threads or min(16, os.cpu_count() or 1)
    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(gen, range(nblocks)))
    return out


# ---------------------------------------------------------------------------
# patterns and parameters
def extract_pattern(y: np.ndarray, m: int, rng: np.random.Generator):
    """A length-m pattern copied from y at a seeded random offset."""
    off = int(rng.integers(0, y.size - m + 1))
    return y[off:off + m].copy(), off


# The paper's best-measured (q, alpha) for HC per text and pattern length
# (Tables 1-3: genome, protein, English; m = 8 .. 1024).
PAPER_QALPHA = {
    "genome": {8: (4, 12), 16: (6, 12), 32: (6, 12), 64: (6, 12), 128: (6, 12),
               256: (6, 12), 512: (6, 12), 1024: (8, 12)},
    "protein": {8: (3, 11), 16: (3, 11), 32: (3, 11), 64: (6, 12), 128: (3, 11),
                256: (3, 11), 512: (4, 12), 1024: (4, 12)},
    "english": {8: (3, 11), 16: (3, 11), 32: (6, 12), 64: (6, 12), 128: (3, 11),
                256: (3, 11), 512: (4, 12), 1024: (4, 12)},
}


def paper_q_alpha(sigma: int, m: int) -> tuple[int, int]:
    """(q, alpha) for an alphabet size and pattern length: the paper's choice
    for the nearest text (sigma <= 8 -> genome, <= 40 -> protein, else English)
    and the nearest m (log scale), with q clamped to m."""
    col = "genome" if sigma <= 8 else ("protein" if sigma <= 40 else "english")
    rows = sorted(PAPER_QALPHA[col])
    lm = math.log2(max(m, 1))
    best = min(rows, key=lambda r: (abs(math.log2(r) - lm), r))
    q, a = PAPER_QALPHA[col][best]
    return min(q, m), a


# ---------------------------------------------------------------------------
# workload recipes
@dataclass(frozen=True)
class Query:
    """One (pattern, text) query of a synthetic workload."""
    n: int
    m: int
    sigma: int
    text_seed: int
    pattern_seed: int
    q: int
    alpha: int


def config_one():
    """Plain HC, one query: n = 1 MiB i.i.d. uniform over sigma = 4 (seed 1),
    m = 16 copied from the text at a seeded offset, (q, alpha) = (6, 12)."""
    n, sigma, m = 1 << 20, 4, 16
    y = uniform_text(n, sigma, seed=1)
    x, off = extract_pattern(y, m, np.random.default_rng(1001))
    q, a = paper_q_alpha(sigma, m)
    return {"x": x, "y": y, "q": q, "alpha": a, "offset": off, "sigma": sigma}


SWEEP_SIGMAS = (2, 4, 20, 95)
SWEEP_MS = (2, 4, 8, 16, 32, 64, 128, 256, 512, 1024)
SKEW_MS = (4, 8, 16, 32, 64, 128, 256, 512, 1024)


def sweep_text(sigma: int, n: int = 1 << 28) -> np.ndarray:
    """Text of the plain-HC sweep: n bytes i.i.d. uniform, seed 100 + sigma."""
    return uniform_text(n, sigma, seed=100 + sigma)


def sweep_patterns(y: np.ndarray, sigma: int, m: int, count: int = 100):
    """``count`` patterns of length m for one sweep cell, copied from y."""
    rng = np.random.default_rng(10_000 * sigma + m)
    return [extract_pattern(y, m, rng)[0] for _ in range(count)]


def skew_text(n: int = 1 << 30) -> np.ndarray:
    """Text of the skewed config: order-2 Markov over sigma = 60, Zipf(1.1)."""
    return markov2_text(n, sigma=60, zipf_s=1.1, seed=3)


def batch_queries(count: int = 4096, seed: int = 4, n_lo: int = 4 << 10,
                  n_hi: int = 64 << 20, m_lo: int = 4, m_hi: int = 512):
    """Batched config: n log-uniform in [n_lo, n_hi], m log-uniform in
    [m_lo, m_hi], sigma drawn from {4, 20}; i.i.d. uniform texts; each pattern
    copied from its own text.  (q, alpha) are the paper's defaults here; the
    autotuner may override them."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        m = int(round(math.exp(rng.uniform(math.log(m_lo), math.log(m_hi)))))
        m = min(m, n)
        sigma = int(rng.choice([4, 20]))
        q, a = paper_q_alpha(sigma, m)
        out.append(Query(n, m, sigma, 1_000_000 + i, 2_000_000 + i, q, a))
    return out


def device_uniform_text(n: int, sigma: int, seed: int, device):
    """n bytes i.i.d. uniform over the sigma-symbol alphabet, drawn on a CUDA
    device with torch's seeded generator (for workloads too large to draw on
    the host; the same seed and device type give the same bytes)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    idx = torch.randint(0, sigma, (n,), generator=g, device=device, dtype=torch.int64)
    lut = torch.from_numpy(alphabet(sigma).copy()).to(device)
    return lut[idx]


def query_inputs(qr: Query):
    """(x, y) of one workload query."""
    y = uniform_text(qr.n, qr.sigma, qr.text_seed)
    x, _ = extract_pattern(y, qr.m, np.random.default_rng(qr.pattern_seed))
    return x, y


def served_texts(count: int = 64, seed: int = 5, n_lo: int = 1 << 10,
                 n_hi: int = 16 << 20):
    """Resident texts of the served config: n log-uniform in [n_lo, n_hi],
    sigma drawn from {4, 20, 95}; returns (n, sigma, text_seed) triples."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        sigma = int(rng.choice([4, 20, 95]))
        out.append((n, sigma, 3_000_000 + i))
    return out


def served_requests(texts, count: int, rate_per_s: float, seed: int = 6,
                    m_lo: int = 2, m_hi: int = 1024):
    """Poisson request stream for the served config: exponential
    inter-arrival gaps at ``rate_per_s``; each request names a text index and
    carries a pattern (m log-uniform in [m_lo, m_hi], at most the text length)
    copied from that text at a seeded offset.  Returns (arrival_s, text_idx,
    m, offset) tuples; the pattern bytes are text[offset:offset+m]."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(count):
        t += float(rng.exponential(1.0 / rate_per_s))
        ti = int(rng.integers(0, len(texts)))
        n = texts[ti][0]
        m = int(round(math.exp(rng.uniform(math.log(m_lo), math.log(m_hi)))))
        m = max(1, min(m, n))
        off = int(rng.integers(0, n - m + 1))
        out.append((t, ti, m, off))
    return out
