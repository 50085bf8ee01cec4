"""CPU oracle for the Hash Chain (HC) exact string matcher (arXiv 2310.15711).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg (and its ``--impl reference`` arm) may import this package.
The product library never does: it shares no code with this module, and this
module loads nothing from it.

The arithmetic lives in ``hc_oracle.c`` (plain C, compiled with gcc into
``oracle/_build/liboracle.so``); this file only marshals arguments.  Functions:

* :func:`naive_search` -- the problem statement (Sec. 1, Sec. 2): every window
  start ``p`` with ``y[p:p+m] == x``, ascending.
* :func:`hash_qgram`, :func:`link_hash` -- ``h`` (Eq. 3, Eq. 4; the backward
  Hash routine of Fig. 4) and ``lambda`` (Eq. 5) with w = 32.
* :func:`preprocess` -- the preprocessing phase (Sec. 3.1, Eq. 1, Eq. 2,
  Fig. 4, first optimisation of Sec. 3.4): returns F, s, F', H_v and,
  optionally, the end positions of the hashed q-grams in call order.
* :func:`hc_search` -- the HC searching phase (Sec. 3.3, Fig. 5 left), with the
  verify/output position read as the start of the scanned window.
* :func:`shc_search` -- the sentinel variant SHC (Sec. 3.4, Fig. 5 right).

Every pin of these functions is in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hc_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_u8p = ctypes.POINTER(ctypes.c_uint8)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_longp = ctypes.POINTER(ctypes.c_long)


def build(force: bool = False) -> str:
    """Compile ``hc_oracle.c`` with gcc into ``oracle/_build/liboracle.so``."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O3", "-std=c99", "-Wall", "-shared", "-fPIC",
                        "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.or_naive_search.restype = ctypes.c_size_t
        lib.or_naive_search.argtypes = [_u8p, ctypes.c_size_t, _u8p,
                                        ctypes.c_size_t, _u64p, ctypes.c_size_t]
        lib.or_hash.restype = ctypes.c_uint32
        lib.or_hash.argtypes = [_u8p, ctypes.c_long, ctypes.c_int, ctypes.c_int,
                                ctypes.c_uint32]
        lib.or_link_hash.restype = ctypes.c_uint32
        lib.or_link_hash.argtypes = [ctypes.c_uint32]
        lib.or_preprocess.restype = ctypes.c_int
        lib.or_preprocess.argtypes = [
            _u8p, ctypes.c_long, ctypes.c_int, ctypes.c_int, _u32p,
            ctypes.POINTER(ctypes.c_int), _u32p, _u32p, _longp, ctypes.c_long,
            _longp, _longp]
        lib.or_hc_search.restype = ctypes.c_size_t
        lib.or_hc_search.argtypes = [_u8p, ctypes.c_long, _u8p, ctypes.c_long,
                                     ctypes.c_int, ctypes.c_int, _u32p, _u64p,
                                     ctypes.c_size_t]
        lib.or_shc_search.restype = ctypes.c_size_t
        lib.or_shc_search.argtypes = [_u8p, ctypes.c_long, _u8p, ctypes.c_long,
                                      ctypes.c_int, ctypes.c_int, _u32p, _u64p,
                                      ctypes.c_size_t]
        _lib = lib
        return lib


def _as_u8(a) -> np.ndarray:
    if isinstance(a, (bytes, bytearray, memoryview)):
        return np.frombuffer(bytes(a), dtype=np.uint8)
    a = np.ascontiguousarray(a)
    if a.dtype != np.uint8:
        raise TypeError("oracle inputs are byte strings (uint8)")
    return a


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


_ERR = ctypes.c_size_t(-1).value


def _collect(call, guess: int) -> np.ndarray:
    """Run ``call(out, cap) -> count`` until ``out`` holds every position."""
    cap = max(int(guess), 1)
    while True:
        out = np.empty(cap, dtype=np.uint64)
        count = call(out, cap)
        if count == _ERR:
            raise ValueError("invalid HC arguments (need 1 <= q <= m, 1 <= alpha <= 15)")
        if count <= cap:
            return out[:count].copy()
        cap = count


def naive_search(x, y) -> np.ndarray:
    """All occurrences of x in y (Sec. 1): ascending uint64 window starts."""
    lib = _load()
    x, y = _as_u8(x), _as_u8(y)
    m, n = x.size, y.size
    if m == 0:
        raise ValueError("m must be >= 1")
    return _collect(lambda out, cap: lib.or_naive_search(
        _ptr(x, ctypes.c_uint8), m, _ptr(y, ctypes.c_uint8), n,
        _ptr(out, ctypes.c_uint64), cap), min(max(n - m + 1, 1), 1 << 16))


def hash_qgram(x, p: int, q: int, alpha: int) -> int:
    """h of the q-gram of x that ends at position p (Eq. 3, Eq. 4, Fig. 4)."""
    lib = _load()
    x = _as_u8(x)
    if not (0 <= p - q + 1 and p < x.size):
        raise IndexError("q-gram out of range")
    return int(lib.or_hash(_ptr(x, ctypes.c_uint8), p, q, alpha // q,
                           (1 << alpha) - 1))


def link_hash(v: int) -> int:
    """lambda(v) = 2^(v mod 32) (Eq. 5, w = 32)."""
    return int(_load().or_link_hash(v))


def preprocess(x, q: int, alpha: int, trace: bool = False) -> dict:
    """Preprocessing(x, m, q, alpha) of Fig. 4.

    Returns a dict with ``F`` (uint32 array of 2^alpha words), ``s``, ``mask``
    (F'), ``hv`` (H_v) and, when ``trace`` is set, ``trace`` (end positions of
    the hashed q-grams, in call order) and ``chain_calls`` (how many of those
    calls belong to the chain phase; the rest are the marking phase).
    """
    lib = _load()
    x = _as_u8(x)
    m = x.size
    if not (1 <= q <= m and 1 <= alpha <= 15):
        raise ValueError("need 1 <= q <= m and 1 <= alpha <= 15")
    F = np.zeros(1 << alpha, dtype=np.uint32)
    s = ctypes.c_int(0)
    mask = ctypes.c_uint32(0)
    hv = ctypes.c_uint32(0)
    tlen = ctypes.c_long(0)
    ccalls = ctypes.c_long(0)
    tcap = 2 * m + 4
    tr = np.zeros(tcap, dtype=np.int64) if trace else None
    rc = lib.or_preprocess(
        _ptr(x, ctypes.c_uint8), m, q, alpha, _ptr(F, ctypes.c_uint32),
        ctypes.byref(s), ctypes.byref(mask), ctypes.byref(hv),
        tr.ctypes.data_as(_longp) if trace else None, tcap if trace else 0,
        ctypes.byref(tlen), ctypes.byref(ccalls))
    if rc != 0:
        raise ValueError("or_preprocess rejected its arguments")
    res = {"F": F, "s": s.value, "mask": mask.value, "hv": hv.value}
    if trace:
        res["trace"] = tr[: min(tlen.value, tcap)].tolist()
        res["chain_calls"] = ccalls.value
        res["calls"] = tlen.value
    return res


def hc_search(x, y, q: int, alpha: int) -> np.ndarray:
    """HC(x, m, y, n, q, alpha) of Fig. 5 left: ascending uint64 positions."""
    lib = _load()
    x, y = _as_u8(x), _as_u8(y)
    m, n = x.size, y.size
    F = np.zeros(1 << alpha, dtype=np.uint32) if 1 <= alpha <= 15 else np.zeros(1, np.uint32)
    return _collect(lambda out, cap: lib.or_hc_search(
        _ptr(x, ctypes.c_uint8), m, _ptr(y, ctypes.c_uint8), n, q, alpha,
        _ptr(F, ctypes.c_uint32), _ptr(out, ctypes.c_uint64), cap),
        min(max(n - m + 1, 1), 1 << 16))


def shc_search(x, y, q: int, alpha: int) -> np.ndarray:
    """SHC of Fig. 5 right (sentinel): same result set as :func:`hc_search`.

    The text is copied into a private writable buffer of n + m bytes first, as
    the sentinel needs (Sec. 3.4)."""
    lib = _load()
    x, y = _as_u8(x), _as_u8(y)
    m, n = x.size, y.size
    ybuf = np.empty(n + m, dtype=np.uint8)
    ybuf[:n] = y
    F = np.zeros(1 << alpha, dtype=np.uint32) if 1 <= alpha <= 15 else np.zeros(1, np.uint32)
    return _collect(lambda out, cap: lib.or_shc_search(
        _ptr(x, ctypes.c_uint8), m, _ptr(ybuf, ctypes.c_uint8), n, q, alpha,
        _ptr(F, ctypes.c_uint32), _ptr(out, ctypes.c_uint64), cap),
        min(max(n - m + 1, 1), 1 << 16))


def hc_search_threaded(x, y, q: int, alpha: int, threads: int) -> np.ndarray:
    """:func:`hc_search` run on ``threads`` host threads over text pieces that
    overlap by m-1 bytes, results concatenated in text order.

    Exact because HC, started at any window, reports every occurrence that
    starts at or after it (its shifts never pass over an occurrence, Sec. 3.3):
    piece k covers the window starts [a_k, a_{k+1}) and reads y[a_k,
    a_{k+1}+m-1).  ctypes releases the GIL during each C call."""
    from concurrent.futures import ThreadPoolExecutor
    x, y = _as_u8(x), _as_u8(y)
    m, n = x.size, y.size
    if threads <= 1 or n < 2 * m:
        return hc_search(x, y, q, alpha)
    nwin = n - m + 1
    bounds = [nwin * k // threads for k in range(threads + 1)]

    def piece(k):
        a, b = bounds[k], bounds[k + 1]
        if a >= b:
            return np.empty(0, np.uint64)
        return hc_search(x, y[a:b + m - 1], q, alpha) + np.uint64(a)

    with ThreadPoolExecutor(threads) as ex:
        parts = list(ex.map(piece, range(threads)))
    return np.concatenate(parts) if parts else np.empty(0, np.uint64)
