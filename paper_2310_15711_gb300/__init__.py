"""Python binding of libhc, the GB300 (sm_103a) Hash Chain string matcher.

Argument marshalling only: every step of the search runs in the library's
CUDA kernels (``include/hc.h`` documents the C ABI; the names here are the
same).  PyTorch supplies device memory and streams.  There is no CPU fallback:
if ``libhc.so`` has not been built, every call raises.

Method: "Efficient Online String Matching through Linked Weak Factors"
(Palmer, Faro, Scafiti; arXiv 2310.15711): preprocessing Sec. 3.1 (Eq. 1-5,
Fig. 4), searching phase Sec. 3.3 (Fig. 5), optimisations Sec. 3.4.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

LIB_PATH = _build.LIB_PATH

HC_OK = 0
HC_ERR_ARG = 1
HC_ERR_CAPACITY = 2
HC_ERR_CUDA = 3
HC_ERR_NOMEM = 4
HC_ERR_TIMEOUT = 5
HC_ERR_ADMISSION = 6
HC_ERR_STATE = 7

_ERR_NAMES = {1: "HC_ERR_ARG", 2: "HC_ERR_CAPACITY", 3: "HC_ERR_CUDA", 4: "HC_ERR_NOMEM",
              5: "HC_ERR_TIMEOUT", 6: "HC_ERR_ADMISSION", 7: "HC_ERR_STATE"}


class HCError(RuntimeError):
    """A libhc call returned an error code."""

    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {_ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None

_c_u8p = ctypes.c_void_p
_vp = ctypes.c_void_p
_sz = ctypes.c_size_t

# name -> (restype, argtypes); the full set of symbols declared in include/hc.h
SIGNATURES = {
    "hc_version": (ctypes.c_int, []),
    "hc_last_error": (ctypes.c_char_p, []),
    "hc_preprocess": (ctypes.c_int, [_vp, _sz, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp)]),
    "hc_filter_free": (None, [_vp]),
    "hc_filter_words": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.POINTER(ctypes.c_uint32)),
                                       ctypes.POINTER(_sz), ctypes.POINTER(ctypes.c_uint32)]),
    "hc_filter_params": (ctypes.c_int, [_vp, ctypes.POINTER(_sz), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "hc_filter_to_device": (ctypes.c_int, [_vp]),
    "hc_search_async": (ctypes.c_int, [_vp, _vp, _sz, _vp, _sz, _vp, _vp]),
    "hc_search": (ctypes.c_int, [_vp, _vp, _vp, _sz, _vp, _sz, ctypes.POINTER(_sz), _vp]),
    "hc_search_ex": (ctypes.c_int, [_vp, _vp, _sz, _vp, _sz, _vp, _vp, _vp]),
    "hc_search_noalloc": (ctypes.c_int, [_vp, _vp, _vp, _vp, _sz, _vp, _sz, _vp, _vp]),
    "hc_batch_create": (ctypes.c_int, [_vp, _sz, ctypes.POINTER(_vp)]),
    "hc_batch_run": (ctypes.c_int, [_vp, _vp]),
    "hc_batch_info": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_uint64),
                                     ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
    "hc_batch_filter": (ctypes.c_int, [_vp, _sz, ctypes.POINTER(ctypes.c_uint32), _sz,
                                       ctypes.POINTER(ctypes.c_uint32)]),
    "hc_batch_destroy": (None, [_vp]),
    "hc_batch_create_tuned": (ctypes.c_int, [_vp, _sz, _vp, ctypes.POINTER(_vp)]),
    "hc_batch_params": (ctypes.c_int, [_vp, _sz, _vp]),
    "hc_tuner_create": (ctypes.c_int, [ctypes.POINTER(_vp)]),
    "hc_tuner_calibrate": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), _sz,
                                          ctypes.POINTER(ctypes.c_uint64), _sz, ctypes.c_uint64,
                                          ctypes.c_uint64, ctypes.c_int, _vp]),
    "hc_tuner_lookup": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_uint64, _vp]),
    "hc_tuner_size": (ctypes.c_int, [_vp, ctypes.POINTER(_sz)]),
    "hc_tuner_entry": (ctypes.c_int, [_vp, _sz, _vp]),
    "hc_tuner_save": (ctypes.c_int, [_vp, ctypes.c_char_p]),
    "hc_tuner_load": (ctypes.c_int, [_vp, ctypes.c_char_p]),
    "hc_tuner_free": (None, [_vp]),
    "hc_server_create": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(_vp)]),
    "hc_server_add_text": (ctypes.c_int, [_vp, _vp, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_uint32)]),
    "hc_server_text_info": (ctypes.c_int, [_vp, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64),
                                           ctypes.POINTER(ctypes.c_double)]),
    "hc_server_submit": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(ctypes.c_uint64)]),
    "hc_server_replay": (ctypes.c_int, [_vp, _vp, _sz, ctypes.POINTER(ctypes.c_uint64),
                                        ctypes.POINTER(ctypes.c_uint64)]),
    "hc_server_poll": (ctypes.c_int, [_vp, _vp, _sz, ctypes.POINTER(_sz), ctypes.c_int64]),
    "hc_server_release": (ctypes.c_int, [_vp, ctypes.c_uint64]),
    "hc_server_drain": (ctypes.c_int, [_vp, ctypes.c_int64]),
    "hc_server_get_stats": (ctypes.c_int, [_vp, _vp]),
    "hc_server_destroy": (None, [_vp]),
    "hc_check_status": (ctypes.c_int, [_vp]),
    "hc_selftest_wait_timeout": (ctypes.c_int, [_vp]),
    "hc_check_bounds": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint64)]),
    "hc_mapped_alloc": (ctypes.c_int, [_sz, ctypes.POINTER(_vp), ctypes.POINTER(_vp)]),
    "hc_mapped_free": (None, [_vp]),
    "hc_kernel_launches": (ctypes.c_uint64, []),
    "hc_timing_enable": (ctypes.c_int, [ctypes.c_int]),
    "hc_timing_report": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_uint64), ctypes.c_int, ctypes.c_int]),
    "hc_timing_kind_name": (ctypes.c_char_p, [ctypes.c_int]),
}


def lib():
    """The loaded libhc.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"libhc.so not found at {LIB_PATH}: build it first "
                    "(python -c 'import __graft_entry__ as g; g.build()'); "
                    "there is no CPU fallback")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib


def _check(rc: int, where: str):
    if rc != HC_OK:
        msg = lib().hc_last_error()
        raise HCError(rc, where, msg.decode() if msg else "")


def _bytes_arg(x):
    if isinstance(x, np.ndarray):
        x = np.ascontiguousarray(x, dtype=np.uint8).tobytes()
    elif not isinstance(x, (bytes, bytearray)):
        x = bytes(x)
    return bytes(x)


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t, dtype_bytes=None):
    if t is None:
        return None
    if isinstance(t, MappedView):
        return ctypes.c_void_p(t.device_address)
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _nbytes(t) -> int:
    """Bytes of a text or pattern tensor (the library reads bytes)."""
    return t.numel() * t.element_size()


def _text_len(y_dev, n) -> int:
    """The text length passed to the library: all of y_dev, or the caller's
    n, which must not exceed the bytes of y_dev (the kernels read n bytes)."""
    have = _nbytes(y_dev) if y_dev is not None else 0
    if n is None:
        return have
    n = int(n)
    if n < 0 or n > have:
        raise ValueError(f"n = {n} does not fit the text buffer ({have} bytes)")
    return n


def _room(buf, entry_bytes: int) -> int:
    """Entries of `entry_bytes` bytes that fit in an output buffer (a CUDA
    tensor of any dtype, or a MappedView of int64 slots)."""
    if isinstance(buf, MappedView):
        return buf.count * 8 // entry_bytes
    return buf.numel() * buf.element_size() // entry_bytes


def _cap_for(pos_dev, cap, entry_bytes: int) -> int:
    """The capacity passed to the library: the caller's cap, which must fit
    in pos_dev, or all of pos_dev (counted in positions of entry_bytes)."""
    if pos_dev is None:
        return 0
    room = _room(pos_dev, entry_bytes)
    if cap is None:
        return room
    cap = int(cap)
    if cap < 0 or cap > room:
        raise ValueError(f"cap {cap} does not fit the output buffer ({room} positions of {entry_bytes} bytes)")
    return cap


def _check_count(count_dev):
    if count_dev is not None and _room(count_dev, 8) < 1:
        raise ValueError("count_dev must hold one uint64")


class MappedView:
    """A run of int64 slots in a MappedBuffer, usable as an output (pos_dev,
    count_dev) of the search calls."""

    def __init__(self, buf: "MappedBuffer", offset: int, count: int):
        self.buf, self.offset, self.count = buf, int(offset), int(count)
        self.device_address = buf.device_address + 8 * self.offset

    def numel(self) -> int:
        return self.count

    def numpy(self) -> np.ndarray:
        return self.buf.array()[self.offset:self.offset + self.count]


class MappedBuffer:
    """hc_mapped_alloc: pinned host memory the kernels write straight into."""

    def __init__(self, count: int):
        h, d = _vp(), _vp()
        _check(lib().hc_mapped_alloc(8 * int(count), ctypes.byref(h), ctypes.byref(d)), "hc_mapped_alloc")
        self._h = h
        self.count = int(count)
        self.device_address = d.value
        self._arr = np.ctypeslib.as_array(ctypes.cast(h, ctypes.POINTER(ctypes.c_int64)), shape=(self.count,))

    def array(self) -> np.ndarray:
        """The buffer as int64 values (read after the writing searches completed)."""
        return self._arr

    def view(self, offset: int = 0, count: int | None = None) -> MappedView:
        count = self.count - offset if count is None else count
        if offset < 0 or count < 0 or offset + count > self.count:
            raise ValueError("view outside the buffer")
        return MappedView(self, offset, count)

    def free(self):
        if self._h is not None and _lib is not None:
            _lib.hc_mapped_free(self._h)
        self._h = None
        self._arr = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


HC_MODE_AUTO = 0
HC_MODE_STAGED = 1
HC_MODE_DIRECT = 2
HC_MODE_DENSE = 3

HC_TUNE_BATCHED = 0
HC_TUNE_SINGLE = 1


class SearchOpts(ctypes.Structure):
    """hc_search_opts (zero = automatic)."""
    _fields_ = [("struct_size", ctypes.c_size_t), ("lane_bytes", ctypes.c_int),
                ("stages", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("mode", ctypes.c_int), ("spill_entries", ctypes.c_uint64),
                ("speculate", ctypes.c_int), ("pos32", ctypes.c_int),
                ("single_pass", ctypes.c_int), ("tile_steps", ctypes.c_int), ("sentinel", ctypes.c_int),
                ("bitmap", ctypes.c_int)]

    def __init__(self, lane_bytes=0, stages=0, ctas_per_sm=0, spill_entries=0, mode=0,
                 speculate=0, pos32=0, single_pass=0, tile_steps=0, sentinel=0, bitmap=0):
        super().__init__(ctypes.sizeof(SearchOpts), int(lane_bytes), int(stages),
                         int(ctas_per_sm), int(mode), int(spill_entries), int(speculate), int(pos32),
                         int(single_pass), int(tile_steps), int(sentinel), int(bitmap))


class HCFilter:
    """An hc_filter: the result of the preprocessing phase (Sec. 3.1)."""

    def __init__(self, handle: ctypes.c_void_p, x: bytes):
        self._h = handle
        self.x = x

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("filter has been freed")
        return self._h

    def params(self):
        m, q, a, s = _sz(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().hc_filter_params(self.handle, ctypes.byref(m), ctypes.byref(q),
                                      ctypes.byref(a), ctypes.byref(s)), "hc_filter_params")
        return {"m": m.value, "q": q.value, "alpha": a.value, "s": s.value}

    def words(self):
        """(F as a uint32 numpy copy, H_v)."""
        p = ctypes.POINTER(ctypes.c_uint32)()
        nw, hv = _sz(), ctypes.c_uint32()
        _check(lib().hc_filter_words(self.handle, ctypes.byref(p), ctypes.byref(nw),
                                     ctypes.byref(hv)), "hc_filter_words")
        return np.ctypeslib.as_array(p, shape=(nw.value,)).copy(), hv.value

    def to_device(self):
        _check(lib().hc_filter_to_device(self.handle), "hc_filter_to_device")

    def free(self):
        if self._h is not None and _lib is not None:
            _lib.hc_filter_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def hc_preprocess(x, q: int, alpha: int) -> HCFilter:
    """hc_preprocess(x, m, q, alpha): the filter of pattern x (host bytes)."""
    xb = _bytes_arg(x)
    out = _vp()
    buf = ctypes.create_string_buffer(xb, len(xb)) if xb else None
    _check(lib().hc_preprocess(ctypes.cast(buf, _vp) if buf is not None else None, len(xb),
                               int(q), int(alpha), ctypes.byref(out)), "hc_preprocess")
    return HCFilter(out, xb)


def hc_search_async(f: HCFilter, y_dev, pos_dev, count_dev, n: int | None = None,
                    cap: int | None = None, stream=None) -> None:
    """hc_search_async: enqueue the search of y_dev (uint8 CUDA tensor) on
    ``stream``; positions go to pos_dev (int64 CUDA tensor holding uint64
    values, or None), the total to count_dev (int64 CUDA tensor, 1 element)."""
    n = _text_len(y_dev, n)
    cap = _cap_for(pos_dev, cap, 8)
    _check_count(count_dev)
    _check(lib().hc_search_async(f.handle, _dev_ptr(y_dev), n, _dev_ptr(pos_dev), int(cap),
                                 _dev_ptr(count_dev), _stream_handle(stream)),
           "hc_search_async")


def hc_search_ex(f: HCFilter, y_dev, pos_dev, count_dev, opts: SearchOpts | None = None,
                 n: int | None = None, cap: int | None = None, stream=None) -> None:
    """hc_search_ex: hc_search_async with explicit launch options (with
    opts.pos32 = 1 the positions are uint32 values and cap counts those)."""
    n = _text_len(y_dev, n)
    # (a pos32 value other than 0 or 1 is the library's to reject)
    cap = _cap_for(pos_dev, cap, 4 if opts is not None and opts.pos32 != 0 else 8)
    _check_count(count_dev)
    _check(lib().hc_search_ex(f.handle, _dev_ptr(y_dev), n, _dev_ptr(pos_dev), int(cap),
                              _dev_ptr(count_dev),
                              ctypes.byref(opts) if opts is not None else None,
                              _stream_handle(stream)), "hc_search_ex")


def hc_search(f: HCFilter, x, y_dev, pos_dev=None, cap: int | None = None, stream=None,
              n: int | None = None, allow_truncated: bool = False):
    """hc_search(filter, x, y, n): synchronous search; returns the total count.

    Writes the first min(count, cap) positions into pos_dev.  Raises HCError
    with code HC_ERR_CAPACITY if the count exceeds cap (after writing them),
    unless ``allow_truncated`` is set (e.g. cap = 0 to size a buffer)."""
    n = _text_len(y_dev, n)
    cap = _cap_for(pos_dev, cap, 8)
    xb = _bytes_arg(x)
    cnt = _sz()
    xbuf = ctypes.create_string_buffer(xb, len(xb))
    rc = lib().hc_search(f.handle, ctypes.cast(xbuf, _vp), _dev_ptr(y_dev), n,
                         _dev_ptr(pos_dev), int(cap), ctypes.byref(cnt), _stream_handle(stream))
    if not (allow_truncated and rc == HC_ERR_CAPACITY):
        _check(rc, "hc_search")
    return cnt.value


def search_positions(f: HCFilter, x, y_dev, stream=None):
    """All occurrence positions of x in y_dev as an int64 CUDA tensor: one
    counting call (cap = 0), then one call into a buffer of that size."""
    import torch
    count = hc_search(f, x, y_dev, None, 0, stream, allow_truncated=True)
    pos = torch.empty(max(count, 1), dtype=torch.int64, device=y_dev.device)
    count2 = hc_search(f, x, y_dev, pos, count, stream)
    assert count2 == count
    return pos[:count]


def hc_search_noalloc(f: HCFilter, F_dev, x_dev, y_dev, pos_dev, count_dev,
                      cap: int | None = None, n: int | None = None, stream=None) -> None:
    """hc_search_noalloc: the search with every buffer supplied by the caller
    (F_dev: the filter's words, x_dev: the pattern, both on the device); the
    library allocates nothing."""
    n = _text_len(y_dev, n)
    cap = _cap_for(pos_dev, cap, 8)
    _check_count(count_dev)
    prm = f.params()
    if F_dev is None or _nbytes(F_dev) < 4 << prm["alpha"]:
        raise ValueError(f"F_dev must hold the filter's {1 << prm['alpha']} words")
    if x_dev is None or _nbytes(x_dev) < prm["m"]:
        raise ValueError(f"x_dev must hold the pattern's {prm['m']} bytes")
    _check(lib().hc_search_noalloc(f.handle, _dev_ptr(F_dev), _dev_ptr(x_dev), _dev_ptr(y_dev), n,
                                   _dev_ptr(pos_dev), int(cap), _dev_ptr(count_dev),
                                   _stream_handle(stream)), "hc_search_noalloc")


class BatchQuery(ctypes.Structure):
    """hc_batch_query."""
    _fields_ = [("x_dev", _vp), ("m", ctypes.c_uint64), ("y_dev", _vp), ("n", ctypes.c_uint64),
                ("q", ctypes.c_int), ("alpha", ctypes.c_int), ("pos_dev", _vp),
                ("cap", ctypes.c_uint64), ("count_dev", _vp), ("lane_bytes", ctypes.c_int),
                ("mode", ctypes.c_int), ("sigma", ctypes.c_int), ("reserved", ctypes.c_int)]


class TuneEntry(ctypes.Structure):
    """hc_tune_entry."""
    _fields_ = [("sigma", ctypes.c_int), ("q", ctypes.c_int), ("alpha", ctypes.c_int),
                ("lane_bytes", ctypes.c_int), ("mode", ctypes.c_int), ("sentinel", ctypes.c_int),
                ("bitmap", ctypes.c_int), ("m", ctypes.c_uint64), ("gbps", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k in ("sigma", "m", "q", "alpha", "lane_bytes", "mode", "gbps",
                                              "sentinel", "bitmap")}


class HCTuner:
    """An hc_tuner: search parameters per (alphabet size, pattern length)
    cell, measured on this GPU by calibrate(); lookups on an empty table give
    the paper's (q, alpha)."""

    def __init__(self):
        h = _vp()
        _check(lib().hc_tuner_create(ctypes.byref(h)), "hc_tuner_create")
        self._h = h

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("tuner has been freed")
        return self._h

    def calibrate(self, sigmas, ms, text_bytes=256 << 20, seed=1, path=0, stream=None):
        """path: HC_TUNE_BATCHED (0, the batched kernels) or HC_TUNE_SINGLE (1)."""
        sa = (ctypes.c_int * len(sigmas))(*[int(v) for v in sigmas])
        ma = (ctypes.c_uint64 * len(ms))(*[int(v) for v in ms])
        _check(lib().hc_tuner_calibrate(self.handle, sa, len(sigmas), ma, len(ms), int(text_bytes),
                                        int(seed), int(path), _stream_handle(stream)),
               "hc_tuner_calibrate")

    def lookup(self, sigma: float, m: int) -> dict:
        e = TuneEntry()
        _check(lib().hc_tuner_lookup(self.handle, float(sigma), int(m), ctypes.byref(e)),
               "hc_tuner_lookup")
        return e.as_dict()

    def entries(self) -> list:
        n = _sz()
        _check(lib().hc_tuner_size(self.handle, ctypes.byref(n)), "hc_tuner_size")
        out = []
        for i in range(n.value):
            e = TuneEntry()
            _check(lib().hc_tuner_entry(self.handle, i, ctypes.byref(e)), "hc_tuner_entry")
            out.append(e.as_dict())
        return out

    def save(self, path: str):
        _check(lib().hc_tuner_save(self.handle, os.fsencode(path)), "hc_tuner_save")

    def load(self, path: str):
        _check(lib().hc_tuner_load(self.handle, os.fsencode(path)), "hc_tuner_load")

    def free(self):
        if self._h is not None and _lib is not None:
            _lib.hc_tuner_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def hc_tuner_create() -> HCTuner:
    return HCTuner()


class HCBatch:
    """An hc_batch: a planned table of (pattern, text) queries.

    queries: list of dicts with keys x_dev, y_dev (uint8 CUDA tensors), q,
    alpha, pos_dev (int64 CUDA tensor or None), count_dev (int64 CUDA tensor
    of one element) and optionally cap, lane_bytes, mode, sigma.  q = 0 (or
    absent) takes the parameters from ``tuner`` (the paper's tables without
    one).  The tensors must stay alive while the batch exists."""

    def __init__(self, queries, tuner: HCTuner | None = None):
        n = len(queries)
        arr = (BatchQuery * max(n, 1))()
        for i, d in enumerate(queries):
            pos = d.get("pos_dev")
            arr[i].x_dev = _dev_ptr(d["x_dev"])
            arr[i].m = _nbytes(d["x_dev"])
            arr[i].y_dev = _dev_ptr(d["y_dev"])
            arr[i].n = _text_len(d["y_dev"], d.get("n"))
            arr[i].q = int(d.get("q", 0))
            arr[i].alpha = int(d.get("alpha", 0))
            arr[i].sigma = int(d.get("sigma", 0))
            arr[i].pos_dev = _dev_ptr(pos) if pos is not None else None
            arr[i].cap = _cap_for(pos, d.get("cap"), 8)
            arr[i].count_dev = _dev_ptr(d["count_dev"])
            arr[i].lane_bytes = int(d.get("lane_bytes", 0))
            arr[i].mode = int(d.get("mode", 0))
        self._keep = (arr, queries)
        h = _vp()
        if tuner is None:
            _check(lib().hc_batch_create(ctypes.cast(arr, _vp), n, ctypes.byref(h)), "hc_batch_create")
        else:
            _check(lib().hc_batch_create_tuned(ctypes.cast(arr, _vp), n, tuner.handle, ctypes.byref(h)),
                   "hc_batch_create_tuned")
        self._h = h
        self._tuner = tuner

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("batch has been destroyed")
        return self._h

    def run(self, stream=None):
        _check(lib().hc_batch_run(self.handle, _stream_handle(stream)), "hc_batch_run")

    def info(self):
        t, r, w = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(lib().hc_batch_info(self.handle, ctypes.byref(t), ctypes.byref(r), ctypes.byref(w)),
               "hc_batch_info")
        return {"tiles": t.value, "records": r.value, "workspace_bytes": w.value}

    def params(self, i: int) -> dict:
        """The (q, alpha, lane_bytes, mode) query i runs with."""
        e = TuneEntry()
        _check(lib().hc_batch_params(self.handle, i, ctypes.byref(e)), "hc_batch_params")
        d = e.as_dict()
        return {k: d[k] for k in ("q", "alpha", "lane_bytes", "mode")}

    def filter(self, i: int, alpha: int):
        F = np.zeros(1 << alpha, dtype=np.uint32)
        hv = ctypes.c_uint32()
        _check(lib().hc_batch_filter(self.handle, i, F.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                     F.size, ctypes.byref(hv)), "hc_batch_filter")
        return F, hv.value

    def destroy(self):
        if self._h is not None and _lib is not None:
            _lib.hc_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class ServerConfig(ctypes.Structure):
    """hc_server_config (zero = default)."""
    _fields_ = [("struct_size", _sz), ("mem_limit", ctypes.c_uint64), ("max_inflight", ctypes.c_int),
                ("max_batch", ctypes.c_int), ("default_cap", ctypes.c_uint64), ("plain", ctypes.c_int),
                ("batch_only", ctypes.c_int), ("max_batch_bytes", ctypes.c_uint64)]

    def __init__(self, mem_limit=0, max_inflight=0, max_batch=0, default_cap=0, plain=0,
                 batch_only=0, max_batch_bytes=0):
        super().__init__(ctypes.sizeof(ServerConfig), mem_limit, max_inflight, max_batch, default_cap,
                         plain, batch_only, max_batch_bytes)


class ServerRequest(ctypes.Structure):
    """hc_server_request."""
    _fields_ = [("text", ctypes.c_uint32), ("q", ctypes.c_int), ("alpha", ctypes.c_int),
                ("lane_bytes", ctypes.c_int), ("mode", ctypes.c_int), ("x", _vp),
                ("m", ctypes.c_uint64), ("cap", ctypes.c_uint64)]


class ServerResult(ctypes.Structure):
    """hc_server_result."""
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int), ("text", ctypes.c_uint32),
                ("q", ctypes.c_int), ("alpha", ctypes.c_int), ("count", ctypes.c_uint64),
                ("npos", ctypes.c_uint64), ("pos", ctypes.POINTER(ctypes.c_uint64)),
                ("submit_ns", ctypes.c_uint64), ("start_ns", ctypes.c_uint64),
                ("done_ns", ctypes.c_uint64), ("batch", ctypes.c_uint64),
                ("batch_size", ctypes.c_uint64)]


class ServerStats(ctypes.Structure):
    """hc_server_stats."""
    _fields_ = [(k, ctypes.c_uint64) for k in (
        "submitted", "completed", "batches", "rejected", "admission_waits", "max_batch", "pending",
        "inflight_bytes", "peak_inflight_bytes", "text_bytes", "mem_limit")]


class HCServer:
    """An hc_server: resident texts, a request queue and a worker thread that
    runs queued requests as batches on up to max_inflight streams."""

    def __init__(self, config: ServerConfig | None = None, tuner: HCTuner | None = None):
        h = _vp()
        _check(lib().hc_server_create(ctypes.byref(config) if config is not None else None,
                                      tuner.handle if tuner is not None else None, ctypes.byref(h)),
               "hc_server_create")
        self._h = h
        self._keep = [tuner]

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("server has been destroyed")
        return self._h

    def add_text(self, y, sigma: int = 0) -> int:
        """Registers a text: a uint8 CUDA tensor (kept by reference; it must
        outlive the server) or host bytes / numpy array (copied)."""
        tid = ctypes.c_uint32()
        if hasattr(y, "is_cuda") and y.is_cuda:
            self._keep.append(y)
            _check(lib().hc_server_add_text(self.handle, _dev_ptr(y), _nbytes(y), 1, int(sigma),
                                            ctypes.byref(tid)), "hc_server_add_text")
        else:
            b = _bytes_arg(y)
            buf = ctypes.create_string_buffer(b, len(b)) if b else None
            _check(lib().hc_server_add_text(self.handle, ctypes.cast(buf, _vp) if buf is not None else None,
                                            len(b), 0, int(sigma), ctypes.byref(tid)), "hc_server_add_text")
        return tid.value

    def text_info(self, text_id: int) -> dict:
        n, sg = ctypes.c_uint64(), ctypes.c_double()
        _check(lib().hc_server_text_info(self.handle, int(text_id), ctypes.byref(n), ctypes.byref(sg)),
               "hc_server_text_info")
        return {"n": n.value, "sigma": sg.value}

    @staticmethod
    def _request(text_id, x, q=0, alpha=0, cap=0, lane_bytes=0, mode=0):
        xb = _bytes_arg(x)
        buf = ctypes.create_string_buffer(xb, len(xb)) if xb else None
        r = ServerRequest(int(text_id), int(q), int(alpha), int(lane_bytes), int(mode),
                          ctypes.cast(buf, _vp) if buf is not None else None, len(xb), int(cap))
        return r, buf

    def submit(self, text_id: int, x, q: int = 0, alpha: int = 0, cap: int = 0, lane_bytes: int = 0,
               mode: int = 0) -> int:
        r, buf = self._request(text_id, x, q, alpha, cap, lane_bytes, mode)
        rid = ctypes.c_uint64()
        _check(lib().hc_server_submit(self.handle, ctypes.byref(r), ctypes.byref(rid)), "hc_server_submit")
        return rid.value

    def replay(self, requests, arrival_s) -> list:
        """requests: list of (text_id, x[, q, alpha, cap]); arrival_s: their
        arrival offsets in seconds (non-decreasing).  Submits each at its time
        from this thread (the GIL is released) and returns the ids."""
        n = len(requests)
        arr = (ServerRequest * max(n, 1))()
        keep = []
        for i, rq in enumerate(requests):
            r, buf = self._request(*rq)
            arr[i] = r
            keep.append(buf)
        t = (ctypes.c_uint64 * max(n, 1))(*[int(round(a * 1e9)) for a in arrival_s])
        ids = (ctypes.c_uint64 * max(n, 1))()
        _check(lib().hc_server_replay(self.handle, ctypes.cast(arr, _vp), n, t, ids), "hc_server_replay")
        return list(ids)[:n]

    def poll(self, max_results: int = 1024, wait_us: int = 0, positions: bool = True) -> list:
        """Completed results as dicts (positions copied to numpy uint64 and
        the library's copy released)."""
        out = (ServerResult * max_results)()
        got = _sz()
        _check(lib().hc_server_poll(self.handle, out, max_results, ctypes.byref(got), int(wait_us)),
               "hc_server_poll")
        res = []
        for i in range(got.value):
            r = out[i]
            d = {k: getattr(r, k) for k in ("id", "status", "text", "q", "alpha", "count", "npos",
                                            "submit_ns", "start_ns", "done_ns", "batch", "batch_size")}
            if positions:
                d["pos"] = (np.ctypeslib.as_array(r.pos, shape=(r.npos,)).copy() if r.npos
                            else np.zeros(0, np.uint64))
            _check(lib().hc_server_release(self.handle, r.id), "hc_server_release")
            res.append(d)
        return res

    def drain(self, timeout_ms: int = -1):
        _check(lib().hc_server_drain(self.handle, int(timeout_ms)), "hc_server_drain")

    def stats(self) -> dict:
        s = ServerStats()
        _check(lib().hc_server_get_stats(self.handle, ctypes.byref(s)), "hc_server_get_stats")
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}

    def destroy(self):
        if self._h is not None and _lib is not None:
            _lib.hc_server_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def hc_batch_create(queries) -> HCBatch:
    return HCBatch(queries)


def hc_batch_create_tuned(queries, tuner: HCTuner | None) -> HCBatch:
    """hc_batch_create_tuned; tuner None uses the paper's tables for q = 0."""
    return HCBatch(queries, tuner)


def hc_check_status(stream=None) -> None:
    _check(lib().hc_check_status(_stream_handle(stream)), "hc_check_status")


def hc_selftest_wait_timeout(stream=None) -> None:
    """Enqueues the self-test whose bounded device wait runs out (about 2 s);
    the next hc_check_status on the stream raises HC_ERR_TIMEOUT."""
    _check(lib().hc_selftest_wait_timeout(_stream_handle(stream)), "hc_selftest_wait_timeout")


def hc_kernel_launches() -> int:
    return int(lib().hc_kernel_launches())


def hc_timing_enable(on: bool = True) -> None:
    _check(lib().hc_timing_enable(1 if on else 0), "hc_timing_enable")


def hc_timing_report(reset: bool = True) -> dict:
    """{kernel family: (milliseconds, launches)} of the timed launches."""
    k = 16
    ms = (ctypes.c_double * k)()
    cnt = (ctypes.c_uint64 * k)()
    _check(lib().hc_timing_report(ms, cnt, k, 1 if reset else 0), "hc_timing_report")
    out = {}
    for i in range(k):
        name = lib().hc_timing_kind_name(i).decode()
        if name:
            out[name] = (float(ms[i]), int(cnt[i]))
    return out


def hc_version() -> int:
    return int(lib().hc_version())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libhc.so for sm_103a (see _build.py)."""
    return _build.build(force=force, verbose=verbose)
