"""Host-side checks of the C-ABI library (no GPU needed).

* libhc.so loads and exports every function that include/hc.h declares, and
  the binding registers exactly those names.
* hc_preprocess (host code of the library) builds the same F and H_v as the
  oracle's Fig. 4 preprocessing, word for word.
* Invalid arguments are rejected with HC_ERR_ARG.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_2310_15711_gb300 as hc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    hc.build()


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for mt in re.finditer(r"^[A-Za-z_][\w \*]*?\b(hc_\w+)\s*\(", src, flags=re.M):
            names.add(mt.group(1))
    return names


def test_library_exports_every_declared_symbol():
    declared = _declared_functions()
    assert {"hc_preprocess", "hc_search", "hc_search_async", "hc_filter_free"} <= declared
    L = ctypes.CDLL(hc.LIB_PATH)
    for name in declared:
        assert hasattr(L, name), name
    assert set(hc.SIGNATURES) == declared


def test_version_and_launch_counter():
    assert hc.hc_version() >= 100
    assert hc.hc_kernel_launches() >= 0


@pytest.mark.parametrize("sigma", [2, 4, 20, 95, 256])
def test_host_filter_equals_oracle_filter(sigma):
    rng = np.random.default_rng(sigma)
    for _ in range(150):
        m = int(rng.choice([1, 2, 3, 5, 8, 13, 16, 31, 64, 200, 1024]))
        q = int(rng.integers(1, min(m, 8) + 1))
        alpha = int(rng.integers(1, 16))
        x = rng.integers(0, sigma, m, dtype=np.uint16).astype(np.uint8) + (0 if sigma == 256 else 40)
        f = hc.hc_preprocess(x, q, alpha)
        F, hv = f.words()
        ref = oracle.preprocess(x, q, alpha)
        assert np.array_equal(F, ref["F"]), (m, q, alpha)
        assert hv == ref["hv"]
        p = f.params()
        assert p == {"m": m, "q": q, "alpha": alpha, "s": alpha // q}
        f.free()


def test_preprocess_rejects_invalid_arguments():
    for x, q, alpha in [(b"abc", 4, 10), (b"abc", 0, 10), (b"abcdefghij", 9, 10),
                        (b"abc", 2, 0), (b"abc", 2, 16), (b"", 1, 10)]:
        with pytest.raises(hc.HCError) as ei:
            hc.hc_preprocess(x, q, alpha)
        assert ei.value.code == hc.HC_ERR_ARG


def test_null_filter_is_rejected():
    L = hc.lib()
    assert L.hc_filter_words(None, None, None, None) == hc.HC_ERR_ARG
    assert L.hc_filter_params(None, None, None, None, None) == hc.HC_ERR_ARG
    assert L.hc_search_async(None, None, 0, None, 0, None, None) == hc.HC_ERR_ARG
    L.hc_filter_free(None)  # no-op


def test_check_bounds_refused_in_the_regular_build():
    import ctypes
    v = ctypes.c_uint64(7)
    assert hc.lib().hc_check_bounds(ctypes.byref(v)) == hc.HC_ERR_STATE
    assert v.value == 0
    assert hc.lib().hc_check_bounds(None) == hc.HC_ERR_ARG


def test_output_capacity_is_counted_in_bytes():
    """The binding derives a search's capacity from the output buffer's bytes
    and the position width (8, or 4 with uint32 positions), and refuses a cap
    the buffer cannot hold, so a narrow buffer is never overrun."""
    import torch
    hc = pytest.importorskip("paper_2310_15711_gb300")
    i64 = torch.zeros(10, dtype=torch.int64)
    i32 = torch.zeros(10, dtype=torch.int32)
    u8 = torch.zeros(64, dtype=torch.uint8)
    assert hc._cap_for(i64, None, 8) == 10 and hc._cap_for(i64, None, 4) == 20
    assert hc._cap_for(i32, None, 8) == 5 and hc._cap_for(i32, None, 4) == 10
    assert hc._cap_for(u8, None, 8) == 8 and hc._cap_for(u8[2:34], 4, 8) == 4
    assert hc._cap_for(None, 123, 8) == 0
    for buf, cap, width in ((i32, 6, 8), (i64, 21, 4), (u8, 9, 8), (i64, -1, 8)):
        with pytest.raises(ValueError):
            hc._cap_for(buf, cap, width)
    with pytest.raises(ValueError):
        hc._check_count(torch.zeros(4, dtype=torch.uint8))
    hc._check_count(torch.zeros(1, dtype=torch.int64))
    assert hc._nbytes(torch.zeros(3, dtype=torch.int32)) == 12


def test_text_length_must_fit_the_text_buffer():
    """An explicit text length larger than the text buffer is refused by the
    binding before any launch (the kernels would read n bytes), for every
    search entry point: they all take n through _text_len."""
    import torch
    hc = pytest.importorskip("paper_2310_15711_gb300")
    y = torch.zeros(100, dtype=torch.uint8)
    assert hc._text_len(y, None) == 100 and hc._text_len(y, 100) == 100 and hc._text_len(y, 0) == 0
    assert hc._text_len(torch.zeros(10, dtype=torch.int32), 40) == 40
    for bad in (101, -1, 1 << 40):
        with pytest.raises(ValueError):
            hc._text_len(y, bad)
    import inspect
    src = inspect.getsource(hc)
    assert "_nbytes(y_dev) if n is None" not in src
    for fn in (hc.hc_search_async, hc.hc_search_ex, hc.hc_search, hc.hc_search_noalloc):
        assert "_text_len(y_dev, n)" in inspect.getsource(fn), fn.__name__
