"""Host-side argument checks of the server API (no GPU): a configuration of
the wrong size or out of range, a foreign tuner handle and NULL handles are
rejected before any device work."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def hc():
    import paper_2310_15711_gb300 as hc
    hc.build()
    hc.lib()
    return hc


def test_bad_configs_rejected(hc):
    L = hc.lib()
    out = ctypes.c_void_p()
    cfg = hc.ServerConfig()
    cfg.struct_size = 8
    assert L.hc_server_create(ctypes.byref(cfg), None, ctypes.byref(out)) == hc.HC_ERR_ARG
    for kw in (dict(max_inflight=17), dict(max_inflight=-1), dict(max_batch=-5),
               dict(max_batch=(1 << 20) + 1), dict(default_cap=(1 << 32) + 1)):
        cfg = hc.ServerConfig(**kw)
        assert L.hc_server_create(ctypes.byref(cfg), None, ctypes.byref(out)) == hc.HC_ERR_ARG, kw
    assert out.value is None
    assert L.hc_server_create(None, None, None) == hc.HC_ERR_ARG
    # a handle that is not a tuner
    junk = ctypes.create_string_buffer(64)
    assert L.hc_server_create(None, ctypes.cast(junk, ctypes.c_void_p), ctypes.byref(out)) == hc.HC_ERR_ARG


def test_null_server_rejected(hc):
    L = hc.lib()
    got = ctypes.c_size_t()
    rid = ctypes.c_uint64()
    tid = ctypes.c_uint32()
    assert L.hc_server_add_text(None, None, 0, 0, 0, ctypes.byref(tid)) == hc.HC_ERR_ARG
    assert L.hc_server_submit(None, None, ctypes.byref(rid)) == hc.HC_ERR_ARG
    assert L.hc_server_poll(None, None, 0, ctypes.byref(got), 0) == hc.HC_ERR_ARG
    assert L.hc_server_release(None, 1) == hc.HC_ERR_ARG
    assert L.hc_server_drain(None, 0) == hc.HC_ERR_ARG
    assert L.hc_server_get_stats(None, None) == hc.HC_ERR_ARG
    assert L.hc_server_replay(None, None, 0, None, None) == hc.HC_ERR_ARG
    L.hc_server_destroy(None)


def test_config_struct_matches_the_header(hc):
    """The binding's hc_server_config has the header's layout, including the
    per-batch text bound (max_batch_bytes, last member); a configuration with
    every field set is accepted by hc_server_create's checks (the server is
    only created where a device exists)."""
    import ctypes as C
    fields = [f for f, _ in hc.ServerConfig._fields_]
    assert fields[-1] == "max_batch_bytes"
    cfg = hc.ServerConfig(max_batch_bytes=123 << 20, max_batch=10, max_inflight=4)
    assert cfg.max_batch_bytes == 123 << 20 and cfg.struct_size == C.sizeof(hc.ServerConfig)
    # the header's struct: size_t, u64, int, int, u64, int, int, u64
    assert C.sizeof(hc.ServerConfig) == 8 + 8 + 4 + 4 + 8 + 4 + 4 + 8
