"""Failure detection on the GPU without a fault: a device-side wait that
runs out.  The self-test kernel waits, with the library's bounded wait, on
an mbarrier that nothing completes; the wait gives up after about 2 s and
sets the status flag exactly as a stalled bulk copy would.  The host must
read HC_ERR_TIMEOUT, the flag must be cleared by that read, and the context
must stay usable: a search right afterwards still equals the oracle."""
import time

import numpy as np
import pytest

import hc_inputs as hi
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


def test_bounded_wait_runs_out_and_the_context_stays_usable(hc):
    hc.hc_check_status()                       # nothing pending before
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    hc.hc_selftest_wait_timeout(stream)
    stream.synchronize()
    waited = time.perf_counter() - t0
    with pytest.raises(hc.HCError) as ei:
        hc.hc_check_status(stream)
    assert ei.value.code == hc.HC_ERR_TIMEOUT
    assert 1.0 < waited < 60.0                 # the 2 s limit, not an early return
    hc.hc_check_status(stream)                 # the read cleared the flag
    # the context still works: an exact search right afterwards
    y = hi.uniform_text(1 << 20, 4, seed=11)
    x, _ = hi.extract_pattern(y, 12, np.random.default_rng(5))
    f = hc.hc_preprocess(x, 4, 12)
    pos = hc.search_positions(f, x, torch.from_numpy(y).cuda())
    got = pos.cpu().numpy().view(np.uint64)
    assert np.array_equal(got, oracle.hc_search(x, y, 4, 12))
    hc.hc_check_status()
    f.free()
