"""rx_match_static: the no-allocation variant of rx_match.

Callers that cannot let the library allocate device memory (they must not
block on the device, or their device-memory budget is fixed) use this entry
point; its scratch is a fixed array inside the library.  This file is
collected last so that a run stopping at the first failure has already run
every other test; it passes both alone in a fresh process and after the
rest of the suite.
"""
import ctypes

import numpy as np
import pytest

import paper_1108_3126_b300 as rx
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1108_3126_b300 import build
    build.build()
    assert torch.cuda.is_available()


def call_static(r, d, o, out, n, stream=None):
    """Straight through the C ABI symbol."""
    st = (stream or torch.cuda.current_stream()).cuda_stream
    return rx.lib().rx_match_static(ctypes.c_void_p(r.handle), n, ctypes.c_void_p(d.data_ptr()),
                                    ctypes.c_void_p(o.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(st))


def case(w):
    s = w.strings
    return (rx.Regex.from_nodes(w.regexes[0]), torch.from_numpy(s.data).cuda(), torch.from_numpy(s.offsets).cuda(),
            s.n)


def test_static_matches_rx_match_on_two_calls_in_a_row():
    """On a stream that rx_match never saw (so no per-stream scratch of
    rx_match exists for it), two rounds of calls give rx_match's results,
    and the device's free memory does not change across them: nothing is
    allocated."""
    cases = [case(synth.cfg_small()), case(synth.cfg_streaming(n=200000))]
    wants = []
    for r, d, o, n in cases:
        want = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
        rx.match(r, d, o, want, n=n)
        wants.append(want)
    gots = [torch.full((n,), 9, dtype=torch.uint8, device="cuda") for _, _, _, n in cases]
    fresh = torch.cuda.Stream()
    # a first call loads the library's module holding the array (the driver
    # places it when the module is loaded) and looks up its address
    r, d, o, n = cases[0]
    assert call_static(r, d, o, gots[0], n, fresh) == 0, rx.last_error()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for rnd in range(2):
        # the second round in the other order: the shared array keeps the
        # previous call's contents, which must not leak into the next result
        order = range(len(cases)) if rnd == 0 else reversed(range(len(cases)))
        for k in order:
            r, d, o, n = cases[k]
            gots[k].fill_(9)
            assert call_static(r, d, o, gots[k], n, fresh) == 0, rx.last_error()
            fresh.synchronize()
            assert torch.equal(gots[k], wants[k]), (rnd, k)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_static_rejects_batches_over_the_limit():
    r = rx.Regex.compile(b"a*")
    s = synth.pack([b"a"] * 262145)
    d, o = torch.from_numpy(s.data).cuda(), torch.from_numpy(s.offsets).cuda()
    out = torch.full((s.n,), 9, dtype=torch.uint8, device="cuda")
    assert call_static(r, d, o, out, s.n) == 3  # RX_ERR_TOO_LARGE
    assert "262144" in rx.last_error()
    torch.cuda.synchronize()
    assert int(out.max().item()) == 9  # nothing ran
    assert call_static(r, d, o, out, 262144) == 0
    torch.cuda.synchronize()
    assert int(out[:262144].min().item()) == 1
