"""The machine of Section 8 (one thread per node, c/n stamp vectors, one
launch per micro-iteration), kept as a prior-art comparison: it must decide
exactly what the oracle and the lockstep kernels decide."""
import numpy as np
import pytest

import oracle
import paper_1108_3126_b300 as rx
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1108_3126_b300 import build
    build.build()
    assert torch.cuda.is_available()


def run(r, s, variant):
    d = torch.from_numpy(np.concatenate([s.data, np.zeros(16, np.uint8)])).cuda()
    o = torch.from_numpy(s.offsets.copy()).cuda()
    out = torch.full((max(s.n, 1),), 7, dtype=torch.uint8, device="cuda")
    rx.match(r, d, o, out, n=s.n, variant=variant)
    torch.cuda.synchronize()
    return out[:s.n].cpu().numpy()


def test_paper_examples():
    for pat, strs in [(b"(a*)*b", [b"aab", b"b", b"", b"ab a"]),
                      (b"(a*)*", [b"", b"a", b"a" * 300 + b"b"]),
                      (b"((((\\e*)*)*|a)*)*b", [b"aaab", b"aaa"]),
                      (b"(ab)|(ac)", [b"ac", b"ab", b"aa"])]:
        s = synth.pack(strs)
        want = np.array([oracle.o2(oracle.parse(pat), w) for w in strs], np.uint8)
        assert (run(rx.Regex.compile(pat), s, rx.VARIANT_PAPER) == want).all(), pat


def test_paper_machine_random():
    for i in range(12):
        e = synth.gen_regex(10 + 4 * i, 8, b"abc", synth.item_seed(0xA0, i), eps_loop_p=0.1)
        s = synth.gen_strings(e, 12, 0, 40, b"abc", synth.item_seed(0xA1, i), p_lang=0.5)
        want = oracle.o2_batch(e, s.data, s.offsets)
        r = rx.Regex.from_nodes(e)
        assert (run(r, s, rx.VARIANT_PAPER) == want).all(), synth.to_pattern(e)
        assert (run(r, s, 0) == want).all()
