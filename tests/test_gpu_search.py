"""GPU parity of unanchored search (rx_search): the earliest end of a
substring the expression matches, against the CPU oracle's search read off
the big-step tables (oracle.o1_search).  Exact integers."""
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


def run_search(r, s: synth.Strings):
    d = torch.from_numpy(np.ascontiguousarray(s.data if s.data.size else np.zeros(1, np.uint8))).cuda()
    o = torch.from_numpy(np.ascontiguousarray(s.offsets)).cuda()
    out = torch.full((max(s.n, 1),), -7, dtype=torch.int64, device="cuda")
    rx.search(r, d, o, out, n=s.n)
    torch.cuda.synchronize()
    return out[:s.n].cpu().numpy()


def embedded(nodes, n, lmax, alpha, seed):
    """Random text over alpha with a language sample of the expression
    spliced in at a random place in about half of the strings."""
    rng = np.random.default_rng(seed)
    lang = synth.gen_strings(nodes, n, 0, max(lmax // 4, 1), alpha, seed + 1, p_lang=1.0)
    out = []
    for i in range(n):
        L = int(rng.integers(0, lmax))
        t = bytes(rng.choice(np.frombuffer(alpha, np.uint8), size=L).tolist())
        if i % 2 == 0:
            p = int(rng.integers(0, L + 1))
            t = t[:p] + lang.get(i) + t[p:]
        out.append(t)
    return synth.pack(out)


def test_random_expressions_vs_oracle():
    for i in range(40):
        alpha = [b"abc", synth.LOWER, b"ab"][i % 3]
        nodes = synth.gen_regex([3, 8, 16, 40][i % 4], 8, alpha, synth.item_seed(0xE0, i), eps_loop_p=0.05)
        r = rx.Regex.from_nodes(nodes, 0, rx.COMPILE_SEARCH)
        if r.info()["search_states"] == 0:
            continue
        s = embedded(nodes, 200, 300, alpha, synth.item_seed(0xE1, i))
        want = oracle.o1_search_batch(nodes, s.data, s.offsets)
        assert (want >= -1).all()
        got = run_search(r, s)
        assert (got == want).all(), (synth.to_pattern(nodes)[:60], np.nonzero(got != want)[0][:8])


def test_edge_cases_and_closed_forms():
    strs = [b"", b"a", b"ab", b"xxab", b"aab", b"ba", b"abab", b"x" * 1000 + b"ab", b"x" * 999]
    s = synth.pack(strs)
    cases = [(b"ab", [-1, -1, 2, 4, 3, -1, 2, 1002, -1]),
             (b"a*", [0] * 9),
             (b"\\e", [0] * 9),
             (b"(a*)*b", [-1, -1, 2, 4, 3, 1, 2, 1002, -1]),
             (b"x(x|a|b)*x", [-1, -1, -1, 2, -1, -1, -1, 2, 2])]
    for pat, want in cases:
        r = rx.Regex.compile(pat, rx.COMPILE_SEARCH)
        assert (run_search(r, s) == np.array(want)).all(), pat
        assert (oracle.o1_search_batch(oracle.parse(pat), s.data, s.offsets) == np.array(want)).all(), pat
    # empty batch
    r = rx.Regex.compile(b"ab", rx.COMPILE_SEARCH)
    assert run_search(r, synth.pack([])).size == 0


def test_full_size_streaming_batch_sampled():
    """The 1,048,576-string streaming batch searched with its 64-node
    expression, in the launch configuration of the full-size run; a sample
    checked against the oracle, and literal search by closed form."""
    w = synth.cfg_streaming()
    nodes = w.regexes[0]
    r = rx.Regex.from_nodes(nodes, 0, rx.COMPILE_SEARCH)
    assert r.info()["search_states"] > 0
    got = run_search(r, w.strings)
    rng = np.random.default_rng(4)
    idx = np.sort(rng.choice(w.strings.n, 1500, replace=False))
    sub = synth.pack([w.strings.get(int(i)) for i in idx])
    want = oracle.o1_search_batch(nodes, sub.data, sub.offsets)
    assert (got[idx] == want).all()
    # literal: earliest end of "qz" by str.find, on every string
    lit = rx.Regex.compile(b"qz", rx.COMPILE_SEARCH)
    g2 = run_search(lit, w.strings)
    for i in rng.choice(w.strings.n, 20000, replace=False):
        t = w.strings.get(int(i))
        k = t.find(b"qz")
        assert g2[i] == (k + 2 if k >= 0 else -1)


def test_unsupported_without_flag():
    r = rx.Regex.compile(b"ab")
    with pytest.raises(rx.RxError) as ei:
        run_search(r, synth.pack([b"ab"]))
    assert ei.value.status == 8
    assert r.info()["search_states"] == 0
