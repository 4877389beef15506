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


def search_long(r, text: bytes, chunk=0):
    d = torch.from_numpy(np.frombuffer(text, np.uint8).copy() if text else np.zeros(1, np.uint8)).cuda()
    out = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    rx.search_long(r, d, len(text), out, chunk_bytes=chunk)
    torch.cuda.synchronize()
    return int(out.item())


def _rare_expressions():
    """Expressions that need the byte c (so a text over {a, b} has no match)
    -- fixed ones and random ones over {a, b, c} filtered that way."""
    pats = [b"c(a|b)*c", b"ca(a|b)*bc", b"(ab|ba)*cc", b"c(a|c)(a|b)", b"((a|b)c)*cc", b"(a*b*)*c(a|b)(a|b)c"]
    out = [oracle.parse(p) for p in pats]
    probe = bytes(np.random.default_rng(1).choice(list(b"ab"), size=3000).tolist())
    i = 0
    while len(out) < 16 and i < 400:
        nodes = synth.gen_regex([8, 16, 30][i % 3], 8, b"abc", synth.item_seed(0xEB, i), eps_loop_p=0.05)
        i += 1
        if oracle.o2_search(nodes, probe) == -1 and oracle.o2_search(nodes, probe + b"c" * 8 + probe) != -1:
            out.append(nodes)
    return out


def test_search_long_chunk_sizes_vs_oracle():
    """Chunked search of texts over {a, b} up to 300 KB with matches of
    c-requiring expressions planted across chunk boundaries, near the end,
    at random, or absent; every chunk size agrees with the streaming oracle
    and with the one-string kernel."""
    rng = np.random.default_rng(0xE8)
    for i, nodes in enumerate(_rare_expressions()):
        r = rx.Regex.from_nodes(nodes, 0, rx.COMPILE_SEARCH)
        if r.info()["search_states"] == 0:
            continue
        sample = synth.gen_strings(nodes, 8, 1, 40, b"abc", synth.item_seed(0xEA, i), p_lang=1.0)
        for trial in range(4):
            L = int(rng.integers(1000, 300000))
            text = bytes(rng.choice(list(b"ab"), size=L).tolist())
            w = sample.get(trial) if sample.n > trial else b"cc"
            if trial == 0:    # across a 1000-byte and a 4096-byte boundary
                p = (L // 4096000) * 4096000 + 4096 * max(1, L // 8192) - len(w) // 2
                p = min(max(p, 0), L)
                text = text[:p] + w + text[p:]
            elif trial == 1:  # near the end
                text = text[:-20] + w + text[-20:]
            elif trial == 2:  # at random, twice
                for _ in range(2):
                    p = int(rng.integers(0, len(text)))
                    text = text[:p] + w + text[p:]
            want = oracle.o2_search(nodes, text)
            if trial < 3:
                assert want > 0
            for chunk in (64, 100, 1000, 4096, 0):
                got = search_long(r, text, chunk)
                assert got == want, (synth.to_pattern(nodes)[:60], trial, chunk, got, want)
            assert run_search(r, synth.pack([text]))[0] == want


def test_search_long_edges():
    r = rx.Regex.compile(b"ab", rx.COMPILE_SEARCH)
    assert search_long(r, b"") == -1
    assert search_long(rx.Regex.compile(b"a*", rx.COMPILE_SEARCH), b"") == 0
    assert search_long(r, b"x" * 5000 + b"ab") == 5002
    assert search_long(r, b"x" * 4095 + b"ab" + b"x" * 9000, 4096) == 4097  # across a chunk boundary
    assert search_long(r, b"x" * 5000, 64) == -1
    with pytest.raises(rx.RxError) as ei:
        search_long(r, b"abc", 10)  # chunk below 64 bytes
    assert ei.value.status == 2


def test_search_long_full_size_literal():
    """1 GiB of the long-text workload searched for a literal placed near
    the end (its first occurrence found by bytes.find)."""
    nodes, text, end = synth.cfg_long(total=1 << 30, with_end=True)
    t = text.tobytes()
    lit = b"zqzqzq"
    k = t.find(lit)
    if k < 0:
        p = len(t) - 1000
        t = t[:p] + lit + t[p + len(lit):]
        k = t.find(lit)
    r = rx.Regex.compile(lit, rx.COMPILE_SEARCH)
    assert search_long(r, t) == k + len(lit)
    # and the workload's own expression: a match ends early
    r2 = rx.Regex.from_nodes(nodes, 0, rx.COMPILE_SEARCH)
    if r2.info()["search_states"]:
        want = oracle.o2_search(nodes, t[:200000])
        assert want >= 0  # the text is made of the expression's samples
        assert search_long(r2, t) == want


def test_rare_matches_vs_oracle():
    """Batch search where matches are rare: strings over {a, b} for
    expressions that need the byte c, with c-containing samples planted in
    some strings at random places (answers spread over the whole length)."""
    rng = np.random.default_rng(0xEC)
    for i, nodes in enumerate(_rare_expressions()):
        r = rx.Regex.from_nodes(nodes, 0, rx.COMPILE_SEARCH)
        if r.info()["search_states"] == 0:
            continue
        sample = synth.gen_strings(nodes, 50, 1, 30, b"abc", synth.item_seed(0xED, i), p_lang=1.0)
        strs = []
        for k in range(400):
            L = int(rng.integers(0, 3000))
            t = bytes(rng.choice(list(b"ab"), size=L).tolist())
            if k % 3:
                p = int(rng.integers(0, L + 1))
                t = t[:p] + sample.get(k % sample.n) + t[p:]
            strs.append(t)
        pk = synth.pack(strs)
        want = oracle.o2_search_batch(nodes, pk.data, pk.offsets)
        assert (want > 100).sum() > 100  # answers far into the strings
        got = run_search(r, pk)
        assert (got == want).all(), (synth.to_pattern(nodes)[:60], np.nonzero(got != want)[0][:8])
