"""GPU parity of the chunked long-string mode (rx_match_long), the sequential
one-thread form (rx_match_seq), the persistent batched form
(rx_match_batch) and the plain one-launch-per-pair form (rx_match_pairs),
against the CPU oracle and against each other.  Exact booleans."""
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


def dev(a):
    return torch.from_numpy(np.array(a, copy=True)).cuda()


def long_match(r, d_text, n, chunk=0):
    out = torch.full((1,), 7, dtype=torch.uint8, device="cuda")
    rx.match_long(r, d_text, n, out, chunk_bytes=chunk)
    torch.cuda.synchronize()
    return int(out.item())


def seq_match(r, d_text, n):
    out = torch.full((1,), 7, dtype=torch.uint8, device="cuda")
    rx.match_seq(r, d_text, n, out)
    torch.cuda.synchronize()
    return int(out.item())


@pytest.fixture(scope="module")
def long_case():
    R = synth.long_regex()
    nodes = synth.wrap_star(R)
    assert synth.n_positions(nodes) == 48
    text, end = synth.star_text(R, 4 << 20, synth.item_seed(0xE0, 0), with_end=True)
    assert oracle.o2(nodes, text[:end].tobytes())
    return nodes, text


def test_long_text_chunk_sizes_vs_seq_and_o2(long_case):
    nodes, text = long_case
    variants = [text, text.copy()]
    variants[1][-1] = ord("a") if variants[1][-1] != ord("a") else ord("b")
    r_memo = rx.Regex.from_nodes(nodes)
    r_bits = rx.Regex.from_nodes(nodes, 0, rx.COMPILE_NO_MEMO)
    assert r_memo.info()["memo_states"] > 0 and r_bits.info()["memo_states"] == 0
    for t in variants:
        d = dev(t)
        n = len(t)
        # O2 on a 1 MiB prefix and on the whole text
        want_full = oracle.o2(nodes, t.tobytes())
        pre = 1 << 20
        want_pre = oracle.o2(nodes, t[:pre].tobytes())
        for r in (r_memo, r_bits):
            assert seq_match(r, d, n) == want_full
            assert seq_match(r, d, pre) == want_pre
            for chunk in (0, 7, 4096, 1 << 20, 3 << 20, n + 5):
                assert long_match(r, d, n, chunk) == want_full, (chunk, r.info()["memo_states"])
            assert long_match(r, d, pre, 1000) == want_pre
    # chunk size 1 on a shorter prefix (one chunk per byte)
    d = dev(text[:50000])
    w = oracle.o2(nodes, text[:50000].tobytes())
    assert long_match(r_memo, d, 50000, 1) == w
    assert long_match(r_bits, d, 50000, 1) == w


def test_long_chunk_size_bound(long_case):
    """chunk_bytes up to 2^32 - 33 is taken (one chunk for a short text),
    2^32 - 32 and above are rejected: a span's byte count, with the bytes
    before it in its first 32-byte block, must fit in 32 bits."""
    nodes, text = long_case
    r = rx.Regex.from_nodes(nodes)
    t = text[:100001]
    d = dev(t)
    assert long_match(r, d, len(t), (1 << 32) - 33) == oracle.o2(nodes, t.tobytes())
    for bad in ((1 << 32) - 32, 1 << 32):
        with pytest.raises(rx.RxError) as ei:
            long_match(r, d, len(t), bad)
        assert rx.STATUS[ei.value.status] == "RX_ERR_INVALID_ARG"


def test_long_random_expressions_and_edges():
    for i in range(30):
        alpha = [b"abc", synth.LOWER, synth.ALL_BYTES][i % 3]
        e = synth.gen_regex(10 + 7 * i, 10, alpha, synth.item_seed(0xE1, i), eps_loop_p=0.05)
        s = synth.gen_strings(e, 3, 0, 30000, alpha, synth.item_seed(0xE2, i), p_lang=0.7)
        for flags in (0, rx.COMPILE_NO_MEMO):
            r = rx.Regex.from_nodes(e, 0, flags)
            for k in range(s.n):
                w = s.get(k)
                want = oracle.o2(e, w)
                d = dev(np.frombuffer(w + b"\0", np.uint8))
                for chunk in (0, 1 + i, 4096):
                    assert long_match(r, d, len(w), chunk) == want, (synth.to_pattern(e)[:60], len(w), chunk)
    # empty string: the expression's nullability
    for pat, want in [(b"a*", 1), (b"a", 0), (b"\\e", 1), (b"(a|\\e)b*", 1)]:
        r = rx.Regex.compile(pat)
        d = dev(np.zeros(16, np.uint8))
        assert long_match(r, d, 0) == want
        assert seq_match(r, d, 0) == want


def test_long_wide_expression_falls_back_to_sequential():
    pat = b"(" + b"|".join(b"x" + bytes([97 + i % 26]) for i in range(400)) + b")*"
    nodes = oracle.parse(pat)
    r = rx.Regex.from_nodes(nodes, 0, rx.COMPILE_NO_MEMO)
    assert r.info()["words"] > 8
    s = synth.gen_strings(nodes, 4, 100, 5000, synth.LOWER, 3, p_lang=0.8)
    for k in range(s.n):
        w = s.get(k)
        d = dev(np.frombuffer(w + b"\0", np.uint8))
        assert long_match(r, d, len(w)) == oracle.o2(nodes, w)


@pytest.mark.slow
def test_long_full_size_vs_o2_and_sequential():
    """The 1 GiB text of the long-text configuration, and the same text with
    its last byte changed: the chunked result equals O2 over the whole text
    (one host thread each, run beside the GPU work) and the one-thread
    sequential GPU run."""
    import threading
    nodes, text, end = synth.cfg_long(with_end=True)
    n = len(text)
    flipped = text.copy()
    flipped[-1] = ord("q") if int(text[-1]) != ord("q") else ord("r")
    want = {}

    def o2_of(key, t):
        want[key] = int(oracle.o2(nodes, t))  # the C call releases the GIL

    threads = [threading.Thread(target=o2_of, args=(k, t)) for k, t in (("text", text), ("flipped", flipped))]
    for th in threads:
        th.start()
    r = rx.Regex.from_nodes(nodes)
    d = torch.from_numpy(text).cuda()
    f = torch.from_numpy(flipped).cuda()
    got = {"text": long_match(r, d, n), "flipped": long_match(r, f, n)}
    seq = {"text": seq_match(r, d, n), "flipped": seq_match(r, f, n)}
    # the text is a member of (R)* up to the end of its last whole 1 MiB
    # segment: the active set stays non-empty over (nearly) the whole gigabyte
    assert end > n - (2 << 20)
    assert long_match(r, d, end) == 1 and seq_match(r, d, end) == 1
    for th in threads:
        th.join()
    assert got == want and seq == want, (got, seq, want)


def batch_case(n_regex=250, max_len=6000, seed=0xE3):
    w = synth.cfg_batched(seed=seed, n_regex=n_regex, max_len=max_len, max_strings=24)
    # add wide expressions (warp class) and no-cache expressions (bitset classes)
    extra_regs, extra_strs, extra_rid = [], [], []
    for i in range(6):
        pat = b"(" + b"|".join(bytes([97 + (i + j) % 26]) + bytes([97 + j % 26]) for j in range(40 + 60 * i)) + b")*"
        nd = oracle.parse(pat)
        extra_regs.append(nd)
        s = synth.gen_strings(nd, 20, 0, 3000, synth.LOWER, synth.item_seed(seed, 900 + i), p_lang=0.7)
        extra_strs += [s.get(k) for k in range(s.n)]
        extra_rid += [n_regex + i] * s.n
    regs = w.regexes + extra_regs
    strs = [w.strings.get(k) for k in range(w.strings.n)] + extra_strs
    rid = np.concatenate([w.regex_of, np.array(extra_rid, np.int32)])
    # interleave the pairs so runs of the same handle are broken up
    order = np.random.default_rng(seed).permutation(len(strs))
    strs = [strs[k] for k in order]
    rid = rid[order]
    return regs, synth.pack(strs), rid


def test_batched_and_plain_forms_vs_o2():
    regs, s, rid = batch_case()
    want = np.zeros(s.n, np.uint8)
    for k in range(s.n):
        want[k] = oracle.o2(regs[rid[k]], s.get(k))
    handles = []
    compiled = {}
    for i, nd in enumerate(regs):
        flags = rx.COMPILE_NO_MEMO if i % 3 == 1 else 0
        compiled[i] = rx.Regex.from_nodes(nd, 0, flags)
    classes = set()
    for k in range(s.n):
        r = compiled[int(rid[k])]
        handles.append(r)
        inf = r.info()
        classes.add((inf["memo_states"] > 0, inf["words"]))
    assert any(w > 8 for _, w in classes) and any(m for m, _ in classes) and any(not m for m, _ in classes)
    d, o = dev(s.data), dev(s.offsets)
    out = torch.full((s.n,), 7, dtype=torch.uint8, device="cuda")
    rx.match_batch(handles, d, o, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert (got == want).all(), np.nonzero(got != want)[0][:10]
    out.fill_(7)
    rx.match_pairs(handles, d, o, out)
    torch.cuda.synchronize()
    assert (out.cpu().numpy() == want).all()


def test_batched_invalid_offsets():
    """Pairs whose offsets decrease (inside the buffer) get RX_RESULT_INVALID
    in every class of the batched kernel -- per-lane classes, the warp
    class, and long cached pairs chunked over a warp -- in the one-call form
    and a prepared batch; the others equal O2; rx_sync_check counts them."""
    regs, s, rid = batch_case(n_regex=120, max_len=9000)
    compiled = [rx.Regex.from_nodes(nd, 0, rx.COMPILE_NO_MEMO if i % 3 == 1 else 0) for i, nd in enumerate(regs)]
    lens = np.diff(s.offsets)
    rng = np.random.default_rng(0xEF)
    cand = np.arange(1, s.n - 1, 3)
    cand = cand[(lens[cand] > 0) & (s.offsets[cand] >= 1)]
    wide = cand[[compiled[int(rid[k])].info()["words"] > 8 for k in cand]]
    longp = cand[lens[cand] > 1500]
    bad = np.unique(np.concatenate([rng.choice(cand, 30, replace=False), wide[:5], longp[:5]]))
    bad = bad[np.concatenate([[True], np.diff(bad) > 1])]
    off = s.offsets.copy()
    for i in bad:
        off[i + 1] = off[i] - 1
    want = np.full(s.n, rx.RESULT_INVALID, np.uint8)
    for k in range(s.n):
        if k not in set(bad.tolist()):
            want[k] = oracle.o2(regs[rid[k]], s.data[off[k]:off[k + 1]].tobytes())
    hs = [compiled[int(i)] for i in rid]
    d, o = dev(s.data), dev(off)
    out = torch.full((s.n,), 7, dtype=torch.uint8, device="cuda")
    rx.sync_check(raise_error=False)
    rx.match_batch(hs, d, o, out)
    got = out.cpu().numpy()
    assert (got == want).all(), np.nonzero(got != want)[0][:10]
    assert rx.sync_check(raise_error=False) == len(bad)
    b = rx.Batch(hs)
    b.set_shape(256, 1500)  # cached pairs above 1500 bytes take a warp (chunked)
    out.fill_(7)
    b.run(d, o, out)
    assert (out.cpu().numpy() == want).all()
    assert rx.sync_check(raise_error=False) == len(bad)
    b.free()


def test_batched_edges():
    r = rx.Regex.compile(b"(ab)*")
    s = synth.pack([b"", b"ab", b"aba", b"abab" * 5000])
    d, o = dev(s.data), dev(s.offsets)
    out = torch.full((s.n,), 7, dtype=torch.uint8, device="cuda")
    rx.match_batch([r] * s.n, d, o, out)
    torch.cuda.synchronize()
    assert out.cpu().numpy().tolist() == [1, 1, 0, 1]
    rx.match_batch([], d, o, out)  # n = 0 is a no-op
    with pytest.raises(rx.RxError):
        rx.match_batch([rx.Regex.compile(b"a", rx.COMPILE_HOST_ONLY)], d, o, out)


def test_batched_long_pairs_chunked_per_warp():
    """Pairs longer than 6 KiB (the default threshold) whose expression has a cache of macro steps run
    one warp per pair (32 chunks, exact transfer functions composed by lane
    0).  Mix them with short pairs of the same and other expressions."""
    rng = np.random.default_rng(0xE9)
    regs, strs, rid = [], [], []
    for i in range(40):
        alpha = [synth.LOWER, synth.ALL_BYTES, b"abc"][i % 3]
        e = synth.gen_regex([12, 40, 100, 300][i % 4], 12, alpha, synth.item_seed(0xEA, i), eps_loop_p=0.05)
        regs.append(e)
        s = synth.gen_strings(e, 8, 0, 70000, alpha, synth.item_seed(0xEB, i), p_lang=0.7, log_len=True)
        for k in range(s.n):
            strs.append(s.get(k))
            rid.append(i)
        # some long ones for sure
        s2 = synth.gen_strings(e, 3, 9000, 70000, alpha, synth.item_seed(0xEC, i), p_lang=0.8)
        for k in range(s2.n):
            strs.append(s2.get(k))
            rid.append(i)
    order = rng.permutation(len(strs))
    strs = [strs[k] for k in order]
    rid = [rid[k] for k in order]
    assert sum(len(w) > 8192 for w in strs) >= 100
    handles = [rx.Regex.from_nodes(nd) for nd in regs]
    assert all(h.info()["memo_states"] > 0 for h in handles)
    pk = synth.pack(strs)
    d, o = dev(pk.data), dev(pk.offsets)
    out = torch.full((pk.n,), 7, dtype=torch.uint8, device="cuda")
    hl = [handles[i] for i in rid]
    rx.match_batch(hl, d, o, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    want = np.array([oracle.o2(regs[rid[k]], strs[k]) for k in range(pk.n)], np.uint8)
    assert (got == want).all(), np.nonzero(got != want)[0][:10]


def _counter_workload(seed):
    """Expressions whose cache states permute under the input, so incoming
    states never merge within a chunk (every prefix stage keeps several),
    with strings 0-70000 bytes; plus random expressions."""
    rng = np.random.default_rng(seed)
    pats = [b"(aaa)*", b"(aaaaa|b)*", b"((ab)*c)*", b"(a(bb)*a|b)*", b"((aa|b)(aa|b)(aa|b))*",
            b"(abc|bca|cab)*", b"(a|b)*a(a|b)(a|b)(a|b)"]
    regs = [oracle.parse(p) for p in pats]
    for i in range(12):
        regs.append(synth.gen_regex([12, 40, 100][i % 3], 10, b"abc", synth.item_seed(0xF1, i), eps_loop_p=0.05))
    strs, rid = [], []
    for i, e in enumerate(regs):
        for k in range(6):
            L = int(rng.choice([int(rng.integers(0, 300)), int(rng.integers(2000, 9000)),
                                int(rng.integers(9000, 70000))]))
            if k % 2 == 0:
                s = synth.gen_strings(e, 1, max(L - 64, 0), L, b"abc", synth.item_seed(0xF2 + i, k), p_lang=1.0)
                w = s.get(0)
            else:
                w = bytes(rng.choice(np.frombuffer(b"abc", np.uint8), size=L).tolist())
            strs.append(w)
            rid.append(i)
    order = rng.permutation(len(strs))
    return regs, [strs[k] for k in order], [rid[k] for k in order]


def test_batched_long_pairs_states_that_never_merge():
    regs, strs, rid = _counter_workload(0xF0)
    handles = [rx.Regex.from_nodes(nd) for nd in regs]
    assert all(h.info()["memo_states"] > 0 for h in handles)
    pk = synth.pack(strs)
    d, o = dev(pk.data), dev(pk.offsets)
    out = torch.full((pk.n,), 7, dtype=torch.uint8, device="cuda")
    rx.match_batch([handles[i] for i in rid], d, o, out)
    torch.cuda.synchronize()
    want = np.array([oracle.o2(regs[rid[k]], strs[k]) for k in range(pk.n)], np.uint8)
    got = out.cpu().numpy()
    assert (got == want).all(), np.nonzero(got != want)[0][:10]
    # (aaa)* on a^L: closed form
    for k in range(pk.n):
        if rid[k] == 0 and set(strs[k]) <= {ord("a")}:
            assert got[k] == (len(strs[k]) % 3 == 0)


def test_prepared_batch_graph_replay_recapture_and_autotune():
    """rx_batch_*: replays of the captured graph, a new capture for new
    buffers, and every autotuned launch shape, all equal to O2."""
    regs, strs, rid = _counter_workload(0xF3)
    for i in range(10):
        alpha = [synth.LOWER, synth.ALL_BYTES][i % 2]
        e = synth.gen_regex([20, 200][i % 2], 12, alpha, synth.item_seed(0xF4, i), eps_loop_p=0.05)
        regs.append(e)
        s = synth.gen_strings(e, 20, 0, 20000, alpha, synth.item_seed(0xF5, i), p_lang=0.6, log_len=True)
        for k in range(s.n):
            strs.append(s.get(k))
            rid.append(len(regs) - 1)
    # wide expressions (no cache): thread, sparse and warp classes in the mix
    for pat in [b"(" + b"|".join(b"x" + bytes([97 + j % 26]) for j in range(150)) + b")*",
                b"(" + b"|".join(bytes([97 + j % 26]) * 2 for j in range(20)) + b")*z"]:
        regs.append(oracle.parse(pat))
        s = synth.gen_strings(regs[-1], 30, 0, 3000, synth.LOWER, 0xF6 + len(regs), p_lang=0.7)
        for k in range(s.n):
            strs.append(s.get(k))
            rid.append(len(regs) - 1)
    handles = [rx.Regex.from_nodes(nd, 0, rx.COMPILE_NO_MEMO if len(nd) > 250 else 0) for nd in regs]
    want = np.array([oracle.o2(regs[rid[k]], strs[k]) for k in range(len(strs))], np.uint8)
    pk = synth.pack(strs)
    d, o = dev(pk.data), dev(pk.offsets)
    b = rx.Batch([handles[i] for i in rid])
    outs = [torch.full((pk.n,), 7, dtype=torch.uint8, device="cuda") for _ in range(2)]
    for rep in range(3):
        for out in outs:
            out.fill_(9)
            b.run(d, o, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert (got == want).all(), (rep, np.nonzero(got != want)[0][:10])
    t = b.autotune(d, o, outs[0])
    assert t["block"] in (128, 256, 512) and t["gb_per_s"] > 0
    assert (outs[0].cpu().numpy() == want).all()
    outs[1].fill_(9)
    b.run(d, o, outs[1])
    torch.cuda.synchronize()
    assert (outs[1].cpu().numpy() == want).all()
    # shapes set by hand: every block size, never / always chunked
    for block, lb in ((128, 1 << 40), (512, 1), (256, 3000)):
        b.set_shape(block, lb)
        outs[1].fill_(9)
        b.run(d, o, outs[1])
        torch.cuda.synchronize()
        assert (outs[1].cpu().numpy() == want).all(), (block, lb)
    for block, lb in ((64, 4096), (256, 0)):
        with pytest.raises(rx.RxError):
            b.set_shape(block, lb)
    b.free()
    # an empty prepared batch
    e = rx.Batch([])
    e.run(0, 0, 0)
    e.free()


def test_batched_full_size_vs_o2():
    """The batched workload at its full size (10,000 expressions, 148,077
    pairs, 844 MB), run as the benchmark runs it: a prepared batch replaying
    its captured graph, before and after the launch-shape autotuner, and the
    unprepared call.  Every pair is checked against O2 for its own
    expression (Thm 5.4)."""
    w = synth.cfg_batched()
    s = w.strings
    assert s.n == 148077
    want = oracle.o2_pairs(w.regexes, w.regex_of, s.data, s.offsets)
    handles = [rx.Regex.from_nodes(nd) for nd in w.regexes]
    hs = rx.handle_array([handles[i] for i in w.regex_of])
    d, o = dev(s.data), dev(s.offsets)
    outs = [torch.full((s.n,), 7, dtype=torch.uint8, device="cuda") for _ in range(3)]
    b = rx.Batch(hs)
    b.run(d, o, outs[0])
    b.autotune(d, o, outs[1])
    outs[1].fill_(7)
    b.run(d, o, outs[1])
    b.free()
    rx.match_batch(hs, d, o, outs[2])
    torch.cuda.synchronize()
    for k, x in enumerate(outs):
        got = x.cpu().numpy()
        bad = np.nonzero(got != want)[0]
        assert bad.size == 0, (k, bad[:10])
    assert 0.2 < want.mean() < 0.8


def wide_tier_pool(count=4):
    """Expressions of more than 256 positions whose cache of macro steps
    outgrows 192 states but fits the wide tier (two-byte ids)."""
    out = []
    for nd in synth.serving_pool(pool=300):
        inf = rx.Regex.from_nodes(nd, 0, rx.COMPILE_HOST_ONLY).info()
        if inf["memo_states"] == 0 and inf["wide_states"] > 0:
            out.append(nd)
        if len(out) == count:
            break
    assert len(out) == count
    return out


def test_batched_wide_tier_vs_o2():
    """Pairs of wide-tier expressions (one warp per pair, 32 chunk functions
    on two-byte state ids, Def 5.2) mixed with cached and uncached pairs:
    every pair equals O2 for its own expression, in the unprepared call, the
    prepared batch and the plain per-pair form; the same expressions
    compiled without the wide tier (bitset warp stepper) agree."""
    wide = wide_tier_pool(4)
    small = synth.gen_regex(60, 10, synth.ALL_BYTES, synth.item_seed(0xFB, 1))
    exprs = wide + [small]
    rng = np.random.default_rng(0xFB)
    parts, rid = [], []
    for k in range(400):
        ri = k % len(exprs)
        hi = int(rng.choice([0, 40, 2000, 30000, 70000], p=[0.05, 0.25, 0.3, 0.3, 0.1]))
        parts.append(synth.gen_strings(exprs[ri], 1, 0, hi, synth.ALL_BYTES, synth.item_seed(0xFC, k),
                                       p_lang=0.7, log_len=True).get(0))
        rid.append(ri)
    s = synth.pack(parts)
    rid = np.array(rid, np.int32)
    want = oracle.o2_pairs(exprs, rid, s.data, s.offsets)
    assert 0.1 < want.mean() < 0.9
    for flags in (0, rx.COMPILE_NO_WIDE):
        handles = [rx.Regex.from_nodes(nd, 0, flags) for nd in exprs]
        assert all((h.info()["wide_states"] > 0) == (flags == 0) for h in handles[:4])
        hs = rx.handle_array([handles[i] for i in rid])
        d, o = dev(s.data), dev(s.offsets)
        outs = [torch.full((s.n,), 7, dtype=torch.uint8, device="cuda") for _ in range(3)]
        rx.match_batch(hs, d, o, outs[0])
        b = rx.Batch(hs)
        b.run(d, o, outs[1])
        b.free()
        rx.match_pairs(hs, d, o, outs[2])
        torch.cuda.synchronize()
        for k, x in enumerate(outs):
            bad = np.nonzero(x.cpu().numpy() != want)[0]
            assert bad.size == 0, (flags, k, bad[:10])


def test_match_wide_tier_vs_o2():
    """rx_match on expressions with only the wide cache tier (one warp per
    string, 32 chunk functions on two-byte ids, rows in shared memory):
    every string equals O2, in input order and in length order, and equals
    the bitset warp stepper (the same expression without the tier)."""
    wide = wide_tier_pool(2)
    for e, nd in enumerate(wide):
        rng = np.random.default_rng(0xFE0 + e)
        parts = [synth.gen_strings(nd, 1, 0, int(rng.choice([0, 30, 500, 5000, 40000])), synth.ALL_BYTES,
                                   synth.item_seed(0xFE1 + e, k), p_lang=0.7, log_len=True).get(0)
                 for k in range(300)]
        s = synth.pack(parts)
        want = oracle.o2_batch(nd, s.data, s.offsets)
        assert 0 < want.sum() < len(want)
        r = rx.Regex.from_nodes(nd)
        r0 = rx.Regex.from_nodes(nd, 0, rx.COMPILE_NO_WIDE)
        assert r.info()["wide_states"] > 0 and r0.info()["wide_states"] == 0
        d, o = dev(s.data), dev(s.offsets)
        for h, sort in ((r, -1), (r, 0), (r, 1), (r0, -1)):
            out = torch.full((s.n,), 7, dtype=torch.uint8, device="cuda")
            rx.match(h, d, o, out, sort=sort)
            torch.cuda.synchronize()
            bad = np.nonzero(out.cpu().numpy() != want)[0]
            assert bad.size == 0, (e, sort, bad[:10])


def test_long_wide_tier_vs_o2():
    """rx_match_long on an expression with only the wide cache tier: segments
    of 32 chunk functions on two-byte ids, composed pairwise (Def 5.2).
    Texts in the language of (e)* and their flipped-last-byte copies, of
    several lengths and segment sizes, equal O2 and the sequential run."""
    wide = None
    for nd in synth.serving_pool(pool=300):
        st = synth.wrap_star(nd)
        inf = rx.Regex.from_nodes(st, 0, rx.COMPILE_HOST_ONLY).info()
        if inf["memo_states"] == 0 and inf["wide_states"] > 0:
            wide = (nd, st)
            break
    assert wide is not None
    nd, st = wide
    r = rx.Regex.from_nodes(st)
    assert r.info()["wide_states"] > 0
    for total, seed in ((0, 1), (100, 2), (5000, 3), (1 << 20, 4), (6 << 20, 5)):
        text = synth.star_text(nd, max(total, 1), seed)[:total]
        texts = [text.tobytes()]
        if total:
            flipped = bytearray(texts[0])
            flipped[-1] ^= 0x55
            texts.append(bytes(flipped))
        for t in texts:
            want = oracle.o2(st, t)
            d = dev(np.frombuffer(t, np.uint8)) if t else dev(np.zeros(1, np.uint8))
            for chunk in (0, 4096, 1 << 20):
                assert long_match(r, d, len(t), chunk) == want, (total, chunk)
            if len(t) <= 1 << 20:
                out = torch.full((1,), 7, dtype=torch.uint8, device="cuda")
                rx.match_seq(r, d, len(t), out)
                torch.cuda.synchronize()
                assert int(out.item()) == want, total
