"""GPU parity: the CUDA lockstep kernels against the CPU oracle, element by
element, through the C ABI (librx.so via the ctypes binding).  Exact work:
every boolean must agree (no tolerance)."""
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
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run(r, s: synth.Strings, variant=0, sort=-1, block=0):
    d = dev(s.data if s.data.size else np.zeros(1, np.uint8))
    o = dev(s.offsets)
    out = torch.full((max(s.n, 1),), 7, dtype=torch.uint8, device="cuda")
    rx.match(r, d, o, out, n=s.n, variant=variant, sort=sort, block=block)
    torch.cuda.synchronize()
    return out[:s.n].cpu().numpy()


def variants_of(r):
    v = r.info()["variants"]
    return [k for k in (rx.VARIANT_MEMO, rx.VARIANT_THREAD, rx.VARIANT_SPARSE, rx.VARIANT_WARP) if v >> k & 1]


def test_small_config_all_variants_vs_o1_o2():
    w = synth.cfg_small()
    nodes = w.regexes[0]
    want2 = oracle.o2_batch(nodes, w.strings.data, w.strings.offsets)
    want1 = oracle.o1_batch(nodes, w.strings.data, w.strings.offsets)
    assert (want1 == want2).all()
    r = rx.Regex.from_nodes(nodes)
    vs = variants_of(r)
    assert rx.VARIANT_MEMO in vs and rx.VARIANT_WARP in vs
    for v in [0] + vs:
        for sort in (0, 1, 2, 3):
            for block in ((0, 257, 128, 512) if v == rx.VARIANT_MEMO else (0,)):
                got = run(r, w.strings, v, sort, block)
                assert (got == want2).all(), (v, sort, block, np.nonzero(got != want2)[0][:10])


@pytest.mark.parametrize("seed", range(4))
def test_streaming_config_reduced_vs_o2(seed):
    w = synth.cfg_streaming(seed=synth.SEED_BASE + 2 + 1000 * seed, n=12000)
    nodes = w.regexes[0]
    want = oracle.o2_batch(nodes, w.strings.data, w.strings.offsets)
    r = rx.Regex.from_nodes(nodes)
    for v in [0] + variants_of(r):
        for block in ((0, 257) if v == rx.VARIANT_MEMO else (0,)):
            got = run(r, w.strings, v, block=block)
            assert (got == want).all(), (v, block, np.nonzero(got != want)[0][:10])
    # a share of both verdicts, and language samples accepted
    assert 0.2 < want.mean() < 0.9
    assert want[w.strings.kind == 1].all()


def test_streaming_config_full_size_sampled():
    """1,048,576 strings in the launch configuration the benchmark times
    (auto variant, length-sorted), checked on a sample against O2."""
    w = synth.cfg_streaming()
    nodes = w.regexes[0]
    r = rx.Regex.from_nodes(nodes)
    got = run(r, w.strings)
    rng = np.random.default_rng(1)
    idx = np.sort(rng.choice(w.strings.n, 4000, replace=False))
    sub = synth.pack([w.strings.get(int(i)) for i in idx])
    want = oracle.o2_batch(nodes, sub.data, sub.offsets)
    assert (got[idx] == want).all()
    # every variant agrees with the default on the whole batch
    for v in variants_of(r):
        assert (run(r, w.strings, v) == got).all(), v


@pytest.mark.parametrize("seed", range(3))
def test_random_expressions_all_alphabets(seed):
    for i in range(25):
        alpha = [b"abc", synth.LOWER, synth.ALL_BYTES][(i + seed) % 3]
        size = [3, 9, 17, 40, 90, 200][i % 6]
        e = synth.gen_regex(size, 12, alpha, synth.item_seed(0xD0 + seed, i), eps_loop_p=0.05)
        s = synth.gen_strings(e, 300, 0, 400, alpha, synth.item_seed(0xD8 + seed, i), p_lang=0.5)
        want = oracle.o2_batch(e, s.data, s.offsets)
        r = rx.Regex.from_nodes(e)
        for v in [0] + variants_of(r):
            got = run(r, s, v)
            assert (got == want).all(), (synth.to_pattern(e)[:80], v)


def test_edge_cases():
    cases = [
        (b"", [b"", b"a"]),
        (b"\\e", [b"", b"a", b"\\e"]),
        (b"(a*)*", [b"", b"a", b"a" * 1000, b"a" * 1000 + b"b"]),
        (b"(a*)*b", [b"aab", b"b", b"", b"aa", b"ba"]),
        (b"((((\\e*)*)*|a)*)*b", [b"aaab", b"aaa", b"b"]),
        (b"\\x00\\xff*", [b"\x00", b"\x00\xff\xff", b"\xff", b""]),
        (b"(ab|ac)*", [b"abac", b"abab" * 300 + b"ac", b"aa", b""]),
    ]
    for pat, strs in cases:
        s = synth.pack(strs)
        want = np.array([oracle.o2(oracle.parse(pat), x) for x in strs], np.uint8)
        r = rx.Regex.compile(pat)
        for v in [0] + variants_of(r):
            assert (run(r, s, v) == want).all(), (pat, v)


def test_empty_batch_and_empty_strings():
    r = rx.Regex.compile(b"a*")
    s = synth.pack([])
    assert run(r, s).size == 0
    s = synth.pack([b""] * 5000)
    assert (run(r, s) == 1).all()
    r2 = rx.Regex.compile(b"a")
    assert (run(r2, s) == 0).all()


def test_wide_expressions_warp_variant():
    # positions beyond the thread variants: 200 and ~2100 positions
    for pat in [b"(" + b"|".join(bytes([97 + i % 26]) * 2 for i in range(100)) + b")*z",
                b"(" + b"|".join(b"x" + bytes([97 + i % 26]) for i in range(1050)) + b")*"]:
        nodes = oracle.parse(pat)
        r = rx.Regex.from_nodes(nodes, 0, rx.COMPILE_NO_MEMO)
        assert r.info()["variants"] >> rx.VARIANT_WARP & 1
        s = synth.gen_strings(nodes, 200, 0, 600, synth.LOWER, 77, p_lang=0.7)
        want = oracle.o2_batch(nodes, s.data, s.offsets)
        for v in variants_of(r):
            assert (run(r, s, v) == want).all(), v


def test_long_strings_and_unaligned_offsets():
    e = synth.gen_regex(64, 10, synth.LOWER, synth.item_seed(0xDA, 0))
    s = synth.gen_strings(e, 64, 1, 70000, synth.LOWER, 99, p_lang=0.8, log_len=True)
    # shift the packing so starts are not 16-byte aligned
    pad = np.frombuffer(b"zzz", np.uint8)
    data = np.concatenate([pad, s.data])
    shifted = synth.Strings(data, s.offsets + 3, s.kind, 0)
    want = oracle.o2_batch(e, s.data, s.offsets)
    r = rx.Regex.from_nodes(e)
    for v in [0] + variants_of(r):
        assert (run(r, shifted, v) == want).all(), v


def test_set_trace_matches_fig61_machine():
    """Row k of rx_trace equals the set evolved by the sequential machine at
    macro step k (Thm 5.4 / 7.2: the lockstep sets are unique)."""
    cases = [(b"(a*)*b", b"aab")]
    for i in range(30):
        e = synth.gen_regex(12 + i, 8, b"abc", synth.item_seed(0xDB, i), eps_loop_p=0.1)
        s = synth.gen_strings(e, 1, 5, 40, b"abc", synth.item_seed(0xDC, i), p_lang=1.0)
        cases.append((synth.to_pattern(e), s.get(0)))
    for pat, w in cases:
        nodes = oracle.parse(pat)
        r = rx.Regex.from_nodes(nodes)
        t = r.tables()
        W = t["words"]
        rows = torch.zeros((len(w) + 1) * W, dtype=torch.int32, device="cuda")
        buf = dev(np.frombuffer(w + b"\0", np.uint8))
        rx.trace(r, buf, len(w), rows)
        torch.cuda.synchronize()
        rows = rows.cpu().numpy().view(np.uint32).reshape(len(w) + 1, W)
        acc, evolved, _ = oracle.o2_trace(nodes, w)
        pos = oracle.positions(nodes)
        for k in range(len(w) + 1):
            got = {pos[q] for q, b in enumerate(t["pos_bit"]) if (int(rows[k][int(b) >> 5]) >> (int(b) & 31)) & 1}
            nb = t["null_bit"]
            got_null = bool((int(rows[k][nb >> 5]) >> (nb & 31)) & 1)
            if not evolved[k][0] and not evolved[k][1] and k > 0:
                # the machine stopped (stuck): the GPU set must be empty from here
                assert not got and not got_null
                continue
            assert got == set(evolved[k][0]), (pat, w, k)
            assert got_null == evolved[k][1], (pat, w, k)
        assert bool(rows[len(w)][t["null_bit"] >> 5] >> (t["null_bit"] & 31) & 1) == acc


def test_seq_and_pairs_forms():
    e = synth.gen_regex(40, 10, synth.LOWER, synth.item_seed(0xDD, 0))
    s = synth.gen_strings(e, 40, 0, 3000, synth.LOWER, 5, p_lang=0.5)
    want = oracle.o2_batch(e, s.data, s.offsets)
    r = rx.Regex.from_nodes(e)
    d, o = dev(s.data), dev(s.offsets)
    out = torch.zeros(s.n, dtype=torch.uint8, device="cuda")
    rx.match_pairs([r] * s.n, d, o, out)
    torch.cuda.synchronize()
    assert (out.cpu().numpy() == want).all()
    for i in range(0, s.n, 7):
        one = torch.zeros(1, dtype=torch.uint8, device="cuda")
        a, b = int(s.offsets[i]), int(s.offsets[i + 1])
        rx.match_seq(r, d[a:] if b > a else d, b - a, one)
        torch.cuda.synchronize()
        assert int(one.item()) == want[i]


def test_autotune_records_and_is_used():
    w = synth.cfg_streaming(seed=synth.SEED_BASE + 77, n=20000)
    nodes = w.regexes[0]
    r = rx.Regex.from_nodes(nodes)
    d, o = dev(w.strings.data), dev(w.strings.offsets)
    out = torch.zeros(w.strings.n, dtype=torch.uint8, device="cuda")
    rx.tune_reset()
    e = rx.autotune(r, d, o, out)
    assert e["gb_per_s"] > 0 and (r.info()["variants"] >> e["variant"]) & 1
    table = rx.tune_table()
    assert len(table) == 2 and {t["len_bucket"] for t in table} == {-1, e["len_bucket"]}
    want = oracle.o2_batch(nodes, w.strings.data, w.strings.offsets)
    for hint in (0, 512, 10 ** 6):
        out.fill_(7)
        rx.match(r, d, o, out, len_hint=hint)
        torch.cuda.synchronize()
        assert (out.cpu().numpy() == want).all()
    rx.tune_reset()
    assert rx.tune_table() == []


def test_errors_do_not_poison_the_context():
    r = rx.Regex.compile(b"ab*")
    with pytest.raises(rx.RxError) as ei:
        rx.match(r, 0, 0, 0, n=3)  # null offsets with n > 0
    assert ei.value.status == 2
    r2 = rx.Regex.compile(b"(" + b"|".join(b"ab" for _ in range(40)) + b")*", rx.COMPILE_NO_MEMO)
    s = synth.pack([b"abab"])
    with pytest.raises(rx.RxError) as ei:
        run(r2, s, rx.VARIANT_MEMO)
    assert ei.value.status == 8
    assert (run(r, synth.pack([b"abbb", b"ba"])) == np.array([1, 0])).all()
