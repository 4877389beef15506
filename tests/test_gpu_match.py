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
        for sort in (0, 1, 2, 3, 4):
            for block in ((0, 257, 128, 512, 130, 4, 12, 20) if v == rx.VARIANT_MEMO else (0,)):
                got = run(r, w.strings, v, sort, block)
                assert (got == want2).all(), (v, sort, block, np.nonzero(got != want2)[0][:10])


@pytest.mark.parametrize("seed", range(4))
def test_streaming_config_reduced_vs_o2(seed):
    w = synth.cfg_streaming(seed=synth.SEED_BASE + 2 + 1000 * seed, n=12000)
    nodes = w.regexes[0]
    want = oracle.o2_batch(nodes, w.strings.data, w.strings.offsets)
    r = rx.Regex.from_nodes(nodes)
    for v in [0] + variants_of(r):
        for block in ((0, 257, 4, 12, 20) if v == rx.VARIANT_MEMO else (0,)):
            got = run(r, w.strings, v, block=block)
            assert (got == want).all(), (v, block, np.nonzero(got != want)[0][:10])
    # a share of both verdicts, and language samples accepted
    assert 0.2 < want.mean() < 0.9
    assert want[w.strings.kind == 1].all()


@pytest.fixture(scope="module")
def streaming_full():
    """The full streaming workload (1,048,576 strings, 537 MB) and O2's
    verdict on every string (all host threads)."""
    w = synth.cfg_streaming()
    want = oracle.o2_batch(w.regexes[0], w.strings.data, w.strings.offsets)
    return w, want


def test_streaming_config_full_size_vs_o2(streaming_full):
    """1,048,576 strings in the launch configuration the benchmark times
    (auto variant, length-sorted), every string against O2 (Thm 5.4: the
    lockstep machine decides the relation of Fig 2.1)."""
    w, want = streaming_full
    nodes = w.regexes[0]
    r = rx.Regex.from_nodes(nodes)
    got = run(r, w.strings)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, bad[:10]
    assert 0.2 < want.mean() < 0.9
    # every variant agrees with O2 on the whole batch
    for v in variants_of(r):
        assert (run(r, w.strings, v) == want).all(), v
    # and the kernels that stage the input with bulk copies, with no wait
    # that gave up
    rx.device_faults(reset=True)
    for block in (4, 12, 20):
        assert (run(r, w.strings, rx.VARIANT_MEMO, block=block) == want).all(), block
    assert rx.device_faults() == 0


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


def invalidate(offsets, idx):
    """Offsets with the strings idx made invalid by a decrease that stays
    inside the buffer: offsets[i+1] = offsets[i] - 1 (string i + 1 then
    starts one byte earlier).  Returns the new offsets."""
    off = np.array(offsets, np.int64, copy=True)
    for i in idx:
        assert off[i] >= 1
        off[i + 1] = off[i] - 1
    assert (off >= 0).all() and off[-1] == offsets[-1]
    return off


def o2_or_invalid(nodes, data, off, bad):
    """O2 on every string with valid offsets, the marker on the others."""
    want = np.full(len(off) - 1, rx.RESULT_INVALID, np.uint8)
    ok = np.ones(len(off) - 1, bool)
    ok[list(bad)] = False
    k = np.nonzero(ok)[0]
    sub = synth.pack([data[off[i]:off[i + 1]].tobytes() for i in k])
    want[k] = oracle.o2_batch(nodes, sub.data, sub.offsets)
    return want


def test_invalid_offsets_marked_counted_and_reported():
    """A string whose offsets decrease is not matched: its result is the
    marker RX_RESULT_INVALID (RX_SEARCH_INVALID for search), the others are
    unaffected, and rx_sync_check reports the count as RX_ERR_INVALID_ARG.
    Every kernel that reads offsets is covered (streaming one- and two-byte,
    bulk-copy staged, per-thread bitset, sparse, warp, search, the
    allocation-free entry point, the plain per-pair form).  Only decreases
    that stay inside the buffer are used; negative offsets take the same
    test in the kernels (0 <= offsets[i] <= offsets[i+1])."""
    w = synth.cfg_streaming(seed=synth.SEED_BASE + 321, n=9000)
    nodes = w.regexes[0]
    s = w.strings
    rng = np.random.default_rng(21)
    bad = np.sort(rng.choice(np.arange(1, s.n - 1, 3), 60, replace=False))
    bad = bad[np.diff(s.offsets)[bad] > 0]
    off = invalidate(s.offsets, bad)
    want = o2_or_invalid(nodes, s.data, off, bad)
    assert want[bad].tolist() == [rx.RESULT_INVALID] * len(bad) and 0 < (want == 1).sum()
    r = rx.Regex.from_nodes(nodes, 0, rx.COMPILE_SEARCH)
    d, o = dev(s.data), dev(off)
    out = torch.full((s.n,), 7, dtype=torch.uint8, device="cuda")
    rx.sync_check(raise_error=False)
    shapes = [(v, sort, block) for v in [0] + variants_of(r) for sort in (0, 1, 2, 3, 4)
              for block in ((0, 257, 4, 12, 20) if v == rx.VARIANT_MEMO else (0,))]
    for v, sort, block in shapes:
        out.fill_(7)
        rx.match(r, d, o, out, n=s.n, variant=v, sort=sort, block=block)
        got = out.cpu().numpy()
        assert (got == want).all(), (v, sort, block, np.nonzero(got != want)[0][:10])
        with pytest.raises(rx.RxError) as ei:
            rx.sync_check()
        assert ei.value.status == 2 and str(len(bad)) in ei.value.message
    # the count itself, over several calls, and a clean call afterwards
    for _ in range(3):
        rx.match(r, d, o, out, n=s.n)
    assert rx.sync_check(raise_error=False) == 3 * len(bad)
    rx.match(r, d, dev(s.offsets), out, n=s.n)
    assert rx.sync_check() == 0
    # the allocation-free entry point and the plain per-pair form
    out.fill_(7)
    rx.match_static(r, d, o, out, n=s.n)
    assert (out.cpu().numpy() == want).all()
    assert rx.sync_check(raise_error=False) == len(bad)
    sub_n = int(bad[4]) + 2
    out.fill_(7)
    rx.match_pairs([r] * sub_n, d, o, out)
    assert (out.cpu().numpy()[:sub_n] == want[:sub_n]).all()
    assert rx.sync_check(raise_error=False) == int((bad < sub_n).sum())
    # search: the marker, and O2's search answer elsewhere
    ends = torch.full((s.n,), 7, dtype=torch.int64, device="cuda")
    rx.search(r, d, o, ends, n=s.n)
    got = ends.cpu().numpy()
    assert (got[bad] == rx.SEARCH_INVALID).all()
    ok = np.setdiff1d(np.arange(s.n), bad)
    sub = synth.pack([s.data[off[i]:off[i + 1]].tobytes() for i in ok])
    assert (got[ok] == oracle.o2_search_batch(nodes, sub.data, sub.offsets)).all()
    assert rx.sync_check(raise_error=False) == len(bad)
    # an expression too wide for the cache and the per-thread sets (warp
    # variant only), and one for the sparse variant
    for pat in (b"(" + b"|".join(b"x" + bytes([97 + i % 26]) for i in range(300)) + b")*",
                b"(" + b"|".join(bytes([97 + i % 26]) * 2 for i in range(50)) + b")*z"):
        nd = oracle.parse(pat)
        rw = rx.Regex.from_nodes(nd, 0, rx.COMPILE_NO_MEMO)
        ws = synth.gen_strings(nd, 3000, 0, 300, synth.LOWER, 5, p_lang=0.7)
        bw = np.arange(1, ws.n - 1, 97)
        bw = bw[np.diff(ws.offsets)[bw] > 0]
        ow = invalidate(ws.offsets, bw)
        ww = o2_or_invalid(nd, ws.data, ow, bw)
        outw = torch.full((ws.n,), 7, dtype=torch.uint8, device="cuda")
        for v in variants_of(rw):
            outw.fill_(7)
            rx.match(rw, dev(ws.data), dev(ow), outw, n=ws.n, variant=v)
            assert (outw.cpu().numpy() == ww).all(), (pat[:20], v)
            assert rx.sync_check(raise_error=False) == len(bw)


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


def test_pair_kernel_fallback_outside_the_byte_window():
    """The two-byte cache applies to 32-byte blocks whose bytes all lie in the
    expression's label window; blocks with other bytes (for some lanes or
    all) take the one-byte path.  Mix such bytes into language samples."""
    rng = np.random.default_rng(5)
    for i in range(6):
        e = synth.gen_regex(64, 10, synth.LOWER, synth.item_seed(0xDE, i))
        r = rx.Regex.from_nodes(e)
        s = synth.gen_strings(e, 3000, 1, 700, synth.LOWER, synth.item_seed(0xDF, i), p_lang=0.8)
        data = s.data.copy()
        # sprinkle bytes outside [0x60, 0x80) into a third of the strings
        for k in range(0, s.n, 3):
            a, b = int(s.offsets[k]), int(s.offsets[k + 1])
            if b > a:
                pos = rng.integers(a, b, size=max(1, (b - a) // 97))
                data[pos] = rng.choice([0x00, 0x41, 0x5F, 0x80, 0x7B, 0xFF], size=len(pos))
        mixed = synth.Strings(data, s.offsets, s.kind, 0)
        want = oracle.o2_batch(e, data, s.offsets)
        for v, block in ((0, 0), (rx.VARIANT_MEMO, 0), (rx.VARIANT_MEMO, 257),
                         (rx.VARIANT_MEMO, 4), (rx.VARIANT_MEMO, 12), (rx.VARIANT_MEMO, 20), (rx.VARIANT_THREAD, 0)):
            got = run(r, mixed, v, block=block)
            assert (got == want).all(), (i, v, block, np.nonzero(got != want)[0][:10])
        # and strings made only of out-of-window bytes
        junk = synth.pack([bytes(rng.integers(0x80, 0x100, size=n).tolist()) for n in rng.integers(0, 300, 200)])
        wantj = oracle.o2_batch(e, junk.data, junk.offsets)
        assert (run(r, junk) == wantj).all()


def test_block_local_kernel_both_table_forms_and_window_bytes():
    """From 4,096 strings rx_match takes the block-local streaming kernel: a
    cache of at most 24 states in the form whose two-byte entries are shared
    addresses, 25-64 states in the form whose entries are offsets / 64.
    Both forms on 9,000 strings, clean and with bytes outside the label
    window sprinkled through a third of them -- inside the blocks that are
    whole for every lane of a round (there such a byte empties the lane's
    set) as well as in first and last blocks -- against O2, also over the
    planner's global order and in input order, and no device fault
    counted."""
    rng = np.random.default_rng(11)
    forms = set()
    rx.device_faults(reset=True)
    for size, i in ((64, 0), (64, 2), (64, 38), (96, 0)):
        e = synth.gen_regex(size, 10, synth.LOWER, synth.item_seed(0xE1, size * 100 + i))
        r = rx.Regex.from_nodes(e)
        k = r.info()["memo_states"]
        assert 0 < k <= 64
        forms.add(k <= 24)
        s = synth.gen_strings(e, 9000, 1, 700, synth.LOWER, synth.item_seed(0xE2, size * 100 + i), p_lang=0.8)
        assert (run(r, s) == oracle.o2_batch(e, s.data, s.offsets)).all(), (size, i, k)
        data = s.data.copy()
        for j in range(0, s.n, 3):
            a, b = int(s.offsets[j]), int(s.offsets[j + 1])
            if b > a:
                pos = rng.integers(a, b, size=max(1, (b - a) // 131))
                data[pos] = rng.choice([0x00, 0x41, 0x5F, 0x80, 0x7B, 0xFF], size=len(pos))
        mixed = synth.Strings(data, s.offsets, s.kind, 0)
        want = oracle.o2_batch(e, data, s.offsets)
        got = run(r, mixed)
        assert (got == want).all(), (size, i, k, np.nonzero(got != want)[0][:10])
        # the same rounds over the planner's global length order, and in
        # input order (lengths mixed within a round: mostly the masked blocks)
        for order in (2, 3):
            assert (run(r, mixed, sort=order) == want).all(), (size, i, k, order)
    assert forms == {True, False}
    assert rx.device_faults() == 0


def test_block_local_rounds_of_mixed_block_counts():
    """6,000 strings (the block-local kernel) of 1 to 20,000 bytes: from 2 KiB
    on the length buckets are log-spaced, so the lanes of a round touch
    different numbers of 32-byte blocks (the loop over whole blocks stops
    at the round's smallest count, the masked loop finishes the rest);
    every seventh string cut to a multiple of 32 bytes (0 to 256), and the
    packing shifted so that the strings start at other offsets within
    their 32-byte blocks.  Both two-byte table forms, against O2."""
    rng = np.random.default_rng(21)
    for size, i in ((64, 0), (64, 38)):
        e = synth.gen_regex(size, 10, synth.LOWER, synth.item_seed(0xE1, size * 100 + i))
        r = rx.Regex.from_nodes(e)
        s = synth.gen_strings(e, 6000, 1, 20000, synth.LOWER, synth.item_seed(0xE3, i), p_lang=0.8, log_len=True)
        pieces = [s.get(j) for j in range(s.n)]
        for j in range(0, s.n, 7):
            pieces[j] = pieces[j][:32 * int(rng.integers(0, 9))]
        packed = synth.pack(pieces)
        assert max(len(x) for x in pieces) > 4096
        want = oracle.o2_batch(e, packed.data, packed.offsets)
        for shift in (0, 5, 17):
            data = np.concatenate([np.full(shift, ord("z"), np.uint8), packed.data])
            shifted = synth.Strings(data, packed.offsets + shift, packed.kind, 0)
            got = run(r, shifted)
            assert (got == want).all(), (size, i, shift, np.nonzero(got != want)[0][:10])


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


def test_host_buffers_pipelined_pieces(streaming_full):
    """rx_match_host on host buffers: the full-size streaming batch (537 MB,
    about nine 64 MiB pieces) equals O2 on every string, the strings at
    every piece cut included."""
    w, want = streaming_full
    nodes = w.regexes[0]
    r = rx.Regex.from_nodes(nodes)
    h_str = torch.from_numpy(w.strings.data).pin_memory()
    h_off = torch.from_numpy(w.strings.offsets).pin_memory()
    h_out = torch.full((w.strings.n,), 7, dtype=torch.uint8).pin_memory()
    rx.match_host(r, h_str, h_off, h_out)
    got = h_out.numpy()
    assert (got == want).all(), np.nonzero(got != want)[0][:10]
    # pageable numpy buffers, a second call on the same stream
    out2 = np.full(w.strings.n, 9, np.uint8)
    rx.match_host(r, w.strings.data, w.strings.offsets, out2)
    assert (out2 == want).all()


def test_host_buffers_many_short_strings_and_offsets_not_at_zero():
    """More than 2^20 strings (pieces cut by count), empty strings, offsets
    that start past byte 0 and end before the buffer does."""
    rng = np.random.default_rng(11)
    e = oracle.parse(b"(a|b)*a(a|b)")  # second-to-last byte is 'a'
    r = rx.Regex.from_nodes(e)
    n = (1 << 20) * 2 + 12345
    lens = rng.integers(0, 6, size=n)
    offs = np.zeros(n + 1, np.int64)
    np.cumsum(lens, out=offs[1:])
    body = rng.choice(np.frombuffer(b"ab", np.uint8), size=int(offs[-1]))
    data = np.concatenate([np.frombuffer(b"zzzzz", np.uint8), body, np.frombuffer(b"zz", np.uint8)])
    offs5 = offs + 5
    out = np.full(n, 7, np.uint8)
    rx.match_host(r, data, offs5, out)
    # closed form of the language: length >= 2 and byte len-2 is 'a'
    ends = offs5[1:]
    want = (lens >= 2) & (data[np.maximum(ends - 2, 0)] == ord("a"))
    assert (out == want.astype(np.uint8)).all()
    # and O2 on every string
    assert (out == oracle.o2_batch(e, data, offs5)).all()


def test_host_buffers_edges_and_errors():
    r = rx.Regex.compile(b"a*")
    out = np.zeros(1, np.uint8)
    rx.match_host(r, np.zeros(1, np.uint8), np.zeros(1, np.int64), out, n=0)
    s = synth.pack([b"", b"aaa", b"ab", b"a" * (70 << 20)])  # one string above the piece size
    got = np.full(4, 7, np.uint8)
    rx.match_host(r, s.data, s.offsets, got)
    assert got.tolist() == [1, 1, 0, 1]
    bad = np.array([0, 5, 3], np.int64)
    with pytest.raises(rx.RxError) as ei:
        rx.match_host(r, np.zeros(8, np.uint8), bad, np.zeros(2, np.uint8))
    assert ei.value.status == 2
    for neg in (np.array([-1, 0], np.int64), np.array([0, 2, -1], np.int64)):
        with pytest.raises(rx.RxError) as ei:
            rx.match_host(r, np.zeros(8, np.uint8), neg, np.zeros(len(neg) - 1, np.uint8))
        assert ei.value.status == 2
    # a decrease in the second piece (pieces hold 2^20 strings): the error is
    # reported after the first piece was queued; the second piece is untouched
    n = (1 << 20) + 16
    offs = np.zeros(n + 1, np.int64)
    offs[(1 << 20) + 5:] = 5
    offs[(1 << 20) + 6] = 3
    got = np.full(n, 7, np.uint8)
    with pytest.raises(rx.RxError) as ei:
        rx.match_host(r, np.zeros(16, np.uint8), offs, got)
    assert ei.value.status == 2
    assert set(np.unique(got[:1 << 20]).tolist()) <= {1, 7} and (got[1 << 20:] == 7).all()
    assert (run(r, synth.pack([b"aa", b"b"])) == np.array([1, 0])).all()


def test_planner_one_launch_and_two_launch_forms():
    """The length planner runs as one cooperative launch when every tile of
    2048 strings gets a resident block, else as two launches; by default
    (order 4) planner and streaming kernel share one cooperative launch
    when the planner's keys fit beside the tables.  1,300,000 short strings
    take the two-launch planner, their first 600,000 the one-launch
    planner; 4,500,000 take the separate planner (the keys no longer fit
    the shared one).  Every form equals the unplanned order and O2 on every
    string, with no barrier wait that gave up."""
    w = synth.cfg_small(n=8)
    nodes = w.regexes[0]
    r = rx.Regex.from_nodes(nodes)
    big = synth.gen_strings(nodes, 4500000, 0, 80, synth.LOWER, synth.item_seed(0xA7, 1), p_lang=0.5)
    rx.device_faults(reset=True)
    for n in (600000, 1300000, 4500000):
        s = big if n == big.n else synth.Strings(big.data[:big.offsets[n]], big.offsets[:n + 1], big.kind[:n], 0)
        want = oracle.o2_batch(nodes, s.data, s.offsets)
        assert (run(r, s, sort=0) == want).all(), n
        for sort in (2, 4, -1):
            assert (run(r, s, sort=sort) == want).all(), (n, sort)
    assert rx.device_faults() == 0
