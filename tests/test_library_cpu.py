"""CPU-side checks of the library: the C ABI loads and exports every symbol
include/rx.h declares, and the host compiler (a1-a4: parse, cont, evolutions,
successor sets) agrees with the oracle.  No kernel runs here: handles are
compiled with RX_COMPILE_HOST_ONLY."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_1108_3126_b300 as rx
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1108_3126_b300 import build
    build.build()


def declared_symbols():
    out = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(rx_\w+)\s*\(", text, flags=re.M):
            out.add(m.group(1))
    return out


def test_exports_every_declared_symbol():
    syms = declared_symbols()
    assert len(syms) >= 20
    lib = ctypes.CDLL(rx.LIB_PATH)
    missing = [s for s in sorted(syms) if not hasattr(lib, s)]
    assert not missing, missing
    # the binding covers the whole header
    assert syms <= set(rx.SIGNATURES), syms - set(rx.SIGNATURES)


def test_version_and_error_strings():
    assert b"sm_103a" in rx.lib().rx_version()
    assert rx.last_error()


def host(pattern_or_nodes, flags=rx.COMPILE_HOST_ONLY):
    if isinstance(pattern_or_nodes, (bytes, str)):
        return rx.Regex.compile(pattern_or_nodes, flags)
    return rx.Regex.from_nodes(pattern_or_nodes, 0, flags)


def bits_to_set(words, pos_bit, null_bit):
    s = set()
    null_bit = int(null_bit)
    for q, b in enumerate(pos_bit):
        b = int(b)
        if (int(words[b >> 5]) >> (b & 31)) & 1:
            s.add(q)
    has_null = bool((int(words[null_bit >> 5]) >> (null_bit & 31)) & 1)
    return s, has_null


def check_against_glushkov(nodes):
    r = host(nodes)
    tree = r.tree()
    t = r.tables()
    # the library numbers nodes in preorder; compare on its tree
    pos = oracle.positions(tree)
    assert t["pos_node"].tolist() == pos
    assert t["cont"].tolist() == oracle.cont(tree).tolist()
    nullable, first, last, follow = oracle.glushkov(tree)
    idx = {p: q for q, p in enumerate(pos)}
    st, st_null = bits_to_set(t["start"], t["pos_bit"], t["null_bit"])
    assert st == {idx[p] for p in first} and st_null == nullable
    for q, p in enumerate(pos):
        f, fn = bits_to_set(t["follow"][q], t["pos_bit"], t["null_bit"])
        assert f == {idx[x] for x in follow[p]}, (q, p)
        assert fn == (p in last)
    # bit layout: distinct bits, null separate, within the declared width
    bits = t["pos_bit"].tolist()
    assert len(set(bits)) == len(bits) and t["null_bit"] not in bits
    assert max(bits + [t["null_bit"]]) < 32 * t["words"]
    info = r.info()
    assert info["positions"] == len(pos) and info["nullable"] == int(nullable)


def test_fig41_tables():
    # (a*)* b: Fig 4.1 numbering differs from preorder; compare through the tree
    nodes = oracle.parse(b"(a*)*b")
    check_against_glushkov(nodes)
    r = host(b"(a*)*b")
    t = r.tables()
    tree = r.tree()
    # preorder: 0 CAT, 1 STAR (p1), 2 STAR (p3), 3 a (p4), 4 b (p2)
    assert tree["kind"].tolist() == [rx.CAT, rx.STAR, rx.STAR, rx.CHAR, rx.CHAR]
    assert t["cont"].tolist() == [-1, 4, 1, 2, -1]  # = Fig 4.1: p1->p2, p3->p1, p4->p3


@pytest.mark.parametrize("seed", range(6))
def test_tables_match_glushkov_random(seed):
    for i in range(40):
        size = 1 + (i * 7 + seed) % 90
        alpha = [b"abc", synth.LOWER, synth.ALL_BYTES][i % 3]
        e = synth.gen_regex(size, 10, alpha, synth.item_seed(0xC0 + seed, i), eps_loop_p=0.1)
        check_against_glushkov(e)


def test_wide_expression_tables():
    # more than 64 and more than 1024 positions: sequential bit layout
    e = synth.gen_regex(400, 14, synth.LOWER, synth.item_seed(0xC9, 1))
    check_against_glushkov(e)
    big = oracle.parse(b"(" + b"|".join(b"ab" for _ in range(700)) + b")*")
    check_against_glushkov(big)


def test_parse_matches_oracle_parser():
    for i in range(150):
        e = synth.gen_regex(1 + i % 60, 9, synth.ALL_BYTES, synth.item_seed(0xCA, i), eps_loop_p=0.05)
        pat = synth.to_pattern(e)
        assert (host(pat).tree() == oracle.parse(pat)).all()
    for pat in [b"", b"()", b"a|", b"|", b"(|)*", b"\\x00\\xff", b"a**|\\e*b", b"\\(\\)\\|\\*\\\\"]:
        assert (host(pat).tree() == oracle.parse(pat)).all(), pat


@pytest.mark.parametrize("bad,pos", [(b"(", 1), (b")", 0), (b"*a", 0), (b"a(b", 3), (b"\\x4", 0), (b"ab)", 2)])
def test_parse_errors(bad, pos):
    with pytest.raises(rx.RxError) as ei:
        host(bad)
    assert ei.value.status == 1 and ei.value.err_pos == pos
    with pytest.raises(ValueError):
        oracle.parse(bad)


def test_malformed_trees_rejected():
    nd = rx.NODE_DTYPE
    shared = np.array([(rx.CAT, 0, 0, 1, 1), (rx.CHAR, 97, 0, -1, -1)], nd)  # one child used twice
    cyc = np.array([(rx.STAR, 0, 0, 1, -1), (rx.STAR, 0, 0, 0, -1)], nd)
    oob = np.array([(rx.ALT, 0, 0, 1, 5), (rx.CHAR, 97, 0, -1, -1)], nd)
    badkind = np.array([(9, 0, 0, -1, -1)], nd)
    for t in (shared, cyc, oob, badkind):
        with pytest.raises(rx.RxError) as ei:
            rx.Regex.from_nodes(t, 0, rx.COMPILE_HOST_ONLY)
        assert ei.value.status == 2
    with pytest.raises(rx.RxError):
        rx.Regex.from_nodes(shared, 7, rx.COMPILE_HOST_ONLY)


def test_limits():
    # more than RX_MAX_POSITIONS positions
    pat = b"a" * 5000
    with pytest.raises(rx.RxError) as ei:
        host(pat)
    assert ei.value.status == 3
    deep = b"(" * 30000 + b"a" + b")" * 30000
    with pytest.raises(rx.RxError) as ei:
        host(deep)
    assert ei.value.status == 3


def test_memo_cache_is_a_cache_of_macro_steps():
    # the cache covers every reachable set; its states are distinct sets
    for i in range(20):
        e = synth.gen_regex(64, 10, synth.LOWER, synth.item_seed(0xCB, i))
        info = host(e, 0 | rx.COMPILE_HOST_ONLY).info()
        assert info["memo_states"] >= 2
        assert info["variants"] & (1 << rx.VARIANT_MEMO)
    no = host(synth.gen_regex(64, 10, synth.LOWER, 5), rx.COMPILE_HOST_ONLY | rx.COMPILE_NO_MEMO).info()
    assert no["memo_states"] == 0 and not (no["variants"] & (1 << rx.VARIANT_MEMO))


def reachable_macro_states(r):
    """Every set reachable from the start by macro steps (Def 5.2 on the
    evolved sets: S' = union of the evolutions of cont p for p in S
    labelled c), plus the empty set; counted from the compiler's Glushkov
    tables, which test_tables_match_glushkov_random pins separately."""
    t = r.tables()
    m, W = len(t["pos_node"]), t["words"]
    nodes = r.tree()

    def bits(words):
        return sum(int(x) << (32 * i) for i, x in enumerate(words))

    fol = {int(t["pos_bit"][p]): bits(t["follow"][p]) for p in range(m)}
    lab = {}
    for p in range(m):
        c = int(nodes["byte"][t["pos_node"][p]])
        lab[c] = lab.get(c, 0) | (1 << int(t["pos_bit"][p]))
    start = bits(t["start"])
    seen, todo = {0, start}, [start]
    while todo:
        S = todo.pop()
        for c, B in lab.items():
            x, nx = S & B, 0
            while x:
                b = (x & -x).bit_length() - 1
                x &= x - 1
                nx |= fol[b]
            if nx not in seen:
                seen.add(nx)
                todo.append(nx)
    return len(seen)


def test_cache_sizes_are_the_reachable_macro_states():
    """The one-byte cache (<= 192 states) and, for sets of more than 256
    positions beyond it, the wide tier (two-byte ids) each hold exactly the
    reachable sets; RX_COMPILE_NO_WIDE and RX_COMPILE_NO_MEMO drop them."""
    for i in range(3):
        e = synth.gen_regex(64, 10, synth.LOWER, synth.item_seed(0xCC, i))
        r = host(e)
        assert r.info()["memo_states"] == reachable_macro_states(r) and r.info()["wide_states"] == 0
    wide = 0
    for nd in synth.serving_pool(pool=120):
        r = host(nd)
        inf = r.info()
        if inf["memo_states"] == 0 and inf["wide_states"] > 0:
            assert inf["words"] > 8 and inf["wide_states"] > 192
            assert inf["wide_states"] == reachable_macro_states(r)
            assert host(nd, rx.COMPILE_HOST_ONLY | rx.COMPILE_NO_WIDE).info()["wide_states"] == 0
            assert host(nd, rx.COMPILE_HOST_ONLY | rx.COMPILE_NO_MEMO).info()["wide_states"] == 0
            wide += 1
            if wide == 2:
                break
    assert wide == 2


def test_host_only_handle_cannot_match():
    r = host(b"abc")
    with pytest.raises(rx.RxError) as ei:
        rx.match(r, 0, 0, 0, n=1, stream=0)
    assert ei.value.status == 2


def test_search_cache_built_only_with_the_flag():
    import paper_1108_3126_b300 as rx
    for pat, want in ((b"ab", 3), (b"(a*)*b", 2), (b"x(x|a|b)*x", 3)):
        r = rx.Regex.compile(pat, rx.COMPILE_SEARCH | rx.COMPILE_HOST_ONLY)
        assert r.info()["search_states"] == want, pat
        r2 = rx.Regex.compile(pat, rx.COMPILE_HOST_ONLY)
        assert r2.info()["search_states"] == 0
    # no cache without the macro-step cache either
    r3 = rx.Regex.compile(b"ab", rx.COMPILE_SEARCH | rx.COMPILE_NO_MEMO | rx.COMPILE_HOST_ONLY)
    assert r3.info()["search_states"] == 0


def test_batch_entry_points_reject_null_arguments():
    import ctypes
    import paper_1108_3126_b300 as rx
    L = rx.lib()
    t = rx.BatchTune(4096, 256, 0.0)
    assert L.rx_batch_set_shape(None, ctypes.byref(t)) == 2
    assert L.rx_batch_run(None, None, None, None, None) == 2
    assert L.rx_batch_autotune(None, None, None, None, None, None) == 2
    L.rx_batch_free(None)


def test_no_cpu_fallback_without_the_library(monkeypatch, tmp_path):
    """Without librx.so every call raises: there is no other path."""
    import paper_1108_3126_b300 as rx
    monkeypatch.setattr(rx, "LIB_PATH", str(tmp_path / "librx.so"))
    monkeypatch.setattr(rx, "_lib", None)
    with pytest.raises(RuntimeError):
        rx.lib()
    with pytest.raises(RuntimeError):
        rx.Regex.compile(b"ab", rx.COMPILE_HOST_ONLY)
