"""Pins for the CPU oracle: what fixes it other than itself.

* the worked examples of the paper (Fig 4.1, Ex 3.3, Ex 4.6, Ex 7.1) from
  ``tests/golden/``;
* exhaustive agreement with the truncated language built denotationally
  (every string of length <= 8 over {a,b,c}) on random small expressions,
  including deliberate epsilon loops;
* identities that hold for regular languages whatever the matcher;
* Glushkov's position automaton (structural recursion) against the same
  brute-force languages;
* O1 (big-step) against O2 (Fig 6.1 machine) on longer strings, as the
  equivalence theorems (Thm 3.2, 4.7, 5.4) require.
Each of these fails under a plausible slip in the oracle: a dropped rule
(Kleene2, Alt2), a wrong cont wiring, a swapped CAT operand, or a missing
psi membership test.
"""
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
ND = oracle.NODE_DTYPE
KIND = {"CHAR": oracle.CHAR, "EPS": oracle.EPS, "STAR": oracle.STAR, "CAT": oracle.CAT, "ALT": oracle.ALT}


def fig41():
    """Read the Fig 4.1 heap: (node array in the figure's numbering, cont)."""
    rows, cont = {}, {}
    for line in open(os.path.join(GOLD, "fig4_1_heap.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        p, kind, a, b, k = line.split()
        i = int(p[1:])
        if kind == "CHAR":
            rows[i] = (oracle.CHAR, ord(a), 0, -1, -1)
        elif kind == "STAR":
            rows[i] = (oracle.STAR, 0, 0, int(a[1:]), -1)
        else:
            rows[i] = (KIND[kind], 0, 0, int(a[1:]), int(b[1:]))
        cont[i] = -1 if k == "null" else int(k[1:])
    nodes = np.array([rows[i] for i in range(len(rows))], ND)
    return nodes, np.array([cont[i] for i in range(len(cont))], np.int32)


def test_fig41_cont():
    nodes, want = fig41()
    assert oracle.cont(nodes, 0).tolist() == want.tolist()


def test_ex71_set_trace():
    nodes, _ = fig41()
    steps, end = [], None
    for line in open(os.path.join(GOLD, "ex7_1_trace.txt")):
        t = line.split()
        if not t or t[0].startswith("#"):
            continue
        if t[0] == "input":
            w = t[1].encode()
        elif t[0] == "step":
            i_ev, i_nx = t.index("evolved"), t.index("next")
            ev = {int(x[1:]) for x in t[i_ev + 1:i_nx]}
            nx = {-1 if x == "null" else int(x[1:]) for x in t[i_nx + 1:]}
            steps.append((ev, nx))
        elif t[0] == "end":
            end = bool(int(t[2]))
    acc, evolved, nexts = oracle.o2_trace(nodes, w, 0)
    assert acc == end
    assert len(nexts) == len(steps) == len(w)
    for k, (ev, nx) in enumerate(steps):
        assert set(evolved[k][0]) == ev and not evolved[k][1]
        assert set(nexts[k]) == nx
    assert evolved[len(w)] == (frozenset(), True)
    assert oracle.o1(nodes, w, 0) == end


def examples():
    out = []
    for line in open(os.path.join(GOLD, "examples.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        cite, pat, inp, want = [x.strip() for x in line.split("|")] if line.count("|") == 3 else _split4(line)
        out.append((cite, pat.encode(), eval(inp, {"__builtins__": {}}), bool(int(want))))
    return out


def _split4(line):
    # patterns may contain '|': the first and the last two fields are fixed
    parts = [x.strip() for x in line.split(" | ")]
    return parts[0], " | ".join(parts[1:-2]), parts[-2], parts[-1]


@pytest.mark.parametrize("cite,pat,w,want", examples())
def test_paper_examples(cite, pat, w, want):
    nodes = oracle.parse(pat)
    assert oracle.o2(nodes, w) == want, cite
    if len(w) <= 2048:
        assert oracle.o1(nodes, w) == want, cite


def test_pointer_equality_positions():
    # Section 3: the two a's of (ab)|(ac) are different positions
    nodes = oracle.parse(b"(ab)|(ac)")
    assert len(oracle.positions(nodes)) == 4


def test_cont_definition_cases():
    # Def 4.4 on each node kind, hand-checked
    n = oracle.parse(b"(a|b)c*")  # CAT(ALT(a,b), STAR(c))
    cat, alt, a, b, star, c = 0, 1, 2, 3, 4, 5
    assert n["kind"].tolist() == [oracle.CAT, oracle.ALT, oracle.CHAR, oracle.CHAR, oracle.STAR, oracle.CHAR]
    k = oracle.cont(n).tolist()
    assert k[cat] == -1 and k[alt] == star and k[a] == star and k[b] == star
    assert k[star] == -1 and k[c] == star


# ------------------------------------------------------------ brute force
ALL = oracle.all_strings(b"abc", 8)
ALL_PACKED = synth.pack(ALL)


def small_regexes(count, seed, max_nodes=12):
    out = []
    for i in range(count):
        size = 1 + i % max_nodes
        out.append(synth.gen_regex(size, 6, b"abc", synth.item_seed(seed, i), eps_loop_p=0.15))
    return out


def test_o1_o2_vs_brute_force():
    for nodes in small_regexes(300, 0xB0)[:300]:
        want = np.concatenate(oracle.brute_language(nodes, b"abc", 8)).astype(np.uint8)
        got1 = oracle.o1_batch(nodes, ALL_PACKED.data, ALL_PACKED.offsets)
        got2 = oracle.o2_batch(nodes, ALL_PACKED.data, ALL_PACKED.offsets)
        pat = synth.to_pattern(nodes)
        assert (got1 == want).all(), pat
        assert (got2 == want).all(), pat


def test_glushkov_vs_brute_force():
    for nodes in small_regexes(25, 0xB1, max_nodes=10):
        want = np.concatenate(oracle.brute_language(nodes, b"abc", 6))
        strs = oracle.all_strings(b"abc", 6)
        got = np.array([oracle.glushkov_accepts(nodes, s) for s in strs])
        assert (got == want).all(), synth.to_pattern(nodes)


def test_brute_language_closed_forms():
    # hand-countable languages: |L((a|b|c)*) cap len<=8| = all 9841 strings,
    # (a|b)(a|b) has exactly 4 strings, a* has 9, (aa)* has 5, eps has 1
    def count(pat):
        return int(sum(x.sum() for x in oracle.brute_language(oracle.parse(pat), b"abc", 8)))

    assert count(b"(a|b|c)*") == 9841
    assert count(b"(a|b)(a|b)") == 4
    assert count(b"a*") == 9
    assert count(b"(aa)*") == 5
    assert count(b"\\e") == 1
    assert count(b"(\\e*|a)*") == 9
    assert count(b"ab*c|b") == 8


def test_identities():
    """e* matches eps; e|e = e; (e*)* = e*; eps e = e; (eps*|e)* = e*;
    e1|e2 = e2|e1; (e1 e2) e3 = e1 (e2 e3); (e1|e2) e3 = e1 e3 | e2 e3."""
    rng = np.random.default_rng(7)
    strs = [bytes(rng.choice(list(b"abc"), size=int(n)).tolist()) for n in rng.integers(0, 12, 150)]
    pk = synth.pack(strs)
    regs = small_regexes(40, 0xB2, max_nodes=9)
    for i, e in enumerate(regs):
        p = synth.to_pattern(e)
        f = synth.to_pattern(regs[(i + 1) % len(regs)])
        g = synth.to_pattern(regs[(i + 2) % len(regs)])
        pairs = [
            (b"(" + p + b")|(" + p + b")", p),
            (b"((" + p + b")*)*", b"(" + p + b")*"),
            (b"\\e(" + p + b")", p),
            (b"(\\e*|(" + p + b"))*", b"(" + p + b")*"),
            (b"(" + p + b")|(" + f + b")", b"(" + f + b")|(" + p + b")"),
            (b"((" + p + b")(" + f + b"))(" + g + b")", b"(" + p + b")((" + f + b")(" + g + b"))"),
            (b"((" + p + b")|(" + f + b"))(" + g + b")", b"(" + p + b")(" + g + b")|(" + f + b")(" + g + b")"),
        ]
        for a, b in pairs:
            na, nb = oracle.parse(a), oracle.parse(b)
            ra = oracle.o2_batch(na, pk.data, pk.offsets)
            rb = oracle.o2_batch(nb, pk.data, pk.offsets)
            assert (ra == rb).all(), (a, b)
            assert (oracle.o1_batch(na, pk.data, pk.offsets) == ra).all(), a
        assert oracle.o1(oracle.parse(b"(" + p + b")*"), b"")


def test_o1_equals_o2_longer_strings():
    for i in range(12):
        e = synth.gen_regex(16 + 4 * i, 8, b"abc", synth.item_seed(0xB3, i), eps_loop_p=0.05)
        s = synth.gen_strings(e, 60, 0, 300, b"abc", synth.item_seed(0xB4, i), p_lang=0.5)
        r1 = oracle.o1_batch(e, s.data, s.offsets)
        r2 = oracle.o2_batch(e, s.data, s.offsets)
        assert (r1 == r2).all(), synth.to_pattern(e)
        # the language samples are members
        lang = s.kind == 1
        assert r2[lang].all()


def test_parse_round_trip_and_errors():
    for i in range(200):
        e = synth.gen_regex(1 + i % 40, 8, synth.ALL_BYTES, synth.item_seed(0xB5, i), eps_loop_p=0.05)
        p = oracle.parse(synth.to_pattern(e))
        assert (p == e).all()
    # precedence: | lowest, then juxtaposition, then postfix *
    n = oracle.parse(b"a|bc*")
    assert n["kind"].tolist() == [oracle.ALT, oracle.CHAR, oracle.CAT, oracle.CHAR, oracle.STAR, oracle.CHAR]
    assert oracle.parse(b"")["kind"].tolist() == [oracle.EPS]
    assert oracle.parse(b"()")["kind"].tolist() == [oracle.EPS]
    assert oracle.parse(b"\\x41")["byte"].tolist() == [0x41]
    for bad, pos in [(b"(", 1), (b")", 0), (b"*a", 0), (b"a(b", 3), (b"\\x4", 0)]:
        with pytest.raises(ValueError) as ei:
            oracle.parse(bad)
        assert ei.value.args[0] == pos, bad


def test_deep_epsilon_loops_terminate():
    # nested (eps*)* towers: only the visited-set of psi stops these loops
    pat = b"((((\\e*)*)*|a)*)*b"
    n = oracle.parse(pat)
    assert oracle.o2(n, b"aaab") and not oracle.o2(n, b"aaa")
    assert oracle.o1(n, b"aaab") and not oracle.o1(n, b"aaa")


# ------------------------------------------------------------ search oracle
def _brute_search(lang_sets, w: bytes) -> int:
    """Earliest end j of a substring w[i:j] in the (truncated) language: the
    definition, checked against sets built denotationally."""
    for j in range(len(w) + 1):
        for i in range(j + 1):
            if w[i:j] in lang_sets[j - i]:
                return j
    return -1


def test_o1_search_vs_brute_force():
    """o1_search against the denotational language on every substring of
    random strings over {a,b,c} of length <= 8 (so every substring is within
    the truncated language)."""
    rng = np.random.default_rng(0xB5)
    for nodes in small_regexes(120, 0xB4):
        lang = oracle.brute_language(nodes, b"abc", 8)
        sets = [set() for _ in range(9)]
        for n in range(9):
            strs = [s for s in oracle.all_strings(b"abc", n) if len(s) == n]
            sets[n] = {s for s, ok in zip(strs, lang[n]) if ok}
        words = [bytes(rng.choice(list(b"abc"), size=int(rng.integers(0, 9))).tolist()) for _ in range(40)]
        pk = synth.pack(words)
        got = oracle.o1_search_batch(nodes, pk.data, pk.offsets)
        for w, g in zip(words, got):
            assert g == _brute_search(sets, w), (synth.to_pattern(nodes), w, g)


def test_o1_search_closed_forms():
    rng = np.random.default_rng(0xB6)
    words = [bytes(rng.choice(list(b"abcx"), size=int(rng.integers(0, 40))).tolist()) for _ in range(300)]
    pk = synth.pack(words)
    lit = oracle.o1_search_batch(oracle.parse(b"ab"), pk.data, pk.offsets)
    cfirst = oracle.o1_search_batch(oracle.parse(b"(a|b)*c"), pk.data, pk.offsets)
    star = oracle.o1_search_batch(oracle.parse(b"a*"), pk.data, pk.offsets)
    twice = oracle.o1_search_batch(oracle.parse(b"x(a|b|c|x)*x"), pk.data, pk.offsets)
    for w, a, b, c, d in zip(words, lit, cfirst, star, twice):
        k = w.find(b"ab")
        assert a == (k + 2 if k >= 0 else -1)
        k = w.find(b"c")
        assert b == (k + 1 if k >= 0 else -1)
        assert c == 0  # nullable: the empty substring at 0
        first = w.find(b"x")
        second = w.find(b"x", first + 1) if first >= 0 else -1
        assert d == (second + 1 if second >= 0 else -1)
    # no string of an empty-ish language: only "" would match \e, found at 0
    assert oracle.o1_search(oracle.parse(b"\\e"), b"abc") == 0
    assert oracle.o1_search(oracle.parse(b"(a*)*b"), b"aaaa") == -1
    assert oracle.o1_search(oracle.parse(b"(a*)*b"), b"aaab") == 4


def test_o2_search_equals_o1_search():
    """The streaming search oracle (Fig 6.1 with the root re-pushed) against
    the big-step one, which the tests above pin to brute force."""
    rng = np.random.default_rng(0xB7)
    for i, nodes in enumerate(small_regexes(150, 0xB8)):
        words = [bytes(rng.choice(list(b"abc"), size=int(rng.integers(0, 60))).tolist()) for _ in range(30)]
        pk = synth.pack(words)
        a = oracle.o1_search_batch(nodes, pk.data, pk.offsets)
        b = oracle.o2_search_batch(nodes, pk.data, pk.offsets)
        assert (a == b).all(), (synth.to_pattern(nodes), np.nonzero(a != b)[0][:5])
    # closed form on a long text
    t = bytes(rng.choice(list(b"abc"), size=200000).tolist()) + b"xyz"
    assert oracle.o2_search(oracle.parse(b"xyz"), t) == len(t)
    assert oracle.o2_search(oracle.parse(b"xyzz"), t) == -1


def test_o2_pairs_is_o2_per_pair_and_o1():
    """The pairs loop decides pair i with O2 for its own expression: it
    equals O2 and O1 called pair by pair, with expressions of different
    sizes (and epsilon loops) interleaved, empty strings included."""
    regs, strs, rid = [], [], []
    for i in range(24):
        e = synth.gen_regex([3, 8, 20, 60][i % 4], 8, b"abc", synth.item_seed(0x0A, i), eps_loop_p=0.2)
        regs.append(e)
        s = synth.gen_strings(e, 12, 0, 40, b"abc", synth.item_seed(0x0B, i), p_lang=0.5)
        strs += [s.get(k) for k in range(s.n)]
        rid += [i] * s.n
    order = np.random.default_rng(3).permutation(len(strs))
    strs = [strs[k] for k in order]
    rid = np.array(rid, np.int32)[order]
    pk = synth.pack(strs)
    got = oracle.o2_pairs(regs, rid, pk.data, pk.offsets, threads=4)
    want2 = np.array([oracle.o2(regs[r], w) for r, w in zip(rid, strs)], np.uint8)
    want1 = np.array([oracle.o1(regs[r], w) for r, w in zip(rid, strs)], np.uint8)
    assert (got == want2).all() and (want1 == want2).all()
    assert 0 < got.sum() < len(got)
