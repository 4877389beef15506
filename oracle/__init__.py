"""CPU oracle for whole-string regular-expression matching -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never calls it, and the
two share no code: the oracle reads the node-array input format and nothing
else.

Everything here follows Rathnayake & Thielecke, "Regular Expression Matching
and Operational Semantics" (SOS 2011):

* ``o1`` -- the big-step relation of Fig 2.1 as a least relation, memoised
  (``oracle.c``).
* ``o1_search`` -- unanchored search (not in the paper): the earliest end j
  of a substring w[i:j] that the expression matches, read off the same
  memoised tables of Fig 2.1 (``oracle.c``).
* ``o2_search`` -- the same answer from the machine of Fig 6.1 with the root
  pushed back at every macro step, for texts too long for O1 (``oracle.c``).
* ``o2`` / ``o2_trace`` -- the sequential lockstep machine of Def 6.2 /
  Fig 6.1 with psi of Def 6.1 (``oracle.c``).
* ``cont`` -- Def 4.4 (``oracle.c``).
* ``brute_language`` -- the language of an expression truncated to strings of
  length <= k over a small alphabet, built from the denotational reading of
  Fig 2.1 (union, concatenation, star as the least fixpoint).
* ``glushkov`` -- textbook nullable / first / last / follow sets by
  structural recursion over the syntax (Glushkov's position automaton), an
  independent statement of what the evolution of Def 5.1 reaches.
* ``parse`` -- an independent reading of the library's text syntax.

Pins (what fixes these functions other than themselves) live in
``tests/test_oracle.py``: the worked examples of Fig 4.1, Ex 3.3, Ex 4.6 and
Ex 7.1 (``tests/golden/``), exhaustive comparison with ``brute_language``,
algebraic identities of regular languages, and brute-force Glushkov automata.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

NODE_DTYPE = np.dtype([("kind", "u1"), ("byte", "u1"), ("pad", "<u2"), ("l", "<i4"), ("r", "<i4")])
CHAR, EPS, STAR, CAT, ALT = 0, 1, 2, 3, 4
O1_MAX_BYTES = 1 << 30


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, SRC])
        os.replace(tmp, LIB)
    return LIB


_lib = None


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P, I, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        lib.or_cont.argtypes = [P, I, I, P]
        lib.or_cont.restype = I
        lib.or_o1.argtypes = [P, I, I, P, I64, I64]
        lib.or_o1.restype = I
        lib.or_o2.argtypes = [P, I, I, P, I64, P, P]
        lib.or_o2.restype = I
        lib.or_o2_batch.argtypes = [P, I, I, P, P, I64, P, I]
        lib.or_o2_batch.restype = I
        lib.or_o1_batch.argtypes = [P, I, I, P, P, I64, P, I64, I]
        lib.or_o1_batch.restype = I
        lib.or_o1_search.argtypes = [P, I, I, P, I64, I64]
        lib.or_o1_search.restype = I64
        lib.or_o1_search_batch.argtypes = [P, I, I, P, P, I64, P, I64, I]
        lib.or_o1_search_batch.restype = I
        lib.or_o2_search.argtypes = [P, I, I, P, I64]
        lib.or_o2_search.restype = I64
        lib.or_o2_search_batch.argtypes = [P, I, I, P, P, I64, P, I]
        lib.or_o2_search_batch.restype = I
        lib.or_o2_pairs.argtypes = [P, P, P, I64, P, P, P, I64, P, I]
        lib.or_o2_pairs.restype = I
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a.size else ctypes.c_void_p(0)


def _nodes(nodes) -> np.ndarray:
    nd = np.ascontiguousarray(nodes)
    assert nd.dtype == NODE_DTYPE
    return nd


def _buf(w) -> np.ndarray:
    if isinstance(w, (bytes, bytearray)):
        return np.frombuffer(bytes(w) + b"\0", np.uint8)
    a = np.ascontiguousarray(w, dtype=np.uint8)
    return np.concatenate([a, np.zeros(1, np.uint8)])


# ------------------------------------------------------------------ C side
def cont(nodes, root: int = 0) -> np.ndarray:
    """Def 4.4: cont of every node, -1 for null."""
    nd = _nodes(nodes)
    out = np.empty(len(nd), np.int32)
    if _L().or_cont(_p(nd), len(nd), root, _p(out)) != 0:
        raise ValueError("malformed tree")
    return out


def o1(nodes, w, root: int = 0, max_bytes: int = O1_MAX_BYTES) -> bool:
    """Big-step matching (Fig 2.1), memoised.  Raises MemoryError when the
    tables for this string length would exceed max_bytes."""
    nd = _nodes(nodes)
    b = _buf(w)
    r = _L().or_o1(_p(nd), len(nd), root, _p(b), len(b) - 1, max_bytes)
    if r < 0:
        raise MemoryError("O1 tables too large for this string")
    return bool(r)


def o1_search(nodes, w, root: int = 0, max_bytes: int = O1_MAX_BYTES) -> int:
    """Unanchored search from the big-step tables: the smallest j such that
    some substring w[i:j] (i <= j) is matched (Fig 2.1), or -1.  Raises
    MemoryError when the tables would exceed max_bytes."""
    nd = _nodes(nodes)
    b = _buf(w)
    r = _L().or_o1_search(_p(nd), len(nd), root, _p(b), len(b) - 1, max_bytes)
    if r == -2:
        raise MemoryError("O1 tables too large for this string")
    return int(r)


def o1_search_batch(nodes, data: np.ndarray, offsets: np.ndarray, root: int = 0, threads: int = 0,
                    max_bytes: int = O1_MAX_BYTES) -> np.ndarray:
    """o1_search per string (int64; -2 marks strings whose tables would be
    too large)."""
    nd = _nodes(nodes)
    n = len(offsets) - 1
    out = np.zeros(max(n, 1), np.int64)
    d = np.ascontiguousarray(data, np.uint8)
    if d.size == 0:
        d = np.zeros(1, np.uint8)
    o = np.ascontiguousarray(offsets, np.int64)
    _L().or_o1_search_batch(_p(nd), len(nd), root, _p(d), _p(o), n, _p(out), max_bytes, threads)
    return out[:n]


def o2_search(nodes, w, root: int = 0) -> int:
    """Unanchored search with the machine of Fig 6.1, the root pushed back at
    every macro step: the earliest end of a matching substring, or -1."""
    nd = _nodes(nodes)
    b = _buf(w)
    r = _L().or_o2_search(_p(nd), len(nd), root, _p(b), len(b) - 1)
    if r == -2:
        raise ValueError("malformed tree")
    return int(r)


def o2_search_batch(nodes, data: np.ndarray, offsets: np.ndarray, root: int = 0, threads: int = 0) -> np.ndarray:
    nd = _nodes(nodes)
    n = len(offsets) - 1
    out = np.zeros(max(n, 1), np.int64)
    d = np.ascontiguousarray(data, np.uint8)
    if d.size == 0:
        d = np.zeros(1, np.uint8)
    o = np.ascontiguousarray(offsets, np.int64)
    _L().or_o2_search_batch(_p(nd), len(nd), root, _p(d), _p(o), n, _p(out), threads)
    return out[:n]


def o2(nodes, w, root: int = 0) -> bool:
    """The sequential lockstep machine of Fig 6.1."""
    nd = _nodes(nodes)
    b = _buf(w)
    r = _L().or_o2(_p(nd), len(nd), root, _p(b), len(b) - 1, None, None)
    if r < 0:
        raise ValueError("malformed tree")
    return bool(r)


def o2_trace(nodes, w, root: int = 0):
    """Run Fig 6.1 recording, per macro step k = 0..L, the set of CHAR nodes
    evolved (Def 5.1) and whether null was reached, and per step k < L the
    list n handed to the next macro step.  Returns (accept, evolved, nexts)
    with evolved a list of (frozenset of node ids, null flag) and nexts a list
    of frozensets of node ids (-1 standing for null)."""
    nd = _nodes(nodes)
    b = _buf(w)
    L = len(b) - 1
    nn = len(nd)
    tr = np.zeros((L + 1) * (nn + 1), np.uint8)
    nt = np.zeros(max(L, 1) * (nn + 1), np.uint8)
    r = _L().or_o2(_p(nd), nn, root, _p(b), L, _p(tr), _p(nt))
    if r < 0:
        raise ValueError("malformed tree")
    tr = tr.reshape(L + 1, nn + 1)
    nt = nt.reshape(-1, nn + 1)[:L]
    evolved = [(frozenset(np.nonzero(row[:nn])[0].tolist()), bool(row[nn])) for row in tr]
    nexts = [frozenset([int(i) if i < nn else -1 for i in np.nonzero(row)[0]]) for row in nt]
    return bool(r), evolved, nexts


def o2_batch(nodes, data: np.ndarray, offsets: np.ndarray, root: int = 0, threads: int = 0) -> np.ndarray:
    nd = _nodes(nodes)
    n = len(offsets) - 1
    out = np.zeros(max(n, 1), np.uint8)
    d = np.ascontiguousarray(data, np.uint8)
    if d.size == 0:
        d = np.zeros(1, np.uint8)
    o = np.ascontiguousarray(offsets, np.int64)
    if _L().or_o2_batch(_p(nd), len(nd), root, _p(d), _p(o), n, _p(out), threads) != 0:
        raise ValueError("malformed tree")
    return out[:n]


def o2_pairs(regexes, regex_of, data: np.ndarray, offsets: np.ndarray, threads: int = 0) -> np.ndarray:
    """O2 (Fig 6.1) per (expression, string) pair: pair i is string i
    against regexes[regex_of[i]] (node arrays, root 0).  A plain loop over
    the pairs on `threads` OpenMP threads (0 = all)."""
    regs = [_nodes(r) for r in regexes]
    ns = np.zeros(len(regs) + 1, np.int64)
    ns[1:] = np.cumsum([len(r) for r in regs])
    nd = np.ascontiguousarray(np.concatenate(regs)) if regs else np.zeros(1, NODE_DTYPE)
    roots = np.zeros(max(len(regs), 1), np.int32)
    pr = np.ascontiguousarray(regex_of, np.int32)
    n = len(offsets) - 1
    assert len(pr) == n
    out = np.zeros(max(n, 1), np.uint8)
    d = np.ascontiguousarray(data, np.uint8)
    if d.size == 0:
        d = np.zeros(1, np.uint8)
    o = np.ascontiguousarray(offsets, np.int64)
    if _L().or_o2_pairs(_p(nd), _p(ns), _p(roots), len(regs), _p(pr), _p(d), _p(o), n, _p(out), threads) != 0:
        raise ValueError("malformed tree")
    return out[:n]


def o1_batch(nodes, data: np.ndarray, offsets: np.ndarray, root: int = 0, threads: int = 0,
             max_bytes: int = O1_MAX_BYTES) -> np.ndarray:
    """O1 per string; 255 marks strings whose tables would be too large."""
    nd = _nodes(nodes)
    n = len(offsets) - 1
    out = np.zeros(max(n, 1), np.uint8)
    d = np.ascontiguousarray(data, np.uint8)
    if d.size == 0:
        d = np.zeros(1, np.uint8)
    o = np.ascontiguousarray(offsets, np.int64)
    _L().or_o1_batch(_p(nd), len(nd), root, _p(d), _p(o), n, _p(out), max_bytes, threads)
    return out[:n]


# ------------------------------------------------------------ Python side
def positions(nodes, root: int = 0) -> list:
    """CHAR nodes in left-to-right order (the canonical position numbering)."""
    nd = _nodes(nodes)
    out, stack = [], [root]
    while stack:
        p = stack.pop()
        k = int(nd["kind"][p])
        if k == CHAR:
            out.append(p)
        elif k == STAR:
            stack.append(int(nd["l"][p]))
        elif k in (CAT, ALT):
            stack.append(int(nd["r"][p]))
            stack.append(int(nd["l"][p]))
    return out


def glushkov(nodes, root: int = 0):
    """Glushkov's construction by structural recursion:
    nullable(e), first(e), last(e) and follow(p) for every CHAR node p.
      a     : not nullable, first = last = {a}
      eps   : nullable, first = last = {}
      e1|e2 : nullable = n1 or n2, first = f1 U f2, last = l1 U l2
      e1 e2 : nullable = n1 and n2, first = f1 U (f2 if n1), last = l2 U (l1 if n2),
              follow(p) += f2 for p in l1
      e*    : nullable, first = f, last = l, follow(p) += f for p in l
    Sets hold CHAR node ids."""
    nd = _nodes(nodes)
    follow = {p: set() for p in range(len(nd)) if int(nd["kind"][p]) == CHAR}

    def rec(p):
        k = int(nd["kind"][p])
        if k == CHAR:
            return False, {p}, {p}
        if k == EPS:
            return True, set(), set()
        if k == STAR:
            _, f, l = rec(int(nd["l"][p]))
            for q in l:
                follow[q] |= f
            return True, set(f), set(l)
        n1, f1, l1 = rec(int(nd["l"][p]))
        n2, f2, l2 = rec(int(nd["r"][p]))
        if k == ALT:
            return n1 or n2, f1 | f2, l1 | l2
        for q in l1:
            follow[q] |= f2
        return n1 and n2, f1 | (f2 if n1 else set()), l2 | (l1 if n2 else set())

    import sys
    old = sys.getrecursionlimit()
    sys.setrecursionlimit(max(old, 10000))
    try:
        nullable, first, last = rec(root)
    finally:
        sys.setrecursionlimit(old)
    return nullable, first, last, follow


def glushkov_accepts(nodes, w: bytes, root: int = 0) -> bool:
    """Run the Glushkov position automaton on w by set simulation."""
    nd = _nodes(nodes)
    nullable, first, last, follow = glushkov(nodes, root)
    if len(w) == 0:
        return nullable
    cur = {p for p in first if int(nd["byte"][p]) == w[0]}
    for c in w[1:]:
        nxt = set()
        for p in cur:
            nxt |= follow[p]
        cur = {q for q in nxt if int(nd["byte"][q]) == c}
    return bool(cur & last)


def brute_language(nodes, alphabet: bytes = b"abc", maxlen: int = 8, root: int = 0) -> list:
    """The language of the expression restricted to strings of length <=
    maxlen over ``alphabet``, as a list (index = length) of boolean arrays over
    the k**len strings of that length in base-k order (first symbol most
    significant).  Built denotationally:
      L(a) = {a}, L(eps) = {""}, L(e1|e2) = L(e1) U L(e2),
      L(e1 e2) = {uv}, L(e*) = least X with X = {""} U L(e) X.
    Concatenation of a length-i set with a length-j set is the outer product
    of their indicator vectors, flattened (base-k digits of u then of v)."""
    nd = _nodes(nodes)
    k = len(alphabet)
    idx = {c: i for i, c in enumerate(alphabet)}

    def empty():
        return [np.zeros(k**n, bool) for n in range(maxlen + 1)]

    def concat(A, B):
        out = empty()
        for i in range(maxlen + 1):
            if not A[i].any():
                continue
            for j in range(maxlen + 1 - i):
                if B[j].any():
                    out[i + j] |= np.outer(A[i], B[j]).reshape(-1)
        return out

    def union(A, B):
        return [a | b for a, b in zip(A, B)]

    def rec(p):
        kind = int(nd["kind"][p])
        if kind == CHAR:
            out = empty()
            c = int(nd["byte"][p])
            if c in idx and maxlen >= 1:
                out[1][idx[c]] = True
            return out
        if kind == EPS:
            out = empty()
            out[0][0] = True
            return out
        if kind == ALT:
            return union(rec(int(nd["l"][p])), rec(int(nd["r"][p])))
        if kind == CAT:
            return concat(rec(int(nd["l"][p])), rec(int(nd["r"][p])))
        inner = rec(int(nd["l"][p]))
        X = empty()
        X[0][0] = True
        while True:
            Y = union(X, concat(inner, X))
            if all((a == b).all() for a, b in zip(X, Y)):
                return X
            X = Y

    return rec(root)


def all_strings(alphabet: bytes = b"abc", maxlen: int = 8) -> list:
    """Every string of length <= maxlen in the order brute_language uses."""
    import itertools
    out = []
    for n in range(maxlen + 1):
        for t in itertools.product(alphabet, repeat=n):
            out.append(bytes(t))
    return out


def parse(pattern: bytes) -> np.ndarray:
    """Independent reader of the library's text syntax, returning a node array
    with the root at node 0 (preorder numbering).  Grammar (left-assoc):
        alt  := cat ('|' cat)*
        cat  := post*            (an empty cat is the constant epsilon)
        post := atom '*'*
        atom := '(' alt ')' | '\\e' | '\\xHH' | '\\' any | any byte but |*()
    Raises ValueError(position) on a syntax error."""
    s = bytes(pattern)
    pos = 0

    def err():
        raise ValueError(pos)

    def node(kind, byte=0, l=None, r=None):
        return (kind, byte, l, r)

    def p_alt():
        nonlocal pos
        t = p_cat()
        while pos < len(s) and s[pos] == ord("|"):
            pos += 1
            t = node(ALT, l=t, r=p_cat())
        return t

    def p_cat():
        items = []
        while pos < len(s) and s[pos] not in b"|)":
            items.append(p_post())
        if not items:
            return node(EPS)
        t = items[0]
        for x in items[1:]:
            t = node(CAT, l=t, r=x)
        return t

    def p_post():
        nonlocal pos
        t = p_atom()
        while pos < len(s) and s[pos] == ord("*"):
            pos += 1
            t = node(STAR, l=t)
        return t

    def p_atom():
        nonlocal pos
        c = s[pos]
        if c == ord("("):
            pos += 1
            t = p_alt()
            if pos >= len(s) or s[pos] != ord(")"):
                err()
            pos += 1
            return t
        if c == ord("*"):
            err()
        if c == ord("\\"):
            if pos + 1 >= len(s):
                err()
            d = s[pos + 1]
            if d == ord("e"):
                pos += 2
                return node(EPS)
            if d == ord("x"):
                h = s[pos + 2:pos + 4]
                if len(h) != 2 or any(ch not in b"0123456789abcdefABCDEF" for ch in h):
                    err()
                pos += 4
                return node(CHAR, int(h, 16))
            pos += 2
            return node(CHAR, d)
        pos += 1
        return node(CHAR, c)

    t = p_alt()
    if pos != len(s):
        err()
    rows = []

    def flat(t):
        i = len(rows)
        rows.append(None)
        kind, byte, l, r = t
        li = flat(l) if l is not None else -1
        ri = flat(r) if r is not None else -1
        rows[i] = (kind, byte, 0, li, ri)
        return i

    import sys
    old = sys.getrecursionlimit()
    sys.setrecursionlimit(max(old, 20000))
    try:
        flat(t)
    finally:
        sys.setrecursionlimit(old)
    return np.array(rows, NODE_DTYPE)
