"""Seeded synthetic workloads for regular-expression matching.

This package only produces inputs (expression trees in the node-array format,
strings, long texts, request streams).  It holds none of the matching
arithmetic: both the CPU oracle and the GPU library consume what it writes.
The heavy lifting is in ``synth.c`` (splitmix64 streams, one independent
substream per item, so results do not depend on thread count).

Node array format (numpy ``NODE_DTYPE``, 12 bytes per node): ``kind`` u8
(0 CHAR, 1 EPS, 2 STAR, 3 CAT, 4 ALT), ``byte`` u8, ``pad`` u16, ``l`` i32,
``r`` i32 (-1 when absent).  Generated trees have their root at node 0.

Workload recipes follow the five benchmark configurations (seed base
``0x5EED0000 + config number``):

1. small: one 16-node expression (depth <= 6) over ``abc``; 4096 strings with
   lengths uniform in [0, 256], half language samples, half uniform random.
2. streaming: one 64-node expression (depth <= 10) over ``a..z``; 1,048,576
   strings with lengths uniform in [1, 1024], half language samples, half
   language samples with 1-3 random edits.
3. batched: 10,000 expressions of 8-512 nodes (log-uniform, depth <= 12, 5%
   deliberate ``(eps*|e)*`` loops) over all 256 bytes; 1-64 strings each
   (log-uniform count), lengths log-uniform in [1, 65536], half language.
4. long: ``(R)*`` with R holding 48 character positions over ``a..z``; one
   1 GiB text made of concatenated language samples of R.
5. serving: Poisson request stream over a pool of 2000 expressions of 8-1024
   nodes (log-uniform), 80% pool reuse, string lengths log-uniform 16 B-16 MiB.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "synth.c")
LIB = os.path.join(HERE, "libsynth.so")

NODE_DTYPE = np.dtype([("kind", "u1"), ("byte", "u1"), ("pad", "<u2"), ("l", "<i4"), ("r", "<i4")])
CHAR, EPS, STAR, CAT, ALT = 0, 1, 2, 3, 4
MIX = (0.40, 0.05, 0.25, 0.15, 0.15)  # char, eps, cat, alt, star
LOWER = bytes(range(ord("a"), ord("z") + 1))
ABC = b"abc"
ALL_BYTES = bytes(range(256))
SEED_BASE = 0x5EED0000


def build(force: bool = False) -> str:
    """Compile synth.c into libsynth.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class _Strings(ctypes.Structure):
    _fields_ = [
        ("bytes", ctypes.POINTER(ctypes.c_uint8)),
        ("offsets", ctypes.POINTER(ctypes.c_int64)),
        ("total", ctypes.c_int64),
        ("n_fallback", ctypes.c_int64),
        ("kind", ctypes.POINTER(ctypes.c_uint8)),
    ]


_lib = None


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.sy_gen_regex.argtypes = [ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_uint64, P, ctypes.c_int]
        lib.sy_gen_regex.restype = ctypes.c_int
        lib.sy_gen_strings.argtypes = [P, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                       ctypes.c_int, ctypes.c_double, ctypes.c_int, P, ctypes.c_int,
                                       ctypes.c_uint64, ctypes.POINTER(_Strings)]
        lib.sy_gen_strings.restype = ctypes.c_int
        lib.sy_gen_star_text.argtypes = [P, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64, P,
                                         ctypes.POINTER(ctypes.c_int64)]
        lib.sy_gen_star_text.restype = ctypes.c_int
        lib.sy_uniform.argtypes = [P, ctypes.c_int64, P, ctypes.c_int, ctypes.c_uint64]
        lib.sy_uniform.restype = None
        lib.sy_uniform_f64.argtypes = [P, ctypes.c_int64, ctypes.c_uint64]
        lib.sy_uniform_f64.restype = None
        lib.sy_item_seed.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.sy_item_seed.restype = ctypes.c_uint64
        lib.sy_free.argtypes = [ctypes.POINTER(_Strings)]
        lib.sy_free.restype = None
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def item_seed(seed: int, i: int) -> int:
    return int(_L().sy_item_seed(seed & (2**64 - 1), i))


def uniform_f64(n: int, seed: int) -> np.ndarray:
    out = np.empty(n, np.float64)
    _L().sy_uniform_f64(_ptr(out), n, seed & (2**64 - 1))
    return out


# ------------------------------------------------------------------ trees
def gen_regex(nodes: int, max_depth: int, alphabet: bytes, seed: int, mix=MIX, eps_loop_p: float = 0.0) -> np.ndarray:
    """Random tree with ``nodes`` nodes (root = 0, preorder numbering)."""
    cap = nodes + 8
    out = np.zeros(cap, NODE_DTYPE)
    mixa = np.asarray(mix, np.float64)
    alpha = np.frombuffer(bytes(alphabet), np.uint8).copy()
    n = _L().sy_gen_regex(nodes, max_depth, _ptr(mixa), _ptr(alpha), len(alpha), eps_loop_p,
                          seed & (2**64 - 1), _ptr(out), cap)
    if n < 0:
        raise RuntimeError("sy_gen_regex failed")
    return out[:n].copy()


def n_positions(nodes: np.ndarray) -> int:
    return int(np.count_nonzero(nodes["kind"] == CHAR))


def make_nodes(spec) -> np.ndarray:
    """Build a node array from a nested tuple spec: ('char', b), ('eps',),
    ('star', e), ('cat', e1, e2), ('alt', e1, e2).  Preorder numbering."""
    rows = []

    def rec(s):
        i = len(rows)
        rows.append(None)
        tag = s[0]
        if tag == "char":
            c = s[1]
            rows[i] = (CHAR, c if isinstance(c, int) else ord(c), 0, -1, -1)
        elif tag == "eps":
            rows[i] = (EPS, 0, 0, -1, -1)
        elif tag == "star":
            c = rec(s[1])
            rows[i] = (STAR, 0, 0, c, -1)
        elif tag in ("cat", "alt"):
            a = rec(s[1])
            b = rec(s[2])
            rows[i] = (CAT if tag == "cat" else ALT, 0, 0, a, b)
        else:
            raise ValueError(tag)
        return i

    rec(spec)
    return np.array(rows, NODE_DTYPE)


def to_pattern(nodes: np.ndarray, root: int = 0) -> bytes:
    """Render a tree in the library's text syntax: '|' lowest, juxtaposition,
    postfix '*', parentheses, '\\e' for the constant epsilon, '\\xHH' and
    backslash escapes for special or unprintable bytes.  Both binary operators
    associate to the left, so parsing the result gives back the same tree."""
    special = set(b"|*()\\")

    def lit(c: int) -> bytes:
        if c in special:
            return b"\\" + bytes([c])
        if 0x21 <= c <= 0x7E:
            return bytes([c])
        return b"\\x%02x" % c

    def rec(p: int) -> bytes:
        k = int(nodes["kind"][p])
        l, r = int(nodes["l"][p]), int(nodes["r"][p])
        if k == CHAR:
            return lit(int(nodes["byte"][p]))
        if k == EPS:
            return b"\\e"
        if k == STAR:
            ck = int(nodes["kind"][l])
            s = rec(l)
            return (b"(" + s + b")" if ck in (CAT, ALT) else s) + b"*"
        if k == CAT:
            a, b = rec(l), rec(r)
            if int(nodes["kind"][l]) == ALT:
                a = b"(" + a + b")"
            if int(nodes["kind"][r]) in (ALT, CAT):
                b = b"(" + b + b")"
            return a + b
        a, b = rec(l), rec(r)
        if int(nodes["kind"][r]) == ALT:
            b = b"(" + b + b")"
        return a + b"|" + b

    return rec(root)


# ---------------------------------------------------------------- strings
@dataclass
class Strings:
    data: np.ndarray  # uint8 [total]
    offsets: np.ndarray  # int64 [n+1]
    kind: np.ndarray  # uint8 [n]: 0 uniform, 1 language, 2 edited language, 3 fallback
    n_fallback: int

    @property
    def n(self) -> int:
        return len(self.offsets) - 1

    def get(self, i: int) -> bytes:
        return self.data[self.offsets[i]:self.offsets[i + 1]].tobytes()


def gen_strings(nodes: np.ndarray, n: int, lmin: int, lmax: int, alphabet: bytes, seed: int, *,
                p_lang: float = 0.5, edited: bool = False, log_len: bool = False) -> Strings:
    """n strings for one tree.  Per item: target length uniform (or
    log-uniform) in [lmin, lmax]; with probability p_lang a language sample,
    otherwise a uniform random string (edited=False) or a language sample
    with 1-3 random edits (edited=True)."""
    res = _Strings()
    nd = np.ascontiguousarray(nodes)
    alpha = np.frombuffer(bytes(alphabet), np.uint8).copy()
    rc = _L().sy_gen_strings(_ptr(nd), len(nd), n, lmin, lmax, int(log_len), p_lang, int(edited), _ptr(alpha),
                             len(alpha), seed & (2**64 - 1), ctypes.byref(res))
    if rc != 0:
        raise RuntimeError("sy_gen_strings failed")
    try:
        total = res.total
        data = np.ctypeslib.as_array(res.bytes, shape=(max(total, 1),))[:total].copy()
        offs = np.ctypeslib.as_array(res.offsets, shape=(n + 1,)).copy()
        kind = np.ctypeslib.as_array(res.kind, shape=(max(n, 1),))[:n].copy()
    finally:
        _L().sy_free(ctypes.byref(res))
    return Strings(data, offs, kind, int(res.n_fallback))


def pack(strs) -> Strings:
    """Pack a list of bytes objects."""
    lens = np.array([len(s) for s in strs], np.int64)
    offs = np.zeros(len(strs) + 1, np.int64)
    np.cumsum(lens, out=offs[1:])
    data = np.frombuffer(b"".join(strs), np.uint8).copy() if strs else np.zeros(0, np.uint8)
    return Strings(data, offs, np.zeros(len(strs), np.uint8), 0)


def uniform_bytes(length: int, alphabet: bytes, seed: int) -> np.ndarray:
    out = np.empty(max(length, 1), np.uint8)
    alpha = np.frombuffer(bytes(alphabet), np.uint8).copy()
    _L().sy_uniform(_ptr(out), length, _ptr(alpha), len(alpha), seed & (2**64 - 1))
    return out[:length]


def star_text(nodes: np.ndarray, total: int, seed: int, piece: int = 4096, with_end: bool = False):
    """A text of ``total`` bytes in the language of (e)* cut at ``total``:
    whole language samples of e (target lengths uniform in [1, piece])
    concatenated, so every prefix stays a prefix of a member of (e)*.  With
    ``with_end`` also returns an offset where a member of (e)* ends (the end
    of the last whole ~1 MiB segment of samples)."""
    out = np.empty(max(total, 1), np.uint8)
    nd = np.ascontiguousarray(nodes)
    last = ctypes.c_int64(0)
    rc = _L().sy_gen_star_text(_ptr(nd), len(nd), total, piece, seed & (2**64 - 1), _ptr(out), ctypes.byref(last))
    if rc != 0:
        raise RuntimeError("sy_gen_star_text failed (language of e holds no non-empty string?)")
    return (out[:total], int(last.value)) if with_end else out[:total]


def wrap_star(nodes: np.ndarray) -> np.ndarray:
    """(e)* with the new star as node 0 (the tree is renumbered by +1)."""
    out = np.zeros(len(nodes) + 1, NODE_DTYPE)
    out[1:] = nodes
    for f in ("l", "r"):
        col = out[f][1:]
        out[f][1:] = np.where(col >= 0, col + 1, -1)
    out[0] = (STAR, 0, 0, 1, -1)
    return out


# ---------------------------------------------------------------- configs
@dataclass
class Workload:
    name: str
    regexes: list  # list of node arrays
    strings: Strings  # packed strings of all pairs
    regex_of: np.ndarray  # int32 [n]: expression index of each string


def cfg_small(seed: int = SEED_BASE + 1, n: int = 4096) -> Workload:
    nodes = gen_regex(16, 6, ABC, item_seed(seed, 0))
    s = gen_strings(nodes, n, 0, 256, ABC, item_seed(seed, 1), p_lang=0.5)
    return Workload("small", [nodes], s, np.zeros(n, np.int32))


def cfg_streaming(seed: int = SEED_BASE + 2, n: int = 1 << 20) -> Workload:
    nodes = gen_regex(64, 10, LOWER, item_seed(seed, 0))
    s = gen_strings(nodes, n, 1, 1024, LOWER, item_seed(seed, 1), p_lang=0.5, edited=True)
    return Workload("streaming", [nodes], s, np.zeros(n, np.int32))


def cfg_batched(seed: int = SEED_BASE + 3, n_regex: int = 10000, max_len: int = 65536,
                max_strings: int = 64) -> Workload:
    """Many expressions, uneven pairs; strings of expression k are contiguous."""
    regexes, parts, rid = [], [], []
    u = uniform_f64(3 * n_regex, item_seed(seed, 0))
    for k in range(n_regex):
        size = int(math.floor(math.exp(math.log(8) + (math.log(513) - math.log(8)) * u[3 * k])))
        size = min(max(size, 8), 512)
        nodes = gen_regex(size, 12, ALL_BYTES, item_seed(seed, 10 + 2 * k), eps_loop_p=0.05)
        cnt = int(math.floor(math.exp(math.log(max_strings + 1) * u[3 * k + 1])))
        cnt = min(max(cnt, 1), max_strings)
        s = gen_strings(nodes, cnt, 1, max_len, ALL_BYTES, item_seed(seed, 11 + 2 * k), p_lang=0.5, log_len=True)
        regexes.append(nodes)
        parts.append(s)
        rid.append(np.full(cnt, k, np.int32))
    data = np.concatenate([p.data for p in parts]) if parts else np.zeros(0, np.uint8)
    lens = np.concatenate([np.diff(p.offsets) for p in parts]) if parts else np.zeros(0, np.int64)
    offs = np.zeros(len(lens) + 1, np.int64)
    np.cumsum(lens, out=offs[1:])
    kind = np.concatenate([p.kind for p in parts]) if parts else np.zeros(0, np.uint8)
    return Workload("batched", regexes, Strings(data, offs, kind, sum(p.n_fallback for p in parts)),
                    np.concatenate(rid) if rid else np.zeros(0, np.int32))


def long_regex(seed: int = SEED_BASE + 4, positions: int = 48) -> np.ndarray:
    """A tree over a..z with exactly ``positions`` character leaves (depth
    <= 12): the first seed of the item stream whose tree has that count."""
    for k in range(100000):
        size = 100 + (k % 60)
        nodes = gen_regex(size, 12, LOWER, item_seed(seed, 1000 + k))
        if n_positions(nodes) == positions:
            return nodes
    raise RuntimeError("no tree with the requested position count")


def cfg_long(seed: int = SEED_BASE + 4, total: int = 1 << 30, with_end: bool = False):
    """(R)* with 48 positions and one text of ``total`` bytes in its prefix
    language.  Returns (nodes of (R)*, text[, an offset where a member ends])."""
    r = long_regex(seed)
    text, end = star_text(r, total, item_seed(seed, 1), with_end=True)
    return (wrap_star(r), text, end) if with_end else (wrap_star(r), text)


def serving_pool(seed: int = SEED_BASE + 5, pool: int = 2000) -> list:
    u = uniform_f64(pool, item_seed(seed, 0))
    out = []
    for k in range(pool):
        size = int(math.floor(math.exp(math.log(8) + (math.log(1025) - math.log(8)) * u[k])))
        size = min(max(size, 8), 1024)
        out.append(gen_regex(size, 14, ALL_BYTES, item_seed(seed, 100 + k)))
    return out
