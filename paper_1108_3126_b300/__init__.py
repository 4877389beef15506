"""Python binding of librx.so (include/rx.h): argument marshalling only.

Every step of matching runs in the CUDA kernels of ``csrc/``; this module
converts Python objects (torch tensors, numpy arrays, bytes) into the plain
pointers and sizes of the C ABI and turns non-zero statuses into
``RxError``.  There is no CPU fallback: if ``librx.so`` has not been built,
every call raises.

Device buffers are passed as torch CUDA tensors (or raw integer device
addresses); streams as ``torch.cuda.Stream``, raw ``cudaStream_t`` integers,
or None for torch's current stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librx.so")

NODE_DTYPE = np.dtype([("kind", "u1"), ("byte", "u1"), ("pad", "<u2"), ("l", "<i4"), ("r", "<i4")])
CHAR, EPS, STAR, CAT, ALT = 0, 1, 2, 3, 4

VARIANT_AUTO, VARIANT_MEMO, VARIANT_THREAD, VARIANT_SPARSE, VARIANT_WARP, VARIANT_PAPER = range(6)
VARIANT_NAMES = {0: "auto", 1: "memo", 2: "thread", 3: "sparse", 4: "warp", 5: "paper"}
COMPILE_HOST_ONLY = 1
COMPILE_NO_MEMO = 2
COMPILE_SEARCH = 4
COMPILE_NO_WIDE = 8
RESULT_INVALID = 2      # result byte of a string with invalid offsets
SEARCH_INVALID = -2     # rx_search result of a string with invalid offsets

STATUS = {0: "RX_OK", 1: "RX_ERR_PARSE", 2: "RX_ERR_INVALID_ARG", 3: "RX_ERR_TOO_LARGE", 4: "RX_ERR_OOM",
          5: "RX_ERR_CUDA", 6: "RX_ERR_TIMEOUT", 7: "RX_ERR_BUSY", 8: "RX_ERR_UNSUPPORTED"}


class RxError(RuntimeError):
    def __init__(self, status: int, message: str, err_pos: int | None = None):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.message = message
        self.err_pos = err_pos


class _Info(ctypes.Structure):
    _fields_ = [("nodes", ctypes.c_int32), ("positions", ctypes.c_int32), ("words", ctypes.c_int32),
                ("nullable", ctypes.c_int32), ("memo_states", ctypes.c_int32), ("variants", ctypes.c_uint32),
                ("device_bytes", ctypes.c_int64), ("search_states", ctypes.c_int32), ("wide_states", ctypes.c_int32)]


class _Opts(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("block", ctypes.c_int32), ("sort", ctypes.c_int32),
                ("len_hint", ctypes.c_int32)]


class TuneEntry(ctypes.Structure):
    _fields_ = [("pos_bucket", ctypes.c_int32), ("len_bucket", ctypes.c_int32), ("memo", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("block", ctypes.c_int32), ("gb_per_s", ctypes.c_float)]


class BatchTune(ctypes.Structure):
    _fields_ = [("long_pair_bytes", ctypes.c_int64), ("block", ctypes.c_int32), ("gb_per_s", ctypes.c_float)]


class ServeCfg(ctypes.Structure):
    _fields_ = [("device_budget_bytes", ctypes.c_int64), ("max_inflight", ctypes.c_int32),
                ("queue_capacity", ctypes.c_int32), ("tick_bytes", ctypes.c_int64),
                ("device_payload", ctypes.c_int32), ("long_threshold", ctypes.c_int32)]


class ServeStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("p50_ns", ctypes.c_double),
                ("p99_ns", ctypes.c_double), ("p999_ns", ctypes.c_double), ("max_ns", ctypes.c_double),
                ("req_per_s", ctypes.c_double), ("gb_per_s", ctypes.c_double), ("ticks", ctypes.c_int64),
                ("peak_inflight", ctypes.c_int64), ("peak_device_bytes", ctypes.c_int64)]


# every symbol include/rx.h declares, with its ctypes signature
P, I32, U32, I64, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_int64, ctypes.c_size_t
SIGNATURES = {
    "rx_compile": ([ctypes.c_char_p, SZ, U32, ctypes.POINTER(P), ctypes.POINTER(SZ)], I32),
    "rx_compile_ast": ([P, SZ, I32, U32, ctypes.POINTER(P)], I32),
    "rx_info": ([P, ctypes.POINTER(_Info)], I32),
    "rx_free": ([P], None),
    "rx_tables": ([P, P, P, P, P, P, P], I32),
    "rx_tree": ([P, P, SZ, ctypes.POINTER(SZ)], I32),
    "rx_match": ([P, SZ, P, P, P, P], I32),
    "rx_match_ex": ([P, SZ, P, P, P, P, ctypes.POINTER(_Opts)], I32),
    "rx_match_static": ([P, SZ, P, P, P, P], I32),
    "rx_match_host": ([P, SZ, P, P, P, P], I32),
    "rx_device_faults": ([I32], I64),
    "rx_sync_check": ([P, ctypes.POINTER(I64)], I32),
    "rx_search": ([P, SZ, P, P, P, P], I32),
    "rx_search_long": ([P, P, I64, I64, P, P], I32),
    "rx_match_batch": ([P, SZ, P, P, P, P], I32),
    "rx_match_pairs": ([P, SZ, P, P, P, P], I32),
    "rx_batch_prepare": ([P, SZ, ctypes.POINTER(P)], I32),
    "rx_batch_run": ([P, P, P, P, P], I32),
    "rx_batch_autotune": ([P, P, P, P, P, ctypes.POINTER(BatchTune)], I32),
    "rx_batch_set_shape": ([P, ctypes.POINTER(BatchTune)], I32),
    "rx_batch_free": ([P], None),
    "rx_match_long": ([P, P, I64, I64, P, P], I32),
    "rx_match_seq": ([P, P, I64, P, P], I32),
    "rx_trace": ([P, P, I64, P, P], I32),
    "rx_serve_create": ([ctypes.POINTER(ServeCfg), ctypes.POINTER(P)], I32),
    "rx_serve_submit": ([P, P, P, I64, ctypes.POINTER(ctypes.c_uint64)], I32),
    "rx_serve_poll": ([P, P, P, P, SZ], SZ),
    "rx_serve_replay": ([P, P, P, P, P, SZ, P, ctypes.POINTER(I64)], I32),
    "rx_serve_drain": ([P, I64], I32),
    "rx_serve_stats": ([P, ctypes.POINTER(ServeStats)], I32),
    "rx_serve_destroy": ([P], I32),
    "rx_autotune": ([P, SZ, P, P, P, P, ctypes.POINTER(TuneEntry)], I32),
    "rx_autotune_table": ([P, SZ], SZ),
    "rx_autotune_reset": ([], None),
    "rx_profile_enable": ([I32], I32),
    "rx_profile_read": ([ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(ctypes.c_double)], I32),
    "rx_last_error": ([], ctypes.c_char_p),
    "rx_version": ([], ctypes.c_char_p),
}

_lib = None


def lib():
    """Load librx.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1108_3126_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def last_error() -> str:
    return lib().rx_last_error().decode(errors="replace")


def _check(status: int, err_pos: int | None = None):
    if status != 0:
        raise RxError(status, last_error(), err_pos)


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if isinstance(x, np.ndarray):
        return int(x.ctypes.data)
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(s) -> int:
    if s is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)


class Regex:
    """A compiled expression (owns an rx_handle)."""

    def __init__(self, handle: int):
        self._h = handle

    @classmethod
    def compile(cls, pattern, flags: int = 0) -> "Regex":
        pat = pattern.encode("latin-1") if isinstance(pattern, str) else bytes(pattern)
        h = P()
        ep = SZ(0)
        st = lib().rx_compile(pat, len(pat), flags, ctypes.byref(h), ctypes.byref(ep))
        _check(st, int(ep.value) if st == 1 else None)
        return cls(h.value)

    @classmethod
    def from_nodes(cls, nodes: np.ndarray, root: int = 0, flags: int = 0) -> "Regex":
        nd = np.ascontiguousarray(nodes)
        if nd.dtype != NODE_DTYPE:
            nd = nd.astype(NODE_DTYPE)
        h = P()
        _check(lib().rx_compile_ast(nd.ctypes.data, len(nd), root, flags, ctypes.byref(h)))
        return cls(h.value)

    @property
    def handle(self) -> int:
        if not self._h:
            raise ValueError("regex was freed")
        return self._h

    def info(self) -> dict:
        i = _Info()
        _check(lib().rx_info(self.handle, ctypes.byref(i)))
        return {f: getattr(i, f) for f, _ in _Info._fields_}

    def tables(self) -> dict:
        inf = self.info()
        nn, m, W = inf["nodes"], inf["positions"], inf["words"]
        cont = np.zeros(nn, np.int32)
        pos_node = np.zeros(max(m, 1), np.int32)
        pos_bit = np.zeros(max(m, 1), np.int32)
        null_bit = ctypes.c_int32(0)
        start = np.zeros(W, np.uint32)
        follow = np.zeros(max(m, 1) * W, np.uint32)
        _check(lib().rx_tables(self.handle, cont.ctypes.data, pos_node.ctypes.data, pos_bit.ctypes.data,
                               ctypes.addressof(null_bit), start.ctypes.data, follow.ctypes.data))
        return {"cont": cont, "pos_node": pos_node[:m], "pos_bit": pos_bit[:m], "null_bit": int(null_bit.value),
                "start": start, "follow": follow[:m * W].reshape(m, W), "words": W}

    def tree(self) -> np.ndarray:
        n = SZ(0)
        _check(lib().rx_tree(self.handle, None, 0, ctypes.byref(n)))
        out = np.zeros(n.value, NODE_DTYPE)
        _check(lib().rx_tree(self.handle, out.ctypes.data, n.value, ctypes.byref(n)))
        return out

    def free(self):
        if self._h:
            lib().rx_free(self._h)
            self._h = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def match(rx: Regex, strings, offsets, out, n: int | None = None, stream=None, variant: int = 0,
          block: int = 0, sort: int = -1, len_hint: int = 0):
    """out[i] = 1 iff the expression matches strings[offsets[i]:offsets[i+1]] (async)."""
    if n is None:
        n = len(offsets) - 1
    o = _Opts(variant, block, sort, min(int(len_hint), 2**31 - 1))
    _check(lib().rx_match_ex(rx.handle, n, _ptr(strings), _ptr(offsets), _ptr(out), _stream(stream),
                             ctypes.byref(o)))


def match_static(rx: Regex, strings, offsets, out, n: int | None = None, stream=None):
    """As match(), with no device allocation by the library: scratch is a
    fixed array inside librx.so (at most 262,144 strings per call; calls
    that overlap on the GPU race on it)."""
    if n is None:
        n = len(offsets) - 1
    _check(lib().rx_match_static(rx.handle, n, _ptr(strings), _ptr(offsets), _ptr(out), _stream(stream)))


def search(rx: Regex, strings, offsets, out_end, n: int | None = None, stream=None):
    """out_end[i] (int64) = earliest end of a substring of string i that the
    expression matches, -1 if none (async; the handle must be compiled with
    COMPILE_SEARCH)."""
    if n is None:
        n = len(offsets) - 1
    _check(lib().rx_search(rx.handle, n, _ptr(strings), _ptr(offsets), _ptr(out_end), _stream(stream)))


def search_long(rx: Regex, text, length: int, out_end, chunk_bytes: int = 0, stream=None):
    """out_end[0] (int64, device) = earliest end of a matching substring of
    one long device text, chunked (async; COMPILE_SEARCH handles)."""
    _check(lib().rx_search_long(rx.handle, _ptr(text), length, chunk_bytes, _ptr(out_end), _stream(stream)))


def device_faults(reset: bool = False) -> int:
    """Bounded device waits that gave up since the last reset (0 normally)."""
    return int(lib().rx_device_faults(1 if reset else 0))


def sync_check(stream=None, raise_error: bool = True) -> int:
    """Synchronise the stream and return (clearing it) the device's count of
    strings the kernels found with invalid offsets since the last check.
    A non-zero count raises RxError (RX_ERR_INVALID_ARG) unless
    raise_error is False."""
    bad = I64(0)
    st = lib().rx_sync_check(_stream(stream), ctypes.byref(bad))
    if st != 0 and (raise_error or st != 2):
        raise RxError(st, last_error())
    return int(bad.value)


def match_host(rx: Regex, strings, offsets, out, n: int | None = None, stream=None):
    """As match(), on HOST buffers (numpy arrays or CPU tensors, pinned for
    full link speed): copies to the device overlap the matching of the
    previous piece; returns when out is written."""
    if n is None:
        n = len(offsets) - 1
    _check(lib().rx_match_host(rx.handle, n, _ptr(strings), _ptr(offsets), _ptr(out), _stream(stream)))


def _handles(regexes) -> np.ndarray:
    if isinstance(regexes, np.ndarray):
        return np.ascontiguousarray(regexes, np.uint64)
    return np.array([r.handle for r in regexes], np.uint64)


def handle_array(regexes) -> np.ndarray:
    """Host array of raw handles (pass to match_batch / match_pairs to avoid
    rebuilding it on every call)."""
    return _handles(regexes)


def match_batch(regexes, strings, offsets, out, stream=None):
    """Pair i = (regexes[i], string i), one persistent launch (async)."""
    hs = _handles(regexes)
    _check(lib().rx_match_batch(hs.ctypes.data, len(hs), _ptr(strings), _ptr(offsets), _ptr(out),
                                _stream(stream)))


class Batch:
    """A prepared batch: pair i = (regexes[i], string i) for a fixed list of
    expressions; run() replays a captured CUDA graph of the batched launch."""

    def __init__(self, regexes):
        self._hs = _handles(regexes)
        self._keep = None if isinstance(regexes, np.ndarray) else list(regexes)
        self.n = len(self._hs)
        h = P()
        _check(lib().rx_batch_prepare(self._hs.ctypes.data, self.n, ctypes.byref(h)))
        self.handle = h.value

    def run(self, strings, offsets, out, stream=None):
        _check(lib().rx_batch_run(self.handle, _ptr(strings), _ptr(offsets), _ptr(out), _stream(stream)))

    def autotune(self, strings, offsets, out, stream=None) -> dict:
        t = BatchTune()
        _check(lib().rx_batch_autotune(self.handle, _ptr(strings), _ptr(offsets), _ptr(out), _stream(stream),
                                       ctypes.byref(t)))
        return {"long_pair_bytes": int(t.long_pair_bytes), "block": int(t.block), "gb_per_s": float(t.gb_per_s)}

    def set_shape(self, block: int, long_pair_bytes: int):
        """Fix the launch shape of later runs (e.g. one autotune() chose)."""
        t = BatchTune(int(long_pair_bytes), int(block), 0.0)
        _check(lib().rx_batch_set_shape(self.handle, ctypes.byref(t)))

    def free(self):
        if getattr(self, "handle", None):
            lib().rx_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def match_pairs(regexes, strings, offsets, out, stream=None):
    """The plain form: one launch per pair (async)."""
    hs = _handles(regexes)
    _check(lib().rx_match_pairs(hs.ctypes.data, len(hs), _ptr(strings), _ptr(offsets), _ptr(out),
                                _stream(stream)))


def match_long(rx: Regex, text, length: int, out, chunk_bytes: int = 0, stream=None):
    _check(lib().rx_match_long(rx.handle, _ptr(text), length, chunk_bytes, _ptr(out), _stream(stream)))


def match_seq(rx: Regex, text, length: int, out, stream=None):
    _check(lib().rx_match_seq(rx.handle, _ptr(text), length, _ptr(out), _stream(stream)))


def trace(rx: Regex, text, length: int, frontiers, stream=None):
    _check(lib().rx_trace(rx.handle, _ptr(text), length, _ptr(frontiers), _stream(stream)))


def _tune_dict(e: TuneEntry) -> dict:
    return {f: getattr(e, f) for f, _ in TuneEntry._fields_}


def autotune(rx: Regex, strings, offsets, out, n: int | None = None, stream=None) -> dict:
    """Time every variant/block choice on this sample batch and record the
    fastest for the expression's bucket (synchronises the stream)."""
    if n is None:
        n = len(offsets) - 1
    e = TuneEntry()
    _check(lib().rx_autotune(rx.handle, n, _ptr(strings), _ptr(offsets), _ptr(out), _stream(stream),
                             ctypes.byref(e)))
    return _tune_dict(e)


def tune_table() -> list:
    k = lib().rx_autotune_table(None, 0)
    arr = (TuneEntry * max(k, 1))()
    k = lib().rx_autotune_table(arr, k)
    return [_tune_dict(arr[i]) for i in range(k)]


def tune_reset():
    lib().rx_autotune_reset()


def profile_enable(on: bool = True):
    """Time every main lockstep kernel with CUDA events on its stream."""
    _check(lib().rx_profile_enable(int(on)))


def profile_read():
    """(library kernel launches, timed main-kernel launches, their summed ms)
    since the last read."""
    a, b, c = I64(0), I64(0), ctypes.c_double(0)
    _check(lib().rx_profile_read(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return int(a.value), int(b.value), float(c.value)


class Server:
    """Continuous-batching matcher (rx_serve_*)."""

    def __init__(self, device_budget_bytes: int = 0, max_inflight: int = 256, queue_capacity: int = 65536,
                 tick_bytes: int = 0, device_payload=False, long_threshold: int = 0):
        """device_payload: False/0 host bytes copied at submit, True/1 device
        pointers, 2 host bytes borrowed until polled (pin them)."""
        cfg = ServeCfg(device_budget_bytes, max_inflight, queue_capacity, tick_bytes, int(device_payload),
                       long_threshold)
        h = P()
        _check(lib().rx_serve_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._s = h.value

    def submit(self, rx: Regex, data, length: int | None = None) -> int:
        t = ctypes.c_uint64(0)
        if isinstance(data, (bytes, bytearray)):
            buf = bytes(data)
            ptr = ctypes.cast(ctypes.c_char_p(buf), ctypes.c_void_p).value if buf else 0
            length = len(buf)
        else:
            ptr = _ptr(data)
            assert length is not None
        _check(lib().rx_serve_submit(self._s, rx.handle, ptr, length, ctypes.byref(t)))
        return int(t.value)

    def replay(self, handles: np.ndarray, payloads: np.ndarray, lens: np.ndarray, arrival_ns: np.ndarray):
        """Submit request i at arrival_ns[i] after the call starts (native
        pacing); returns (tickets, largest lateness in ns)."""
        n = len(lens)
        hs = np.ascontiguousarray(handles, np.uint64)
        ps = np.ascontiguousarray(payloads, np.uint64)
        ls = np.ascontiguousarray(lens, np.int64)
        ar = np.ascontiguousarray(arrival_ns, np.int64)
        tk = np.zeros(max(n, 1), np.uint64)
        late = I64(0)
        _check(lib().rx_serve_replay(self._s, hs.ctypes.data, ps.ctypes.data, ls.ctypes.data, ar.ctypes.data, n,
                                     tk.ctypes.data, ctypes.byref(late)))
        return tk[:n], int(late.value)

    def poll(self, max_n: int = 4096):
        tick = np.zeros(max_n, np.uint64)
        res = np.zeros(max_n, np.uint8)
        st = np.zeros(max_n, np.int32)
        k = lib().rx_serve_poll(self._s, tick.ctypes.data, res.ctypes.data, st.ctypes.data, max_n)
        return tick[:k], res[:k], st[:k]

    def drain(self, timeout_ms: int = 60000):
        _check(lib().rx_serve_drain(self._s, timeout_ms))

    def stats(self) -> dict:
        s = ServeStats()
        _check(lib().rx_serve_stats(self._s, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in ServeStats._fields_}

    def close(self):
        if self._s:
            _check(lib().rx_serve_destroy(self._s))
            self._s = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
