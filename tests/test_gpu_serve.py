"""GPU serving (rx_serve_*): continuous batching gives every request the
same result alone as in a mix with others (exact), under admission by a
device-memory budget, with host or device payloads; results agree with the
CPU oracle."""
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


def workload(seed=0xF0, n_req=300):
    pool = []
    for i in range(12):
        size = [8, 20, 64, 200, 500, 1000][i % 6]
        pool.append(synth.gen_regex(size, 14, synth.LOWER if i % 2 else synth.ALL_BYTES, synth.item_seed(seed, i)))
    # a wide expression without the macro-step cache (warp class)
    pool.append(oracle.parse(b"(" + b"|".join(bytes([97 + j % 26]) + bytes([97 + (j * 7) % 26])
                                               for j in range(300)) + b")*"))
    rng = np.random.default_rng(seed)
    reqs = []
    for k in range(n_req):
        ri = int(rng.integers(0, len(pool)))
        nodes = pool[ri]
        alpha = synth.ALL_BYTES if ri % 2 == 0 and ri < 12 else synth.LOWER
        lmax = int(rng.choice([64, 4096, 70000, 3 << 20], p=[0.4, 0.4, 0.17, 0.03]))
        s = synth.gen_strings(nodes, 1, 0, lmax, alpha, synth.item_seed(seed + 1, k), p_lang=0.6, log_len=True)
        reqs.append((ri, s.get(0)))
    return pool, reqs


def compile_pool(pool):
    out = []
    for i, nd in enumerate(pool):
        out.append(rx.Regex.from_nodes(nd, 0, rx.COMPILE_NO_MEMO if i % 3 == 2 else 0))
    return out


def serve_all(handles, reqs, **kw):
    srv = rx.Server(**kw)
    tickets = {}
    for k, (ri, w) in enumerate(reqs):
        while True:
            try:
                t = srv.submit(handles[ri], w)
                break
            except rx.RxError as e:
                assert e.status == 7  # busy: drain some
                srv.drain(60000)
        tickets[t] = k
    srv.drain(120000)
    res = np.full(len(reqs), 9, np.uint8)
    got = 0
    while got < len(reqs):
        tk, r, st = srv.poll(4096)
        assert (st == 0).all()
        for a, b in zip(tk, r):
            res[tickets[int(a)]] = b
        got += len(tk)
    stats = srv.stats()
    srv.close()
    return res, stats


def test_mix_equals_alone_equals_oracle():
    pool, reqs = workload()
    handles = compile_pool(pool)
    mixed, stats = serve_all(handles, reqs, max_inflight=64, tick_bytes=4096)
    assert stats["completed"] == len(reqs) and stats["p99_ns"] >= stats["p50_ns"] > 0
    assert stats["peak_inflight"] > 1  # requests really overlapped
    for k in range(0, len(reqs), 5):
        alone, _ = serve_all(handles, [reqs[k]], max_inflight=4, tick_bytes=1 << 16)
        assert alone[0] == mixed[k], k
    for k, (ri, w) in enumerate(reqs):
        if len(w) <= 200000:
            assert mixed[k] == oracle.o2(pool[ri], w), (k, len(w))


def test_chunked_long_requests_and_warp_ticks_agree():
    """The three ways a long request can run -- the chunked mode on its own
    stream (long_threshold low), warp ticks (32 spans per tick composed from
    the saved state), and lane ticks only (tick larger than any request) --
    give the same answers, equal to O2."""
    pool, reqs = workload(seed=0xF8, n_req=160)
    handles = compile_pool(pool)
    a, _ = serve_all(handles, reqs, max_inflight=64, tick_bytes=512, long_threshold=8192)
    b, _ = serve_all(handles, reqs, max_inflight=64, tick_bytes=512)
    c, _ = serve_all(handles, reqs, max_inflight=64, tick_bytes=1 << 23)
    assert (a == b).all() and (b == c).all()
    for k, (ri, w) in enumerate(reqs):
        if len(w) <= 200000:
            assert b[k] == oracle.o2(pool[ri], w), (k, len(w))
    # many requests took warp ticks (more than two 512-byte ticks left), some
    # more than 32 of them, and some the chunked mode
    lens = np.array([len(w) for _, w in reqs])
    assert (lens > 1024).sum() >= 20 and (lens > 8192).sum() >= 8 and (lens > 32 * 512 * 2).sum() >= 5


def test_wide_requests_agree():
    """Requests whose set is too wide for one thread (the warp class, a
    sixteenth of the tick bytes per tick), from a few bytes to 600 KB,
    beside short requests of other expressions: every one agrees with O2."""
    wide = oracle.parse(b"(" + b"|".join(bytes([97 + j % 26]) + bytes([97 + (j * 5) % 26])
                                         for j in range(200)) + b")*")
    small = synth.gen_regex(40, 10, synth.LOWER, synth.item_seed(0xF9, 0))
    pool = [wide, small]
    rng = np.random.default_rng(0xF9)
    reqs = []
    for k in range(40):
        ri = k % 2
        lo, hi = ((100 << 10, 600 << 10) if k % 4 == 0 else (0, 60 << 10)) if ri == 0 else (0, 5000)
        s = synth.gen_strings(pool[ri], 1, lo, hi, synth.LOWER, synth.item_seed(0xFA, k), p_lang=0.8)
        reqs.append((ri, s.get(0)))
    handles = [rx.Regex.from_nodes(wide, 0, rx.COMPILE_NO_MEMO), rx.Regex.from_nodes(small)]
    assert handles[0].info()["words"] > 8
    assert sum(len(w) > (64 << 10) for ri, w in reqs if ri == 0) >= 5
    got, _ = serve_all(handles, reqs, max_inflight=64)
    want = np.array([oracle.o2(pool[ri], w) for ri, w in reqs], np.uint8)
    assert (got == want).all(), np.nonzero(got != want)[0]
    assert 0 < want.sum() < len(want)


def test_wide_tier_requests_agree():
    """Expressions of more than 256 positions whose cache of macro steps
    outgrows 192 states get the wide tier (two-byte state ids): each of
    their requests takes warp ticks of 32 chunk functions composed from the
    saved state, whatever its length.  Requests from empty to 1 MB, with
    small ticks so that long ones cross many, agree with O2 and with the
    same expressions served by the bitset warp stepper (no wide tier)."""
    wide = []
    for nd in synth.serving_pool(pool=300):
        inf = rx.Regex.from_nodes(nd, 0, rx.COMPILE_HOST_ONLY).info()
        if inf["memo_states"] == 0 and inf["wide_states"] > 0:
            wide.append(nd)
        if len(wide) == 3:
            break
    small = synth.gen_regex(40, 10, synth.ALL_BYTES, synth.item_seed(0xFD, 0))
    pool = wide + [small]
    rng = np.random.default_rng(0xFD)
    reqs = []
    for k in range(48):
        ri = k % len(pool)
        hi = int(rng.choice([0, 100, 20000, 300000, 1 << 20], p=[0.05, 0.25, 0.35, 0.25, 0.1]))
        w = synth.gen_strings(pool[ri], 1, 0, hi, synth.ALL_BYTES, synth.item_seed(0xFE, k), p_lang=0.7,
                              log_len=True).get(0)
        reqs.append((ri, w))
    sub = synth.pack([w for _, w in reqs])
    want = oracle.o2_pairs(pool, np.array([ri for ri, _ in reqs], np.int32), sub.data, sub.offsets)
    assert 0 < want.sum() < len(want)
    got = {}
    for flags in (0, rx.COMPILE_NO_WIDE):
        handles = [rx.Regex.from_nodes(nd, 0, flags) for nd in pool]
        assert all((h.info()["wide_states"] > 0) == (flags == 0) for h in handles[:3])
        got[flags], _ = serve_all(handles, reqs, max_inflight=32, tick_bytes=1024)
        bad = np.nonzero(got[flags] != want)[0]
        assert bad.size == 0, (flags, bad)


def test_small_budget_admission_is_exact():
    pool, reqs = workload(seed=0xF5, n_req=80)
    handles = compile_pool(pool)
    want, _ = serve_all(handles, reqs, max_inflight=256, tick_bytes=1 << 15)
    tight, st = serve_all(handles, reqs, max_inflight=256, tick_bytes=1000, device_budget_bytes=100000)
    assert (tight == want).all()
    assert st["peak_device_bytes"] <= max(100000, max(len(w) for _, w in reqs) * 3)


def test_device_payload_mode():
    pool, reqs = workload(seed=0xF7, n_req=60)
    handles = compile_pool(pool)
    want, _ = serve_all(handles, reqs, max_inflight=32)
    srv = rx.Server(max_inflight=32, device_payload=True)
    bufs = [torch.from_numpy(np.frombuffer(w + b"\0", np.uint8).copy()).cuda() for _, w in reqs]
    torch.cuda.synchronize()
    tickets = {}
    for k, (ri, w) in enumerate(reqs):
        tickets[srv.submit(handles[ri], bufs[k], len(w))] = k
    srv.drain(60000)
    got = np.full(len(reqs), 9, np.uint8)
    tk, r, st = srv.poll(1000)
    assert (st == 0).all()
    for a, b in zip(tk, r):
        got[tickets[int(a)]] = b
    assert (got == want).all()
    srv.close()


def test_borrowed_host_payload_mode():
    """Payload mode 2: host bytes (page-locked) read by the server when it
    admits a request, with no copy at submit.  Results equal the copying
    mode's, which equal O2 (want); an invalid mode is rejected."""
    pool, reqs = workload(seed=0xF8, n_req=80)
    handles = compile_pool(pool)
    want, _ = serve_all(handles, reqs, max_inflight=32)
    srv = rx.Server(max_inflight=32, device_payload=2)
    bufs = [torch.from_numpy(np.frombuffer(w + b"\0", np.uint8).copy()).pin_memory() for _, w in reqs]
    tickets = {}
    for k, (ri, w) in enumerate(reqs):
        tickets[srv.submit(handles[ri], bufs[k], len(w))] = k
    srv.drain(60000)
    got = np.full(len(reqs), 9, np.uint8)
    tk, r, st = srv.poll(1000)
    assert (st == 0).all()
    for a, b in zip(tk, r):
        got[tickets[int(a)]] = b
    assert (got == want).all()
    assert (want == np.array([oracle.o2(pool[ri], w) for ri, w in reqs], np.uint8)).all()
    srv.close()
    with pytest.raises(rx.RxError):
        rx.Server(device_payload=3)


def test_serving_full_scale_replay_vs_o2():
    """The serving workload at its full scale: 2000 pool expressions plus
    expressions compiled on arrival (20% of requests), 20,000 requests at
    200k req/s through native paced replay, device-resident payloads drawn
    log-uniform from 16 B to 16 MiB (the long ones run the chunked mode).
    Every request with the same (expression, payload) must get the same
    answer, and each of the ~3900 distinct pairs equals O2."""
    pool_nodes = synth.serving_pool(pool=2000)
    pool = [rx.Regex.from_nodes(nd) for nd in pool_nodes]
    rng = np.random.default_rng(0x5EED0005)
    npay = 96
    lens = np.exp(rng.uniform(np.log(16), np.log(16 << 20), npay)).astype(np.int64)
    owners = rng.integers(0, len(pool), npay)
    datas = [synth.gen_strings(pool_nodes[owners[k]], 1, int(lens[k]), int(lens[k]), synth.ALL_BYTES,
                               synth.item_seed(0x5EED0005, 10 + k), p_lang=0.5).data for k in range(npay)]
    bufs = [torch.from_numpy(np.concatenate([x, np.zeros(16, np.uint8)])).cuda() for x in datas]
    fresh_nodes = [synth.gen_regex(int(np.exp(rng.uniform(np.log(8), np.log(1025)))), 14, synth.ALL_BYTES,
                                   synth.item_seed(0x5EED0005, 100000 + k)) for k in range(512)]
    fresh = [rx.Regex.from_nodes(nd) for nd in fresh_nodes]
    torch.cuda.synchronize()
    nreq, rate = 20000, 200000.0
    arrive = np.cumsum(rng.exponential(1.0 / rate, nreq))
    pick = rng.integers(0, npay, nreq)
    reuse = rng.random(nreq) < 0.8
    key = [("p", int(owners[pick[k]])) if reuse[k] else ("f", k % len(fresh)) for k in range(nreq)]
    handles = np.array([(pool[i] if kd == "p" else fresh[i]).handle for kd, i in key], np.uint64)
    payloads = np.array([bufs[int(p)].data_ptr() for p in pick], np.uint64)
    plen = np.array([len(datas[int(p)]) for p in pick], np.int64)
    srv = rx.Server(max_inflight=8192, device_payload=True)
    tickets, _ = srv.replay(handles, payloads, plen, (arrive * 1e9).astype(np.int64))
    srv.drain(600000)
    where = {int(t): k for k, t in enumerate(tickets)}
    res = np.full(nreq, 9, np.uint8)
    got = 0
    while got < nreq:
        tk, r, st = srv.poll(8192)
        assert len(tk) > 0 and (st == 0).all()
        for a, b in zip(tk, r):
            res[where[int(a)]] = b
        got += len(tk)
    stats = srv.stats()
    srv.close()
    assert stats["completed"] == nreq and stats["peak_inflight"] > 1
    seen = {}
    for k in range(nreq):
        pair = (key[k], int(pick[k]))
        assert seen.setdefault(pair, res[k]) == res[k], pair
    for ((kd, i), p), v in seen.items():
        nd = pool_nodes[i] if kd == "p" else fresh_nodes[i]
        assert v == oracle.o2(nd, datas[p].tobytes()), (kd, i, p, len(datas[p]))
    assert 0 < sum(int(v) for v in seen.values()) < len(seen)
