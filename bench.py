"""Benchmark: matched input GB/s of the lockstep matcher on B300.

Headline workload (N=1): one random 64-node expression over a..z against
1,048,576 strings with lengths uniform in [1, 1024] (~537 MB packed, int64
offsets), half language samples and half edited language samples, seeded.
A step is one call of the public batch entry point (rx_match: one launch in
which each block orders its own strings by length in shared memory and runs
the lockstep steps and the accept test) over the whole batch, inputs
resident in HBM (537 MB, larger than the 126 MB L2, so no flush is needed
between steps).

At N=1 the same JSON line also carries, under "configs", the other four
workloads: small (16 nodes, 4096 strings; with Section 8's machine timed on
a sample), batched (10,000 expressions, 148,077 pairs, prepared batch against
one launch per pair), long (1 GiB text, chunked against sequential) and
serving (Poisson sweep, device and host payloads, against one synchronous
call per request), each with its roofline fraction, the oracle on the host
cores and the clocks seen.  --workload runs one of them alone.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload streaming|small|batched|long|serving] [--no-extra]

Under torchrun each rank runs the headline workload on its own GPU
(replicas, weak scaling); rank 0 prints one JSON line.  --impl reference
times the CPU oracle (the Fig 6.1 machine) on a bounded sample of the
headline workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "matched input GB/s (bit-exact) & % of HBM roofline; serving p50/p99 latency"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


# DRAM bytes (read + write) per launch of the dominant kernel from an ncu
# capture, keyed by a hash of that kernel's sources at capture time (null
# when they have changed since).  Captured on the full launch (1,048,576
# strings, 0.55 GB on the device): 564.86 MB read + 5.59 MB written.
TRAFFIC = {("k_stream_local<MemoPairA>", "0c96693f52f5b019"): 570.5e6}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("stream.cu", "steppers.cuh", "rx_internal.h", "plan.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1108_3126_b300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


STREAMING_WORKLOAD = ("streaming: 1 regex x 64 AST nodes (depth<=10) over a..z; 1,048,576 strings L~U[1,1024] "
                      "(half language samples, half 1-3 random edits); int64 offsets")


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The largest value over all ranks (timing aggregation: the job is as
    slow as its slowest rank).  Works with gloo (CPU) and nccl (CUDA)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_baseline_streaming(w, seconds_budget: float = 12.0, max_strings: int = 200000):
    """The oracle (Fig 6.1 machine, as it stands) on the host cores over a
    bounded prefix of the workload; returns (GB/s, cores, description)."""
    import oracle
    cores = len(os.sched_getaffinity(0))
    nodes = w.regexes[0]
    s = w.strings
    # probe 2000 strings to size the sample to the budget
    k = min(2000, s.n)
    t = time.perf_counter()
    oracle.o2_batch(nodes, s.data, s.offsets[:k + 1], threads=cores)
    dt = max(time.perf_counter() - t, 1e-6)
    rate = s.offsets[k] / dt
    target_bytes = rate * seconds_budget
    n = int(np.searchsorted(s.offsets, target_bytes))
    n = max(1000, min(n, max_strings, s.n))
    t = time.perf_counter()
    oracle.o2_batch(nodes, s.data, s.offsets[:n + 1], threads=cores)
    dt = time.perf_counter() - t
    nbytes = int(s.offsets[n])
    return nbytes / dt / 1e9, cores, f"first {n} strings ({nbytes / 1e6:.1f} MB) of the workload, O2 on {cores} threads"


def cpu_baseline_o1(w, cores: int, n: int = 300):
    """The memoised big-step oracle (O1, Fig 2.1) on the first n strings,
    one thread and all threads; GB/s each."""
    import oracle
    nodes, s = w.regexes[0], w.strings
    n = min(n, s.n)
    res = {}
    for th in (1, cores):
        t = time.perf_counter()
        oracle.o1_batch(nodes, s.data, s.offsets[:n + 1], threads=th)
        res[f"GB/s_{th}_threads"] = round(int(s.offsets[n]) / (time.perf_counter() - t) / 1e9, 4)
    res["sample"] = f"first {n} strings ({int(s.offsets[n]) / 1e6:.1f} MB)"
    return res


def run_reference(args, world, rank):
    """CPU oracle arm: each step = O2 over a bounded sample of the workload."""
    if rank != 0:
        return
    import oracle
    import synth
    w = synth.cfg_streaming()
    cores = len(os.sched_getaffinity(0))
    nodes = w.regexes[0]
    s = w.strings
    total_steps = args.steps + args.warmup
    per_step = int(min(20000, max(64, 20000 * 20 // max(total_steps, 1))))
    times, nbytes = [], []
    for i in range(total_steps):
        a = (i * per_step) % max(s.n - per_step, 1)
        sub_off = s.offsets[a:a + per_step + 1] - s.offsets[a]
        sub = s.data[s.offsets[a]:s.offsets[a + per_step]]
        t = time.perf_counter()
        oracle.o2_batch(nodes, sub, sub_off, threads=cores)
        dt = time.perf_counter() - t
        if i >= args.warmup:
            times.append(dt)
            nbytes.append(int(sub_off[-1]))
    tot_t, tot_b = sum(times), sum(nbytes)
    val = tot_b / tot_t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": STREAMING_WORKLOAD, "strings": s.n, "total_bytes": int(s.offsets[-1]),
                       "sample_strings_per_step": per_step},
            "cpu_baseline": {"value": val, "unit": "GB/s", "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} consecutive strings per step, O2 (Fig 6.1 machine), {cores} threads"},
            "e2e": {"value": val, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_streaming(args, world, rank, local):
    import torch
    import torch.distributed as dist

    import paper_1108_3126_b300 as rx
    import synth
    from paper_1108_3126_b300 import build as rxbuild

    rxbuild.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = synth.cfg_streaming(n=args.strings)
    nodes = w.regexes[0]
    s = w.strings
    n = s.n
    total_bytes = int(s.offsets[-1])
    d_str = torch.from_numpy(s.data).to(dev)
    d_off = torch.from_numpy(s.offsets).to(dev)
    d_out = torch.zeros(n, dtype=torch.uint8, device=dev)
    t0 = time.perf_counter()
    r = rx.Regex.from_nodes(nodes)
    compile_us = (time.perf_counter() - t0) * 1e6
    info = r.info()
    stream = torch.cuda.current_stream(dev)
    variant = {"auto": 0, "memo": 1, "thread": 2, "sparse": 3, "warp": 4}[args.variant]
    # with --autotune the autotuner measures every variant / block choice on
    # this batch once (before the timed region) and rx_match's automatic
    # choice uses it; by default the library's built-in choice is used (the
    # tuner's earlier result for this bucket), so profiled runs of the same
    # command launch the same kernels
    rx.tune_reset()
    tuned = rx.autotune(r, d_str, d_off, d_out, n=n, stream=stream) if (variant == 0 and args.autotune) else None

    def step():
        rx.match(r, d_str, d_off, d_out, n=n, stream=stream, variant=variant)

    step()
    torch.cuda.synchronize(dev)
    # the clock sampler starts first; the warm-up steps then run right before
    # the timed region, so the GPU is busy (not ramping up from idle) when
    # timing begins
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    rx.profile_read()
    rx.profile_enable(True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    rx.profile_enable(False)
    ms = e0.elapsed_time(e1) / args.steps
    launches, timed, kms = rx.profile_read()
    clk = clocks.stop()
    ms = max_over_ranks(ms, world, dev)
    value = world * total_bytes / (ms * 1e-3) / 1e9
    # the timed kernel of a step is the streaming kernel (one launch per
    # step); the planner and the launch gaps are the rest of the step
    kernel_ms = kms / max(args.steps, 1)
    alg_bytes = total_bytes + 8 * (n + 1) + n
    peak, peak_kind = peaks()
    achieved = alg_bytes / (kernel_ms * 1e-3) / 1e9
    accepted = int(d_out.sum().item())

    # the other kernel variants on the same batch (informational)
    variants = {}
    for name, v, blk, srt in ((("memo_pair", 1, 0, -1), ("memo_pair_planner_apart", 1, 0, 2),
                               ("memo_pair_tma32x3", 1, 4, -1), ("memo_pair_tma64x2", 1, 12, -1),
                               ("memo_pair_tma64x3", 1, 20, -1), ("memo_single", 1, 257, -1),
                               ("thread", 2, 0, -1), ("sparse", 3, 0, -1), ("warp", 4, 0, -1))
                              if not args.quick else ()):
        if not (info["variants"] >> v) & 1:
            continue
        reps = max(3, min(50, args.steps // 20))
        for _ in range(2):
            rx.match(r, d_str, d_off, d_out, n=n, stream=stream, variant=v, block=blk, sort=srt)
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            rx.match(r, d_str, d_off, d_out, n=n, stream=stream, variant=v, block=blk, sort=srt)
        b.record(stream)
        torch.cuda.synchronize(dev)
        vms = a.elapsed_time(b) / reps
        variants[name] = {"GB/s": round(total_bytes / (vms * 1e-3) / 1e9, 1), "ms": round(vms, 4)}

    # unanchored search over the same batch (earliest end of a matching
    # substring), informational
    search = None
    if not args.quick:
        rs = rx.Regex.from_nodes(nodes, 0, rx.COMPILE_SEARCH)
        if rs.info()["search_states"]:
            d_end = torch.empty(n, dtype=torch.int64, device=dev)
            for _ in range(2):
                rx.search(rs, d_str, d_off, d_end, n=n, stream=stream)
            sms = _time(lambda: rx.search(rs, d_str, d_off, d_end, n=n, stream=stream), 20, stream, dev)
            search = {"GB/s": round(total_bytes / (sms * 1e-3) / 1e9, 1), "ms": round(sms, 4),
                      "search_states": rs.info()["search_states"], "found": int((d_end >= 0).sum().item()),
                      "note": "batch bytes / time; a string is read only up to its first match"}
        rs.free()

    # end to end through the public API with host buffers: compile the
    # expression, then rx_match_host (strings + offsets from pinned host
    # memory, copies of each 64 MiB piece overlapped with matching the
    # previous one, booleans read back)
    h_str = torch.from_numpy(s.data).pin_memory()
    h_off = torch.from_numpy(s.offsets).pin_memory()
    h_out = torch.empty(n, dtype=torch.uint8).pin_memory()
    e2e_steps = max(3, min(20, args.steps // 100))

    def e2e_step():
        rr = rx.Regex.from_nodes(nodes)
        rx.match_host(rr, h_str, h_off, h_out, n=n, stream=stream)
        rr.free()

    if args.quick:
        e2e_steps = 1
    e2e_step()
    if world > 1:
        dist.barrier()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    b.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = a.elapsed_time(b) / e2e_steps
    e2e_ms = max_over_ranks(e2e_ms, world, dev)
    e2e_val = world * total_bytes / (e2e_ms * 1e-3) / 1e9
    if not torch.equal(h_out, d_out.cpu()):
        raise SystemExit("rx_match_host disagrees with rx_match on the same batch")
    # the host-to-device link alone: the same bytes copied from pinned memory
    # (the ceiling of the end-to-end rate)
    scratch = torch.empty_like(d_str)
    link_ms = _time(lambda: (scratch.copy_(h_str, non_blocking=True), d_off.copy_(h_off, non_blocking=True)),
                    max(3, e2e_steps), stream, dev)
    link_gbs = total_bytes / (link_ms * 1e-3) / 1e9
    del scratch

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.quick:
        v, cores, desc = cpu_baseline_streaming(w)
        cpu = {"value": v, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": desc,
               "o1_big_step": cpu_baseline_o1(w, cores)}

    if rank != 0:
        return
    chosen_v = tuned["variant"] if tuned else (variant or (1 if info["memo_states"] else 2))
    chosen_b = tuned["block"] if tuned else 0
    # the block-local kernel takes the absolute-address form of the two-byte
    # cache when it fits in 3 planes of 8 states (MemoPairT::abs_fits)
    local = "k_stream_local<MemoPairA>" if 0 < info["memo_states"] <= 24 else "k_stream_local<MemoPairP>"
    kname = {1: ("k_stream<MemoS>" if (chosen_b & 1) or not info.get("pair", True) else
                 "k_stream_tma<MemoPairP>" if chosen_b & 28 else
                 local if chosen_b in (0, 768) and n >= 4096 else "k_stream<MemoPairP>"),
             2: "k_stream<Thread1S|Thread2S>", 3: "k_thread<SparseStep>", 4: "k_warp"}[chosen_v]
    src_hash = kernel_source_hash()
    traffic = TRAFFIC.get((kname, src_hash))
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 5), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": STREAMING_WORKLOAD,
                   "total_bytes": total_bytes, "strings": n, "positions": info["positions"],
                   "memo_states": info["memo_states"], "variant": args.variant,
                   "l2": "inputs (537 MB) larger than the 126 MB L2; no flush",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "kernel": kname, "kernel_ms": round(kernel_ms, 5),
                     "algorithmic_bytes_per_launch": alg_bytes, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"
                     if peak_kind == "measured" else "fallback 6.4 TB/s"},
        "e2e": {"value": round(e2e_val, 2), "unit": "GB/s", "h2d_bytes_per_step": total_bytes + 8 * (n + 1),
                "d2h_bytes_per_step": n, "includes": "rx_compile_ast + rx_match_host (H2D, match, D2H) per step",
                "h2d_link_gbs": round(link_gbs, 2), "of_link": round(e2e_val / link_gbs, 3)},
        "gpu_launches": int(launches),
        "gpu_launches_per_step": launches / args.steps,
        "device_faults": rx.device_faults(),
        "clocks": clk,
        "cpu_baseline": cpu,
        "variants": variants,
        "search": search,
        "autotune": tuned,
        "compile_us": round(compile_us, 1),
        "accepted": accepted,
        "kernel_src": src_hash,
    }
    # the other four configurations (N=1 only), each with its forms, roofline
    # fraction, oracle baseline and clocks, as extra keys of this line
    if world == 1 and not args.quick and not args.no_extra:
        extra = {}
        for name, fn in CONFIG_RESULTS.items():
            t0 = time.perf_counter()
            extra[name] = fn(args, dev)
            extra[name]["wall_s"] = round(time.perf_counter() - t0, 1)
        line["configs"] = extra
    print(json.dumps(line))


def _dev_setup(local):
    import torch
    from paper_1108_3126_b300 import build as rxbuild
    rxbuild.build()
    torch.cuda.set_device(local)
    return torch.device("cuda", local)


def _time(fn, reps, stream, dev):
    import torch
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize(dev)
    return a.elapsed_time(b) / reps


MIN_SECONDS = [0.3]  # --min-seconds


def _timed(fn, stream, dev, min_s: float | None = None, max_reps: int = 2000, min_reps: int = 3):
    """Mean ms of fn over enough repetitions to last about min_s (default
    --min-seconds; CUDA events on `stream`), and the number of repetitions."""
    if min_s is None:
        min_s = MIN_SECONDS[0]
    one = _time(fn, 1, stream, dev)
    reps = int(max(min_reps, min(max_reps, (min_s * 1e3) / max(one, 1e-3))))
    return _time(fn, reps, stream, dev), reps


def _roofline(alg_bytes, kernel_ms, kernel, step_ms=None):
    peak, kind = peaks()
    ach = alg_bytes / (kernel_ms * 1e-3) / 1e9 if kernel_ms else None
    d = {"bound": "hbm", "kernel": kernel, "kernel_ms": round(kernel_ms, 5) if kernel_ms else None,
         "algorithmic_bytes_per_launch": int(alg_bytes), "achieved": round(ach, 1) if ach else None,
         "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4) if ach else None,
         "peak_source": f"{kind} (MEASURED_PEAKS.json hbm_gbs)" if kind == "measured" else "fallback 6.4 TB/s"}
    if step_ms:
        d["step_frac"] = round(alg_bytes / (step_ms * 1e-3) / 1e9 / peak, 4)
    return d


def _cpu_o2(fn_sample, budget_s: float, k0: int = 1):
    """Time the oracle's O2 (as it stands) on a bounded sample: fn_sample(k)
    runs O2 on the first k units and returns (bytes, description, all units
    done); k grows until one run takes about budget_s.  Returns (GB/s,
    description) of the last run."""
    k = k0
    while True:
        t = time.perf_counter()
        nbytes, desc, done = fn_sample(k)
        dt = time.perf_counter() - t
        if dt >= 0.5 * budget_s or done:
            return nbytes / max(dt, 1e-9) / 1e9, desc
        k = max(k + 1, int(k * min(16.0, budget_s / max(dt, 1e-3))))


def cfg_small_result(args, dev):
    """Config 1 (plain method, small): one 16-node expression over {a,b,c},
    4096 strings of 0-256 bytes.  The streaming form (rx_match), the batched
    form (rx_match_batch and a prepared batch), the plain form (one launch
    per pair), Section 8's machine (one launch per micro-step, a sample of
    strings), the oracle on the host cores; plus the plain form's per-launch
    cost on 1-byte strings."""
    import torch
    import oracle
    import paper_1108_3126_b300 as rx
    import synth
    w = synth.cfg_small()
    nodes, s = w.regexes[0], w.strings
    n, total = s.n, int(s.offsets[-1])
    r = rx.Regex.from_nodes(nodes)
    d_str = torch.from_numpy(s.data).to(dev)
    d_off = torch.from_numpy(s.offsets).to(dev)
    out = torch.zeros(n, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    want = oracle.o2_batch(nodes, s.data, s.offsets)
    clocks = Clocks(dev.index)
    clocks.start()
    forms = {}

    def check(name):
        torch.cuda.synchronize(dev)
        if not (out.cpu().numpy() == want).all():
            raise SystemExit(f"config 1: {name} disagrees with O2")

    for _ in range(3):
        rx.match(r, d_str, d_off, out, n=n, stream=stream)
    check("rx_match")
    rx.profile_read()
    rx.profile_enable(True)
    ms, reps = _timed(lambda: rx.match(r, d_str, d_off, out, n=n, stream=stream), stream, dev)
    rx.profile_enable(False)
    launches, timed, kms = rx.profile_read()
    kernel_ms = kms / max(timed, 1)
    forms["streaming"] = {"ms": round(ms, 5), "GB/s": round(total / (ms * 1e-3) / 1e9, 3),
                          "launches_per_call": round(launches / reps, 2)}
    hs = rx.handle_array([r] * n)
    rx.match_batch(hs, d_str, d_off, out, stream=stream)
    check("rx_match_batch")
    ms_b, _ = _timed(lambda: rx.match_batch(hs, d_str, d_off, out, stream=stream), stream, dev)
    forms["batched_call"] = {"ms": round(ms_b, 5), "GB/s": round(total / (ms_b * 1e-3) / 1e9, 3)}
    plan = rx.Batch(hs)
    plan.run(d_str, d_off, out, stream=stream)
    check("prepared batch")
    ms_p, _ = _timed(lambda: plan.run(d_str, d_off, out, stream=stream), stream, dev)
    plan.free()
    forms["batched_prepared"] = {"ms": round(ms_p, 5), "GB/s": round(total / (ms_p * 1e-3) / 1e9, 3)}
    out.fill_(7)
    rx.match_pairs(hs, d_str, d_off, out, stream=stream)
    check("rx_match_pairs")
    ms_pl = _time(lambda: rx.match_pairs(hs, d_str, d_off, out, stream=stream), 2, stream, dev)
    forms["plain_per_pair"] = {"ms": round(ms_pl, 3), "GB/s": round(total / (ms_pl * 1e-3) / 1e9, 4),
                               "launches": n, "us_per_pair": round(1e3 * ms_pl / n, 2)}
    # the plain form's fixed cost per pair: the same number of 1-byte strings
    one = synth.pack([b"a"] * n)
    o_str, o_off = torch.from_numpy(one.data).to(dev), torch.from_numpy(one.offsets).to(dev)
    ms_1 = _time(lambda: rx.match_pairs(hs, o_str, o_off, out, stream=stream), 2, stream, dev)
    forms["plain_per_pair"]["us_per_pair_1_byte"] = round(1e3 * ms_1 / n, 2)
    # Section 8's machine: one launch per micro-step, flags read back by the
    # host; timed on the first strings of the batch
    k = args.paper_strings
    sub = synth.Strings(s.data[:s.offsets[k]], s.offsets[:k + 1], s.kind[:k], 0)
    p_str, p_off = torch.from_numpy(sub.data).to(dev), torch.from_numpy(sub.offsets).to(dev)
    pout = torch.zeros(k, dtype=torch.uint8, device=dev)
    t0 = time.perf_counter()
    rx.match(r, p_str, p_off, pout, n=k, stream=stream, variant=rx.VARIANT_PAPER)
    torch.cuda.synchronize(dev)
    pdt = time.perf_counter() - t0
    if not (pout.cpu().numpy() == want[:k]).all():
        raise SystemExit("config 1: Section 8 machine disagrees with O2")
    pbytes = int(sub.offsets[-1])
    forms["paper_section8"] = {"strings": k, "bytes": pbytes, "s": round(pdt, 3),
                               "GB/s": round(pbytes / pdt / 1e9, 6), "ms_per_string": round(1e3 * pdt / k, 2)}
    clk = clocks.stop()
    # the oracle on the host cores, the whole batch repeated to ~2 s
    cores = len(os.sched_getaffinity(0))

    def o2_rep(kk):
        for _ in range(kk):
            oracle.o2_batch(nodes, s.data, s.offsets, threads=cores)
        return kk * total, f"the whole batch x{kk}, O2 on {cores} threads", False

    cpu_v, cpu_desc = _cpu_o2(o2_rep, 2.0) if not args.no_cpu_baseline else (None, "skipped")
    t = time.perf_counter()
    oracle.o1_batch(nodes, s.data, s.offsets, threads=cores)
    o1_gbs = total / (time.perf_counter() - t) / 1e9
    st = forms["streaming"]
    return {"workload": "small: 1 regex x 16 AST nodes (depth<=6) over {a,b,c}; 4096 strings L~U[0,256], "
                        "half language samples, half uniform random",
            "value": st["GB/s"], "unit": "GB/s", "ms_per_step": st["ms"], "strings": n, "total_bytes": total,
            "accepted": int(want.sum()), "forms": forms,
            "roofline": _roofline(total + 8 * (n + 1) + n, kernel_ms, "k_stream (rx_match)", st["ms"]),
            "batched_over_plain": round(ms_pl / ms_p, 1), "streaming_over_paper_section8":
                round(st["GB/s"] / max(forms["paper_section8"]["GB/s"], 1e-12), 1),
            "cpu_baseline": {"value": cpu_v, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": cpu_desc,
                             "o1_big_step_GB/s": round(o1_gbs, 5)},
            "clocks": clk, "parity": "every string equal to O2 (each form)"}


def cfg_batched_result(args, dev):
    """Config 3: 10,000 expressions x 1-64 strings each, one persistent
    launch (prepared batch replayed from its captured graph, after the
    launch-shape autotuner), against one launch per pair."""
    import torch
    import oracle
    import paper_1108_3126_b300 as rx
    import synth
    t0 = time.perf_counter()
    w = synth.cfg_batched(n_regex=args.regexes)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    handles = [rx.Regex.from_nodes(nd) for nd in w.regexes]
    compile_s = time.perf_counter() - t0
    hs = rx.handle_array([handles[i] for i in w.regex_of])
    s = w.strings
    n, total = s.n, int(s.offsets[-1])
    d_str = torch.from_numpy(s.data).to(dev)
    d_off = torch.from_numpy(s.offsets).to(dev)
    out = torch.zeros(n, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    clocks = Clocks(dev.index)
    clocks.start()
    # one call per step, nothing prepared
    for _ in range(3):
        rx.match_batch(hs, d_str, d_off, out, stream=stream)
    rx.profile_read()
    rx.profile_enable(True)
    ms_call, _ = _timed(lambda: rx.match_batch(hs, d_str, d_off, out, stream=stream), stream, dev)
    rx.profile_enable(False)
    launches, timed, kms = rx.profile_read()
    kernel_ms = kms / max(timed, 1)
    res_batch = out.cpu().numpy().copy()
    # prepared batch: expressions fixed once, every step a replay of the
    # captured graph, after the launch-shape autotuner
    plan = rx.Batch(hs)
    tuned = None
    if args.long_pair_bytes > 0:
        plan.set_shape(args.batch_block, args.long_pair_bytes)
    elif not args.no_autotune:
        tuned = plan.autotune(d_str, d_off, out, stream=stream)
    for _ in range(3):
        plan.run(d_str, d_off, out, stream=stream)
    ms, reps = _timed(lambda: plan.run(d_str, d_off, out, stream=stream), stream, dev)
    if not (out.cpu().numpy() == res_batch).all():
        raise SystemExit("prepared batch disagrees with rx_match_batch")
    plan.free()
    out.fill_(7)
    rx.match_pairs(hs, d_str, d_off, out, stream=stream)  # warm
    plain_ms = _time(lambda: rx.match_pairs(hs, d_str, d_off, out, stream=stream), 1, stream, dev)
    if not (out.cpu().numpy() == res_batch).all():
        raise SystemExit("batched and plain forms disagree")
    # the plain form's fixed cost per pair: 1-byte strings for the first
    # 20,000 pairs' expressions
    k1 = min(n, 20000)
    one = synth.pack([b"a"] * k1)
    o_str, o_off = torch.from_numpy(one.data).to(dev), torch.from_numpy(one.offsets).to(dev)
    ms_1 = _time(lambda: rx.match_pairs(hs[:k1], o_str, o_off, out[:k1], stream=stream), 1, stream, dev)
    clk = clocks.stop()
    cores = len(os.sched_getaffinity(0))
    rng = np.random.default_rng(0x5EED0003)
    perm = rng.permutation(n)

    def o2_pairs(kk):
        kk = min(kk, n)
        idx = np.sort(perm[:kk])
        sub = synth.pack([s.get(int(i)) for i in idx])
        got = oracle.o2_pairs(w.regexes, w.regex_of[idx], sub.data, sub.offsets, threads=cores)
        if not (got == res_batch[idx]).all():
            raise SystemExit("batched form disagrees with O2")
        mb = int(sub.offsets[-1]) / 1e6
        return int(sub.offsets[-1]), f"{kk} random pairs ({mb:.1f} MB), O2 on {cores} threads, equal to the GPU", \
            kk >= n

    cpu_v, cpu_desc = _cpu_o2(o2_pairs, args.cpu_seconds, 2000) if not args.no_cpu_baseline else (None, "skipped")
    infos = [h.info() for h in handles]
    for h in handles:
        h.free()
    value = total / (ms * 1e-3) / 1e9
    return {"workload": f"batched uneven: {len(handles)} regexes 8-512 AST nodes (log-uniform, depth<=12, "
                        "5% (eps*|e)* loops) over 256 bytes; 1-64 strings each, L log-uniform 1 B-64 KiB",
            "value": round(value, 2), "unit": "GB/s", "ms_per_step": round(ms, 4), "steps": reps,
            "pairs": n, "total_bytes": total, "positions_max": max(i["positions"] for i in infos),
            "memo_share": round(sum(1 for i in infos if i["memo_states"]) / len(infos), 3),
            "gen_s": round(gen_s, 1), "compile_s": round(compile_s, 2),
            "form": "prepared batch, graph replay" + (" (autotuned)" if tuned else ""), "autotune": tuned,
            "unprepared_call": {"ms": round(ms_call, 4), "GB/s": round(total / (ms_call * 1e-3) / 1e9, 2),
                                "gpu_launches_per_call": launches / max(timed, 1)},
            "plain_per_pair": {"ms": round(plain_ms, 2), "GB/s": round(total / (plain_ms * 1e-3) / 1e9, 3),
                               "launches": n, "us_per_pair": round(1e3 * plain_ms / n, 2),
                               "us_per_pair_1_byte": round(1e3 * ms_1 / k1, 2)},
            "batched_over_plain": round(plain_ms / ms, 1),
            "roofline": _roofline(total + 8 * (n + 1) + n, kernel_ms, "k_batch (unprepared call)", ms),
            "cpu_baseline": {"value": cpu_v, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": cpu_desc},
            "clocks": clk, "accepted": int(res_batch.sum())}


def cfg_long_result(args, dev):
    """Config 4: one 1 GiB text against (R)* with 48 positions: exact
    chunked mode (rx_match_long) against the one-thread sequential run
    (rx_match_seq), the oracle on one host core."""
    import torch
    import oracle
    import paper_1108_3126_b300 as rx
    import synth
    nodes, text, end = synth.cfg_long(total=args.long_bytes, with_end=True)
    r = rx.Regex.from_nodes(nodes)
    d = torch.from_numpy(text).to(dev)
    n = len(text)
    out = torch.zeros(1, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    clocks = Clocks(dev.index)
    clocks.start()
    for _ in range(3):
        rx.match_long(r, d, n, out, stream=stream)
    rx.profile_read()
    rx.profile_enable(True)
    ms, reps = _timed(lambda: rx.match_long(r, d, n, out, stream=stream), stream, dev)
    rx.profile_enable(False)
    launches, timed, kms = rx.profile_read()
    chunked = int(out.item())
    pre = min(n, args.seq_bytes)
    seq_ms = _time(lambda: rx.match_seq(r, d, pre, out, stream=stream), 1, stream, dev)
    rx.match_long(r, d, pre, out, stream=stream)
    torch.cuda.synchronize(dev)
    agree_prefix = int(out.item())
    rx.match_seq(r, d, pre, out, stream=stream)
    torch.cuda.synchronize(dev)
    if int(out.item()) != agree_prefix:
        raise SystemExit("chunked and sequential runs disagree")
    clk = clocks.stop()
    # mean size of the active set along the first 256 KiB (GPU set trace)
    tl = min(n, 256 << 10)
    W = r.tables()["words"]
    rows = torch.zeros((tl + 1) * W, dtype=torch.int32, device=dev)
    rx.trace(r, d, tl, rows, stream=stream)
    torch.cuda.synchronize(dev)
    rw = rows.cpu().numpy().view(np.uint32)
    mean_active = float(np.unpackbits(rw.view(np.uint8)).sum()) / (tl + 1)

    def o2_prefix(kk):
        nb = min(n, kk << 20)
        want = oracle.o2(nodes, text[:nb])
        rx.match_long(r, d, nb, out, stream=stream)
        torch.cuda.synchronize(dev)
        if int(out.item()) != int(want):
            raise SystemExit("chunked mode disagrees with O2 on a prefix")
        return nb, f"first {nb >> 20} MiB of the text, O2 on 1 thread (equal to the chunked GPU result)", nb >= n

    cpu_v, cpu_desc = _cpu_o2(o2_prefix, args.cpu_seconds, 4) if not args.no_cpu_baseline else (None, "skipped")
    kernel_ms = kms / max(reps, 1)
    return {"workload": "long text: (R)* with 48 positions over a..z, one 1 GiB text of concatenated language "
                        "samples of R", "value": round(n / (ms * 1e-3) / 1e9, 2), "unit": "GB/s",
            "ms_per_step": round(ms, 4), "steps": reps, "bytes": n, "memo_states": r.info()["memo_states"],
            "accepted": chunked, "last_whole_sample_end": end, "mean_active_set": round(mean_active, 2),
            "sequential_gpu": {"bytes": pre, "ms": round(seq_ms, 2), "GB/s": round(pre / (seq_ms * 1e-3) / 1e9, 4)},
            "chunked_over_sequential": round((n / ms) / (pre / seq_ms), 1),
            "roofline": _roofline(n, kernel_ms, "k_chunk_stage + k_span_tasks (timed kernels of a step)", ms),
            "gpu_launches_per_step": launches / max(reps, 1),
            "cpu_baseline": {"value": cpu_v, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": cpu_desc},
            "clocks": clk}


def _serving_sweep(rx, pool, owners, datas, bufs, fresh_nodes, rates, args, payload_mode, rng):
    """One Poisson replay per arrival rate through a new server; bufs are the
    payloads as the mode takes them (device tensors for mode 1, page-locked
    host tensors for mode 2)."""
    points, compile_us, fresh_all = [], [], []
    for rate in rates:
        nreq = int(min(args.max_requests, max(200, rate * args.seconds)))
        arrive = np.cumsum(rng.exponential(1.0 / rate, nreq))
        pick = rng.integers(0, len(datas), nreq)
        reuse = rng.random(nreq) < 0.8
        handles = np.zeros(nreq, np.uint64)
        for k in range(nreq):
            if reuse[k]:
                handles[k] = pool[int(owners[int(pick[k])])].handle
            else:
                # an expression outside the pool: compiled on arrival (cost reported separately)
                t0 = time.perf_counter()
                h = rx.Regex.from_nodes(fresh_nodes[k % len(fresh_nodes)])
                compile_us.append((time.perf_counter() - t0) * 1e6)
                fresh_all.append(h)
                handles[k] = h.handle
        payloads = np.array([bufs[int(p)].data_ptr() for p in pick], np.uint64)
        lens = np.array([len(datas[int(p)]) for p in pick], np.int64)
        srv = rx.Server(max_inflight=8192, device_payload=payload_mode)
        _, late = srv.replay(handles, payloads, lens, (arrive * 1e9).astype(np.int64))
        srv.drain(600000)
        st = srv.stats()
        srv.close()
        # req/s = completed / (first submission -> last completion); the part
        # of that span after the last arrival is the drain of the requests
        # still in flight then
        span = st["completed"] / max(st["req_per_s"], 1e-9)
        window = float(arrive[-1] - arrive[0])
        points.append({"rate_target": rate, "requests": nreq, "submit_late_ms": round(late / 1e6, 3),
                       "arrival_window_s": round(window, 4), "drain_ms": round(1e3 * max(span - window, 0.0), 2),
                       "req_per_s": round(st["req_per_s"], 1), "GB/s": round(st["gb_per_s"], 2),
                       "offered_GB/s": round(rate * float(lens.mean()) / 1e9, 2),
                       "p50_ms": round(st["p50_ns"] / 1e6, 3), "p99_ms": round(st["p99_ns"] / 1e6, 3),
                       "max_ms": round(st["max_ns"] / 1e6, 3),
                       "ticks": st["ticks"], "peak_inflight": st["peak_inflight"],
                       "mean_bytes": int(lens.mean())})
    for h in fresh_all:
        h.free()
    return points, compile_us


def cfg_serving_result(args, dev):
    """Config 5: Poisson arrivals of (regex, string) requests over a pool of
    2000 compiled expressions (80% reuse; 20% compiled on arrival), swept
    over arrival rates, with payloads resident on the device and with
    payloads in page-locked host memory (read by the server when it admits a
    request, payload mode 2); p50/p99 latency and throughput, against the
    plain per-request form."""
    import torch
    import oracle
    import paper_1108_3126_b300 as rx
    import synth
    pool_nodes = synth.serving_pool(pool=args.pool)
    pool = [rx.Regex.from_nodes(nd) for nd in pool_nodes]
    rng = np.random.default_rng(0x5EED0005)
    # payloads: log-uniform 16 B - 16 MiB, half from a pool expression's language
    npay = args.payloads
    lens = np.exp(rng.uniform(np.log(16), np.log(16 << 20), npay)).astype(np.int64)
    owners = rng.integers(0, len(pool), npay)
    datas = []
    for k in range(npay):
        s = synth.gen_strings(pool_nodes[owners[k]], 1, int(lens[k]), int(lens[k]), synth.ALL_BYTES,
                              synth.item_seed(0x5EED0005, 10 + k), p_lang=0.5)
        datas.append(np.ascontiguousarray(s.data))
    dbufs = [torch.from_numpy(np.concatenate([x, np.zeros(16, np.uint8)])).to(dev) for x in datas]
    hbufs = [torch.from_numpy(x).pin_memory() for x in datas]
    torch.cuda.synchronize(dev)
    fresh_nodes = [synth.gen_regex(int(np.exp(rng.uniform(np.log(8), np.log(1025)))), 14, synth.ALL_BYTES,
                                   synth.item_seed(0x5EED0005, 100000 + k)) for k in range(4096)]
    clocks = Clocks(dev.index)
    clocks.start()
    dev_points, compile_us = _serving_sweep(rx, pool, owners, datas, dbufs, fresh_nodes, args.rates, args, 1,
                                            np.random.default_rng(0x5EED0015))
    host_points, _ = _serving_sweep(rx, pool, owners, datas, hbufs, fresh_nodes, args.rates, args, 2,
                                    np.random.default_rng(0x5EED0015))
    # plain per-request form: one synchronous call per request
    out = torch.zeros(1, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    lat = []
    nb = 0
    prng = np.random.default_rng(0x5EED0025)
    t0 = time.perf_counter()
    for k in range(args.plain_requests):
        p = int(prng.integers(0, npay))
        ts = time.perf_counter()
        if len(datas[p]) > (1 << 20):
            rx.match_long(pool[int(owners[p])], dbufs[p], len(datas[p]), out, stream=stream)
        else:
            rx.match_seq(pool[int(owners[p])], dbufs[p], len(datas[p]), out, stream=stream)
        torch.cuda.synchronize(dev)
        lat.append(time.perf_counter() - ts)
        nb += len(datas[p])
    el = time.perf_counter() - t0
    clk = clocks.stop()
    # the host-to-device link (a 256 MiB page-locked copy), the ceiling of
    # the host-payload mode's input rate
    hp = torch.empty(256 << 20, dtype=torch.uint8).pin_memory()
    dp = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    dp.copy_(hp, non_blocking=True)
    link_ms = _time(lambda: dp.copy_(hp, non_blocking=True), 5, stream, dev)
    link_gbs = (256 << 20) / (link_ms * 1e-3) / 1e9
    del hp, dp
    # the oracle on the host cores: O2 on random requests' (expression, payload)
    cores = len(os.sched_getaffinity(0))
    order = np.random.default_rng(0x5EED0035).permutation(npay)

    def o2_req(kk):
        kk = min(kk, npay)
        idx = order[:kk]
        sub = synth.pack([datas[int(i)].tobytes() for i in idx])
        oracle.o2_pairs([pool_nodes[int(owners[int(i)])] for i in idx], np.arange(kk, dtype=np.int32), sub.data,
                        sub.offsets, threads=cores)
        mb = int(sub.offsets[-1]) / 1e6
        return int(sub.offsets[-1]), f"{kk} random payloads with their expressions ({mb:.1f} MB), O2 on {cores} " \
                                     "threads", kk >= npay

    cpu_v, cpu_desc = _cpu_o2(o2_req, args.cpu_seconds, 16) if not args.no_cpu_baseline else (None, "skipped")
    best = max(dev_points, key=lambda q: q["req_per_s"])
    best_h = max(host_points, key=lambda q: q["req_per_s"])
    plain_rps = args.plain_requests / el
    for h in pool:
        h.free()
    return {"workload": f"serving: Poisson arrivals, pool of {len(pool)} regexes 8-1024 nodes, 80% reuse, "
                        f"payloads log-uniform 16 B-16 MiB ({npay} payloads)",
            "value": best["GB/s"], "unit": "GB/s", "req_per_s": best["req_per_s"],
            "sweep_device_payloads": dev_points, "sweep_host_payloads": host_points,
            "host_link_GB/s": round(link_gbs, 1),
            "link_note": "host payloads (mode 2, page-locked, borrowed until polled): every payload crosses the "
                         "host link once, so the offered input exceeds the link above about link / mean bytes "
                         "requests per second",
            "plain_per_request": {"requests": args.plain_requests, "req_per_s": round(plain_rps, 1),
                                  "GB/s": round(nb / el / 1e9, 3),
                                  "p50_ms": round(1e3 * float(np.median(lat)), 3),
                                  "p99_ms": round(1e3 * float(np.quantile(lat, 0.99)), 3)},
            "served_over_plain_req_per_s": round(best["req_per_s"] / plain_rps, 1),
            "served_host_over_plain_req_per_s": round(best_h["req_per_s"] / plain_rps, 1),
            "compile_on_miss_us_mean": round(float(np.mean(compile_us)), 1) if compile_us else None,
            "cpu_baseline": {"value": cpu_v, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": cpu_desc},
            "clocks": clk}


CONFIG_RESULTS = {"small": cfg_small_result, "batched": cfg_batched_result, "long": cfg_long_result,
                  "serving": cfg_serving_result}


def run_config(args, world, rank, local):
    """One of the other configs alone: its own JSON line."""
    dev = _dev_setup(local)
    r = CONFIG_RESULTS[args.workload](args, dev)
    line = {"metric": METRIC, "n_gpus": world, "higher_is_better": True, "dtype": "u8", "data": "synthetic",
            "scaling": "weak", "vs_baseline": None, "config": {"workload": r.pop("workload")}}
    line.update(r)
    if rank == 0:
        print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="streaming", choices=["streaming", "small", "batched", "long", "serving"])
    ap.add_argument("--regexes", type=int, default=10000, help="batched: number of expressions")
    ap.add_argument("--long-bytes", type=int, default=1 << 30, help="long: text length")
    ap.add_argument("--seq-bytes", type=int, default=64 << 20, help="long: prefix timed sequentially")
    ap.add_argument("--pool", type=int, default=2000, help="serving: compiled expressions")
    ap.add_argument("--payloads", type=int, default=768, help="serving: payloads (device and host copies)")
    ap.add_argument("--rates", type=float, nargs="+", default=[1000, 3000, 10000, 30000, 100000, 200000])
    ap.add_argument("--seconds", type=float, default=0.5, help="serving: arrival window per rate")
    ap.add_argument("--max-requests", type=int, default=60000)
    ap.add_argument("--plain-requests", type=int, default=300)
    ap.add_argument("--paper-strings", type=int, default=48, help="small: strings timed on Section 8's machine")
    ap.add_argument("--cpu-seconds", type=float, default=8.0, help="CPU-baseline budget per config")
    ap.add_argument("--min-seconds", type=float, default=0.3,
                    help="timed loops of the other configs last about this long (0: three repetitions)")
    ap.add_argument("--variant", default="auto", choices=["auto", "memo", "thread", "sparse", "warp"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="batched: skip the launch-shape autotuner")
    ap.add_argument("--long-pair-bytes", type=int, default=0,
                    help="batched: fix the long-pair threshold (with --batch-block) instead of autotuning")
    ap.add_argument("--batch-block", type=int, default=256, help="batched: threads per block with --long-pair-bytes")
    ap.add_argument("--no-extra", action="store_true",
                    help="streaming: skip the other four configs (run by default at N=1)")
    ap.add_argument("--strings", type=int, default=1 << 20, help="batch size (default: the full workload)")
    ap.add_argument("--quick", action="store_true",
                    help="skip the variant sweep, e2e repeats, CPU baseline and the other configs")
    ap.add_argument("--autotune", action="store_true", help="run the autotuner on the batch before timing")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    MIN_SECONDS[0] = args.min_seconds
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    try:
        if args.workload == "streaming":
            run_streaming(args, world, rank, local)
        else:
            run_config(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
