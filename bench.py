"""Benchmark: exact edit distance (Landau-Vishkin BFS) on one GB300.

Headline (one "step"): the n = 10^9 pair (256 symbols with Zipf(1.1)
frequencies, 10^4 edits planted in geometric bursts), solved by one
persistent launch of the single-pair kernel with the strings resident in
HBM.  Metric: diagonal-extensions per second (one extension = one (round,
diagonal) cell of Algorithm 1), with compared string bytes per second
against the measured HBM bandwidth as the roofline.

Extra keys of the same line (skipped with --quick): every other workload
of the suite, each measured once after the timed region -- n = 10^6 (100
edits), the three n = 10^8 pairs (k = 10, 10^3, 10^5), 4096 uneven pairs in
one batched launch against one pair at a time, and 512 served pairs
(Poisson arrivals, continuous batching: p50/p99 latency and capacity).

--workload small|mid|large|batch|serve|lcplen times one workload alone.

--impl reference times the CPU oracle (test infrastructure, plain C) on the
host on the same sample as the line's cpu_baseline; there is no other
reference implementation of this method to install.

Multi-GPU: a single pair does not shard (every round needs its neighbours'
values), so --gpus N runs N replicas (one process per GPU under torchrun);
value = units processed by all ranks / max time over ranks.  Batched pairs
are sharded over ranks by estimated cost (longest processing time first).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FALLBACK_HBM = 6800.0


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ------------------------------------------------------------------ env
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Dist:
    def __init__(self):
        self.ws, self.rank, self.local = dist_env()
        self.pg = None
        if self.ws > 1:
            import torch.distributed as td

            td.init_process_group("gloo")
            self.pg = td

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, v: float) -> float:
        if not self.pg:
            return v
        import torch

        t = torch.tensor([v], dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, v: float) -> float:
        if not self.pg:
            return v
        import torch

        t = torch.tensor([v], dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM, "fallback"


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons during the timed region:
    the sampler (every 25 ms) is running before start() returns, and stop()
    keeps the samples taken between the two calls."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.th = None
        self.t_begin = 0.0

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "25"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()
        t0 = time.monotonic()
        while not self.lines and time.monotonic() - t0 < 5.0 and self.proc.poll() is None:
            time.sleep(0.005)
        self.t_begin = time.monotonic()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        t_end = time.monotonic()
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.th:
            self.th.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        inside = [ln for t, ln in self.lines if self.t_begin <= t <= t_end + 0.03]
        if not inside:  # a region shorter than one period: the first sample after it began
            inside = [ln for t, ln in self.lines if t >= self.t_begin][:1]
        for ln in inside:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


TUNE_TABLE = os.path.join(ROOT, "paper_2306_17461_gb300", "tune_table.tsv")

# the translation unit of lv_tiles_kernel: the sources its counters depend on
TILE_KERNEL_SOURCES = ("ed_device.cuh", "lv_kernels.cuh", "lv_round.cuh", "lv_tiles.cu")


def src_hash() -> str:
    h = hashlib.sha256()
    cs = os.path.join(ROOT, "paper_2306_17461_gb300", "csrc")
    for f in TILE_KERNEL_SOURCES:
        with open(os.path.join(cs, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profile_traffic(name: str):
    """dram bytes per launch from a committed ncu summary, if it was taken on
    the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(p):
        return None
    src, traffic = None, None
    with open(p) as f:
        for line in f:
            if line.startswith("source_hash:"):
                src = line.split(":", 1)[1].strip()
            if line.startswith("traffic_bytes_per_launch:"):
                traffic = float(line.split(":", 1)[1].strip())
    if src != src_hash():
        return None
    return traffic


# ------------------------------------------------------------------ workloads
DEFAULT_KS = "10,1000,100000"

# What bounds each single-pair workload (from the kernel's phase timers and
# ncu counters): the k sequential rounds, each waiting on the alignment
# path's slide, unless the slides stream whole strings.
REGIME = {
    "small": "round latency (n = 1e6 fits in L2; 1e2 rounds)",
    "mid_k10": "HBM streaming: ten slides of about 1e7 bytes each",
    "mid_k1000": "round chain: every round waits on the path's slide of about 1e5 bytes",
    "mid_k100000": "scattered start-row loads of 2e5 diagonals a round (L1 throughput)",
    "large": "round chain: 1e4 sequential rounds, a slide of about 2e6 bytes after each burst",
}


def make_workload(name: str, args):
    from paper_2306_17461_gb300 import workloads as W

    if name == "mid":
        ks = [int(x) for x in args.ks.split(",")]
        pairs = [W.single_mid(k, n=args.n or 10**8) for k in ks]
        desc = f"single pair, n={args.n or 10**8} sigma=4 uniform, planted k in {ks}, one launch per pair"
        tags = [f"mid_k{k}" for k in ks]
    elif name == "small":
        pairs = [W.single_small(n=args.n or 10**6)]
        desc = f"single pair, n={args.n or 10**6} sigma=4 uniform, 100 planted edits"
        tags = ["small"]
    elif name == "large":
        pairs = [W.single_large(n=args.n or 10**9)]
        desc = (f"single pair, n={args.n or 10**9} Zipf(1.1) over 256 symbols, 1e4 edits in geometric bursts "
                "(mean 20 edits, mean gap 4)")
        tags = ["large"]
    elif name == "lcplen":
        ks = [int(x) for x in (args.ks if args.ks != DEFAULT_KS else "10000,50000").split(",")]
        skews = [float(x) for x in args.skews.split(",")]
        pairs = [W.lcp_length_pair(k, p0, n=args.n or 10**7) for k in ks for p0 in skews]
        desc = (f"Fig. 4 setting: n={args.n or 10**7}, two symbols with P(0) in {skews}, "
                f"planted k in {ks}, one launch per pair")
        tags = [f"lcplen_k{k}_p{p0}" for k in ks for p0 in skews]
    else:
        raise ValueError(name)
    return pairs, desc, tags


def lpt_shard(costs, ws: int):
    """Pairs split over ws ranks by longest processing time first: each pair,
    costliest first, goes to the rank with the least cost so far.  Returns
    one sorted index list per rank."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * ws
    out = [[] for _ in range(ws)]
    for i in order:
        r = min(range(ws), key=lambda j: (load[j], j))
        out[r].append(i)
        load[r] += costs[i]
    return [sorted(x) for x in out]


def pair_record(pair, k, st, ms, peak):
    """Per-pair figures of one timed run of the single-pair kernel."""
    cb = st["compared_bytes"]
    gbs = cb / (ms / 1e3) / 1e9 if ms else 0.0
    return {"k": k, "planted": pair.edits, "n": int(pair.A.size), "m": int(pair.B.size), "ms": round(ms, 4),
            "ns_per_round": round(ms * 1e6 / max(1, k), 1), "ext": st["extensions"],
            "ext_per_s": st["extensions"] / (ms / 1e3) if ms else None, "compared_bytes": cb,
            "gbs": round(gbs, 2), "frac": gbs / peak, "long_slides": st["long_slides"],
            "open_slides": st["open_slides"], "phase_ms": [round(x, 3) for x in st["phase_ms"]],
            "build_ms": round(st["build_ms"], 4), "hash_queries": st["hash_queries"],
            "avg_lcp": st["slide_chars"] / max(1, st["extensions"])}


# ------------------------------------------------------------------ GPU arm
def time_pairs(ed, ctxs, dA, dB, stream, steps, warmup, flush=None):
    """Runs every pair once per step through ed_distance_dev (pair i on
    context ctxs[i]); returns the CUDA-event time of each step (ms) and each
    pair's (k, stats, kernel ms) of the timed steps."""
    import torch

    for _ in range(warmup):
        for i in range(len(dA)):
            ed.ed_distance_dev(ctxs[i].h, dA[i], dB[i], stream)
    torch.cuda.synchronize()
    evs, recs = [], []
    for s in range(steps):
        if flush is not None:
            flush.fill_(s & 255)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(len(dA)):
            k = ed.ed_distance_dev(ctxs[i].h, dA[i], dB[i], stream)
            recs.append((i, k, ed.ed_last_stats(ctxs[i].h)))
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    return [e0.elapsed_time(e1) for e0, e1 in evs], recs


def pair_contexts(ed, args, D, pairs, lcp_mode=None):
    """One context per pair: with the tuning table, each pair's launch
    parameters come from its row (the expected distance given as the
    pair's planted edit count, as a caller that knows its data would)."""
    tune = 1 if (args.tune and os.path.exists(TUNE_TABLE)) else 0
    extra = {}
    if lcp_mode is not None:
        extra["lcp_mode"] = lcp_mode
    return [ed.Context(device=D.local, block_rounds=args.block_rounds, hash_block=args.hash_block, tune=tune,
                       distance_hint=int(p.edits) if tune else 0, **extra) for p in pairs], tune


def summarize(pairs, tags, recs, peak):
    per = {}
    for i, pair in enumerate(pairs):
        mine = [r for r in recs if r[0] == i]
        ms = statistics.median(r[2]["kernel_ms"] for r in mine)
        per[tags[i]] = pair_record(pair, mine[0][1], mine[0][2], ms, peak)
        per[tags[i]]["regime"] = REGIME.get(tags[i], "")
    return per


def run_single(args, D: Dist):
    import torch

    from paper_2306_17461_gb300 import binding as ed

    torch.cuda.set_device(D.local)
    dev = torch.device("cuda", D.local)
    pairs, desc, tags = make_workload(args.workload, args)
    lcp_mode = {"auto": None, "direct": ed.ED_LCP_DIRECT, "hash": ed.ED_LCP_HASH, "bhash": ed.ED_LCP_BHASH}[args.lcp]
    ctxs, tuned = pair_contexts(ed, args, D, pairs, lcp_mode)
    dA = [torch.from_numpy(p.A).to(dev) for p in pairs]
    dB = [torch.from_numpy(p.B).to(dev) for p in pairs]
    stream = torch.cuda.current_stream()
    # inputs smaller than L2 (129 MB): flush it between timed steps by
    # writing 256 MB, outside the steps' events
    in_bytes = sum(int(p.A.size + p.B.size) for p in pairs)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev) if in_bytes < (256 << 20) else None
    l2_note = ("flushed between steps (256 MB written outside the timed events)" if flush is not None
               else "no flush: the strings exceed the 129 MB L2")
    torch.cuda.synchronize()
    D.barrier()
    clocks = Clocks(D.local)
    clocks.start()
    step_ms, recs = time_pairs(ed, ctxs, dA, dB, stream, args.steps, args.warmup, flush)
    D.barrier()
    clk = clocks.stop()
    ms = sum(step_ms)
    ext = sum(r[2]["extensions"] for r in recs)
    cbytes = sum(r[2]["compared_bytes"] for r in recs)
    kms = sum(r[2]["kernel_ms"] for r in recs)
    launches = sum(r[2]["kernel_launches"] for r in recs)
    peak, peak_src = peaks()
    per = summarize(pairs, tags, recs, peak)
    # e2e: host buffers through ed_distance (H2D inside the timed region)
    hA = [torch.from_numpy(p.A).pin_memory() for p in pairs]
    hB = [torch.from_numpy(p.B).pin_memory() for p in pairs]
    for i in range(len(pairs)):
        ed.ed_distance(ctxs[i].h, hA[i], hB[i])
    torch.cuda.synchronize()
    D.barrier()
    t0 = time.perf_counter()
    e_ext = 0
    for _ in range(args.steps):
        for i in range(len(pairs)):
            ed.ed_distance(ctxs[i].h, hA[i], hB[i])
            e_ext += ed.ed_last_stats(ctxs[i].h)["extensions"]
    e2e_s = D.max(time.perf_counter() - t0)
    h2d = sum(int(p.A.size + p.B.size) for p in pairs)
    for c in ctxs:
        c.close()
    secs = D.max(ms / 1e3)
    ext_all = D.sum(ext)
    achieved = (cbytes / (kms / 1e3)) / 1e9 if kms else 0.0
    head = per[tags[0]] if len(tags) == 1 else None
    res = {
        "metric": "diagonal-extensions/s",
        "value": ext_all / secs,
        "unit": "ext/s",
        "n_gpus": D.ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": desc, "lcp": args.lcp, "pairs_per_step": len(pairs), "l2": l2_note,
                   "parallelism": f"replicas x{D.ws}",
                   "launch": "tuning table, distance hint = planted edits" if tuned else "built-in defaults"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
                     "kernel": "lv_tiles_kernel",
                     "traffic": profile_traffic(f"lv_tiles_{args.workload}.md")
                     if args.lcp in ("auto", "direct") and args.ks == DEFAULT_KS and not args.n else None,
                     "algorithmic_bytes_per_launch": cbytes / max(1, len(recs)),
                     "ns_per_round": head["ns_per_round"] if head else None,
                     "limiter": head["regime"] if head else "see per_pair"},
        "e2e": {"value": D.sum(e_ext) / e2e_s, "unit": "ext/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": 8 * len(pairs)},
        "gpu_launches": int(launches),
        "clocks": clk,
        "per_pair": per,
    }
    return res, pairs


def run_single_extra(args, D: Dist, name: str, reps: int = 3):
    """One single-pair workload measured after the headline (median of reps
    kernel times per pair)."""
    import torch

    from paper_2306_17461_gb300 import binding as ed

    dev = torch.device("cuda", D.local)
    sub = argparse.Namespace(**vars(args))
    sub.n = 0
    sub.ks = DEFAULT_KS
    pairs, desc, tags = make_workload(name, sub)
    ctxs, _ = pair_contexts(ed, args, D, pairs)
    dA = [torch.from_numpy(p.A).to(dev) for p in pairs]
    dB = [torch.from_numpy(p.B).to(dev) for p in pairs]
    in_bytes = sum(int(p.A.size + p.B.size) for p in pairs)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev) if in_bytes < (256 << 20) else None
    _, recs = time_pairs(ed, ctxs, dA, dB, torch.cuda.current_stream(), reps, 1, flush)
    for c in ctxs:
        c.close()
    peak, _ = peaks()
    out = summarize(pairs, tags, recs, peak)
    del dA, dB, flush
    torch.cuda.empty_cache()
    return out


def batch_workload(npairs: int, rank: int, ws: int):
    from paper_2306_17461_gb300 import workloads as W

    ns, ks, sig = W.batch_shapes(npairs)
    costs = [float(ns[p]) + float(ks[p]) ** 2 for p in range(npairs)]
    mine = lpt_shard(costs, ws)[rank]
    pairs = [W.make_pair(4, int(ns[p]), int(ks[p]), sigma=int(sig[p]), extra=p + 1) for p in mine]
    return mine, pairs


def run_batch(args, D: Dist):
    import torch

    from paper_2306_17461_gb300 import binding as ed

    torch.cuda.set_device(D.local)
    dev = torch.device("cuda", D.local)
    npairs = args.npairs
    mine, pairs = batch_workload(npairs, D.rank, D.ws)
    ctx = ed.Context(device=D.local)
    dA = [torch.from_numpy(p.A).to(dev) for p in pairs]
    dB = [torch.from_numpy(p.B).to(dev) for p in pairs]
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        ed.ed_distance_batch_dev(ctx.h, dA, dB)
    D.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(D.local)
    clocks.start()
    # the batch call runs on the legacy default stream, which torch's
    # default stream is: events there bracket the device work
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    ext = launches = 0
    batch_ms = tile_ms = 0.0
    for _ in range(args.steps):
        ed.ed_distance_batch_dev(ctx.h, dA, dB)
        st = ed.ed_last_stats(ctx.h)
        ext += st["extensions"]
        launches += st["kernel_launches"]
        batch_ms += st["phase_ms"][5]
        tile_ms += st["kernel_ms"] - st["phase_ms"][5]
    ev1.record()
    torch.cuda.synchronize()
    secs = D.max(ev0.elapsed_time(ev1) / 1e3)
    clk = clocks.stop()
    # one-pair-at-a-time baseline on the same pairs (single-pair kernel)
    ev2 = torch.cuda.Event(enable_timing=True)
    ev3 = torch.cuda.Event(enable_timing=True)
    ev2.record()
    for i in range(len(pairs)):
        ed.ed_distance_dev(ctx.h, dA[i], dB[i], torch.cuda.default_stream())
    ev3.record()
    torch.cuda.synchronize()
    one_s = D.max(ev2.elapsed_time(ev3) / 1e3)
    ctx.close()
    total_pairs = npairs * args.steps
    res = {
        "metric": "batched pairs/s",
        "value": total_pairs / secs,
        "unit": "pairs/s",
        "n_gpus": D.ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": secs * 1e3 / args.steps,
        "higher_is_better": True,
        "scaling": "strong",
        "vs_baseline": None,
        "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": f"{npairs} pairs, n log-uniform [1e3,1e6], sigma 4/64, edit rate log-uniform [1e-4,5e-2]",
                   "parallelism": f"pairs sharded over {D.ws} GPUs by estimated cost (LPT)",
                   "l2": "no flush: the pairs' strings (about 1.2 GB) exceed the 129 MB L2"},
        "ext_per_s": D.sum(ext) / secs,
        "batch_kernel_ms_per_step": batch_ms / args.steps,
        "tile_kernel_ms_per_step": tile_ms / args.steps,
        "one_at_a_time_pairs_per_s": D.sum(len(pairs)) / one_s,
        "speedup_vs_one_at_a_time": (total_pairs / secs) / (D.sum(len(pairs)) / one_s),
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    return res, None


def serve_run(ed, ctx, pairs, arrivals):
    """Submits pairs at the given arrival times (seconds; None = all at once)
    and polls them to completion.  Returns (latencies in s, span in s, ks)."""
    lat = [None] * len(pairs)
    ks = [None] * len(pairs)
    tickets = {}
    t0 = time.perf_counter()
    i = 0
    while i < len(pairs) or tickets:
        now = time.perf_counter() - t0
        while i < len(pairs) and (arrivals is None or arrivals[i] <= now):
            try:
                tickets[ed.ed_submit(ctx.h, pairs[i].A, pairs[i].B)] = i
                i += 1
            except ed.EdError as e:
                if e.code != ed.ED_EBUSY:
                    raise
                break
        for t in list(tickets):
            st, k = ed.ed_poll(ctx.h, t)
            if st == ed.ED_OK:
                j = tickets.pop(t)
                ks[j] = k
                lat[j] = (time.perf_counter() - t0) - (arrivals[j] if arrivals is not None else 0.0)
        time.sleep(0.0002)
    return lat, time.perf_counter() - t0, ks


def run_serve(args, D: Dist):
    import torch

    from paper_2306_17461_gb300 import binding as ed
    from paper_2306_17461_gb300 import workloads as W

    torch.cuda.set_device(D.local)
    pairs = W.serve_pairs(args.npairs_serve)
    rates = [float(r) for r in args.rates.split(",")]
    ctx = ed.Context(device=D.local, max_inflight=1024)
    serve_run(ed, ctx, pairs[:8], None)  # warm-up
    out = []
    for ri, rate in enumerate(rates):
        lat, span, _ = serve_run(ed, ctx, pairs, W.poisson_arrivals(rate, len(pairs), seed_extra=ri))
        L = np.array(lat) * 1e3
        out.append({"rate_req_s": rate, "pairs_per_s": len(pairs) / span,
                    "p50_ms": float(np.percentile(L, 50)), "p99_ms": float(np.percentile(L, 99)),
                    "span_s": span})
        log(f"serve rate {rate}: {out[-1]}")
    # capacity: every request submitted at once, served concurrently
    lat, span, _ = serve_run(ed, ctx, pairs, None)
    capacity = len(pairs) / span
    cnt = ed.ed_serve_counters(ctx.h)
    ctx.close()
    # the same pairs one at a time through the synchronous call (host strings)
    one = ed.Context(device=D.local)
    t0 = time.perf_counter()
    for p in pairs:
        ed.ed_distance(one.h, p.A, p.B)
    one_rate = len(pairs) / (time.perf_counter() - t0)
    one.close()
    log(f"serve capacity {capacity:.2f} pairs/s, one at a time {one_rate:.2f} pairs/s")
    best = max(out, key=lambda r: r["pairs_per_s"])
    res = {
        "metric": "served pairs/s",
        "value": best["pairs_per_s"],
        "unit": "pairs/s",
        "n_gpus": D.ws,
        "steps": len(rates),
        "warmup": 8,
        "ms_per_step": best["span_s"] * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": f"{len(pairs)} pairs, n log-uniform [1e2,1e7], edit rate log-uniform [1e-3,1e-1], Poisson arrivals",
                   "rates": rates},
        "sweep": out,
        "p50_ms": best["p50_ms"],
        "p99_ms": best["p99_ms"],
        "capacity_pairs_per_s": capacity,
        "one_at_a_time_pairs_per_s": one_rate,
        "speedup_vs_one_at_a_time": capacity / one_rate,
        "engine_steps": cnt["steps"],
        "tile_slices": cnt["slices"],
    }
    return res, None


def extras(args, D: Dist):
    """Every other workload of the suite, measured once after the headline."""
    out = {}
    for name in ("small", "mid"):
        t0 = time.perf_counter()
        out.update(run_single_extra(args, D, name))
        log(f"extra {name}: {time.perf_counter() - t0:.1f} s")
    sub = argparse.Namespace(**vars(args))
    sub.steps, sub.warmup = 2, 1
    t0 = time.perf_counter()
    b, _ = run_batch(sub, D)
    out["batch"] = {k: b[k] for k in ("value", "unit", "ms_per_step", "ext_per_s", "batch_kernel_ms_per_step",
                                      "tile_kernel_ms_per_step", "one_at_a_time_pairs_per_s",
                                      "speedup_vs_one_at_a_time", "gpu_launches", "clocks")}
    out["batch"]["workload"] = b["config"]["workload"]
    log(f"extra batch: {time.perf_counter() - t0:.1f} s")
    t0 = time.perf_counter()
    s, _ = run_serve(sub, D)
    out["serve"] = {k: s[k] for k in ("p50_ms", "p99_ms", "sweep", "capacity_pairs_per_s",
                                      "one_at_a_time_pairs_per_s", "speedup_vs_one_at_a_time",
                                      "engine_steps", "tile_slices")}
    out["serve"]["served_pairs_per_s"] = s["value"]
    out["serve"]["workload"] = s["config"]["workload"]
    log(f"extra serve: {time.perf_counter() - t0:.1f} s")
    return out


# ------------------------------------------------------------------ CPU (oracle)
def cpu_sample(pairs, budget_s: float, threads: int = 1):
    """The oracle (Algorithm 1, char-by-char LCP; with threads > 1 the
    diagonals of a round in parallel) on the host, on a bounded sample of
    the workload: each pair runs whole if it fits its share of the budget,
    else for a number of rounds sized to it.  Returns (ext/s, threads,
    description, seconds)."""
    import oracle

    ext_total, t_total, parts = 0, 0.0, []
    share = budget_s / max(1, len(pairs))
    for p in pairs:
        rounds = 64
        while True:
            t0 = time.perf_counter()
            k, r, ext = oracle.lv(p.A, p.B, max_rounds=rounds, nthreads=threads, with_stats=True)
            dt = time.perf_counter() - t0
            if k >= 0 or dt > share / 4:
                break
            rounds *= 2
        ext_total += ext
        t_total += dt
        parts.append(f"n={p.A.size}: {r} rounds{' (whole pair)' if k >= 0 else ''}")
    return ext_total / t_total, threads, "; ".join(parts), t_total


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_baseline(pairs, budget_s: float):
    """The sequential oracle on one core (the line's value), with the
    all-core figure (OpenMP over the diagonals of a round) beside it."""
    v, cores, sample, secs = cpu_sample(pairs, budget_s, 1)
    nall = os.cpu_count() or 1
    va, _, sample_all, secs_all = cpu_sample(pairs, budget_s, nall)
    return {"value": v, "unit": "ext/s", "cores": cores, "kind": "oracle", "sample": sample, "seconds": secs,
            "cpu": cpu_model(), "all_cores": {"value": va, "cores": nall, "sample": sample_all,
                                              "seconds": secs_all}}


def run_reference(args, D: Dist):
    if D.rank != 0:
        return None
    name = args.workload if args.workload in ("mid", "small", "large") else "large"
    pairs, desc, _ = make_workload(name, args)
    # each step: the sample the GPU line's cpu_baseline times (the oracle on
    # one core, each pair whole when it fits the budget)
    vals = []
    for _ in range(args.warmup):
        cpu_sample(pairs, args.cpu_budget, 1)
    t0 = time.perf_counter()
    sample = ""
    for _ in range(args.steps):
        v, cores, sample, _ = cpu_sample(pairs, args.cpu_budget, 1)
        vals.append(v)
    span = time.perf_counter() - t0
    v = statistics.median(vals)
    return {
        "metric": "diagonal-extensions/s",
        "value": v,
        "unit": "ext/s",
        "n_gpus": D.ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": span * 1e3 / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8",
        "data": "synthetic",
        "impl": "reference",
        "config": {"workload": desc, "lcp": "direct (char by char)"},
        "cpu_baseline": {"value": v, "unit": "ext/s", "cores": 1, "kind": "oracle",
                         "sample": sample, "cpu": cpu_model()},
        "e2e": {"value": v, "unit": "ext/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="large", choices=["mid", "small", "large", "batch", "serve", "lcplen"])
    ap.add_argument("--lcp", default="auto", choices=["auto", "direct", "hash", "bhash"],
                    help="auto: the tuning table's choice (direct without a table)")
    ap.add_argument("--no-tune", dest="tune", action="store_false",
                    help="built-in launch parameters instead of the tuning table")
    ap.add_argument("--hash-block", type=int, default=0, help="block size b of --lcp bhash (0: 32)")
    ap.add_argument("--ks", default=DEFAULT_KS)
    ap.add_argument("--skews", default="0.5,0.9,0.99,0.999,0.9999")
    ap.add_argument("--block-rounds", type=int, default=0, help="rounds per temporal block (0: 32)")
    ap.add_argument("--n", type=int, default=0)
    ap.add_argument("--npairs", type=int, default=4096)
    ap.add_argument("--npairs-serve", type=int, default=512)
    ap.add_argument("--rates", default="8")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="the headline workload only (no extra keys)")
    args = ap.parse_args()
    D = Dist()
    try:
        if args.impl == "reference":
            res = run_reference(args, D)
            if res is not None:
                print(json.dumps(res), flush=True)
            return
        if args.workload == "batch":
            res, pairs = run_batch(args, D)
        elif args.workload == "serve":
            res, pairs = run_serve(args, D)
        else:
            res, pairs = run_single(args, D)
            if D.rank == 0 and not args.no_cpu_baseline:
                res["cpu_baseline"] = cpu_baseline(pairs, args.cpu_budget)
            if args.workload == "large" and not args.quick and not args.n and D.ws == 1:
                res["configs"] = dict(res["per_pair"], **extras(args, D))
        if D.rank == 0:
            print(json.dumps(res), flush=True)
    finally:
        D.close()


if __name__ == "__main__":
    main()
