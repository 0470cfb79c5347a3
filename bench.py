#!/usr/bin/env python3
"""Throughput of AMS-sort on GB300: two-level sample sort of 2^28 uniform uint64 keys
(r1 = r2 = 256 groups, overpartitioning b = 4), keys/s, per GPU or summed over ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ams|reference]
                    [--workload two_level_u64|two_level_u64_2e26|segmented_u32|single_level_u32|serving]
                    [--no-extras]

One step sorts the whole input once (out of place, so every step sees the same
unsorted input; the 2 GiB input and output exceed the L2 cache, so no flush is
needed).  The headline is timed without per-kernel events; a second pass with
events gives the kernel shares.  Under torchrun every rank sorts its own input
(replicas, weak scaling).  On one GPU the default run appends, to the same JSON line,
every other configuration of the evaluation: `configs` (ms per sort of the
single-level 2^20 uint32 sort, the six two-level 2^28 uint64 distributions and the
two 2^27 pair sorts), `segmented` (100,000 uint32 segments, against one plain call
per segment) and `serving` (a Poisson stream of mixed requests against the server
and against one-at-a-time plain sorts replayed at the same arrival times).  Prints
one JSON line on rank 0.  `--impl reference` times the CPU oracle on a bounded
sample of the same workload instead.
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
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "keys/s & HBM-roofline frac at 2^28 u64; p50/p99 latency of mixed-size requests"
WORKLOADS = {
    "two_level_u64": dict(n=1 << 28, bits=64, kt=1, levels=2, buckets=[256, 256], b=4, a=0,
                          dist="uniform", dtype="u64",
                          desc="2-level AMS-sort, 2^28 uniform uint64 keys, r=256x256, b=4"),
    # the profiling case: same kernels and leaf sizes (about 4096 keys) at a quarter of
    # the keys, 512 MiB in and out (above L2, small enough for ncu's replay passes)
    "two_level_u64_2e26": dict(n=1 << 26, bits=64, kt=1, levels=2, buckets=[256, 64], b=4, a=0,
                               dist="uniform", dtype="u64",
                               desc="2-level AMS-sort, 2^26 uniform uint64 keys, r=256x64, b=4"),
    # batched segmented sort: 100,000 uint32 segments, log-uniform lengths rescaled to
    # ~2^28 keys in total, one launch sequence for all segments
    "segmented_u32": dict(n=1 << 28, bits=32, kt=0, levels=1, buckets=[16], b=4, a=0,
                          dist="uniform", dtype="u32", segments=100000,
                          desc="segmented sort, 100,000 uint32 segments (log-uniform lengths, ~2^28 keys)"),
    "single_level_u32": dict(n=1 << 20, bits=32, kt=0, levels=1, buckets=[256], b=1, a=16,
                             dist="uniform", dtype="u32",
                             desc="1-level sample sort, 2^20 uniform uint32 keys, 256 buckets, a=16"),
}
KIND_BYTES = {"classify": 1, "scatter": 2, "basecase": 2}  # key passes per element
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _traffic(kind):
    """DRAM bytes per launch of `kind` from the committed ncu summary, if the kernel
    source has not changed since the capture."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)[kind]
        src = os.path.join(ROOT, "paper_1410_6754_gb300", "csrc", t["source"])
        with open(src, "rb") as f:
            if hashlib.sha256(f.read()).hexdigest()[:16] != t["sha256_16"]:
                return None
        return float(t["bytes_per_launch"])
    except Exception:
        return None


class ClockSampler:
    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={CLOCK_FIELDS}", "--format=csv",
                                       "-lms", "100", "-i", str(gpu_index)],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.strip() for r in self.f.read().splitlines()[1:] if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            c = [x.strip() for x in r.split(",")]
            if len(c) < 9:
                continue
            try:
                sm.append(float(c[1].split()[0]))
                mx.append(float(c[2].split()[0]))
            except ValueError:
                continue
            for nm, v in zip(names, c[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x, dist, device):
    """The largest value of x over all ranks (x itself without a process group)."""
    if not dist:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank, seconds):
    """Whole-job rate of replicas: every rank processes units_per_rank in `seconds`
    (the slowest rank's time)."""
    return world * units_per_rank / seconds


def _dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def _gpu_index(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [x.strip() for x in vis.split(",") if x.strip()]
        if local_rank < len(ids):
            return ids[local_rank]
    return str(local_rank)


def run_reference(args, wl):
    """CPU oracle (single thread, numpy stable sort) on a bounded sample per step."""
    rank, world, _ = _dist_env()
    if rank != 0:
        return 0
    import numpy as np

    import oracle as O
    from paper_1410_6754_gb300 import inputs as I
    full = wl["n"]
    probe = I.generate(wl["dist"], 1 << 18, 0, wl["bits"])
    t0 = time.perf_counter()
    O.sort_keys(wl["kt"], probe)
    per_key = (time.perf_counter() - t0) / len(probe)
    budget = 120.0 / max(1, args.steps + args.warmup)
    # the probe's cost per key grows with log2 of the size: halve m until
    # m * per_key * log2(m) / 18 fits the per-step budget
    m = 1 << (int(min(full, max(1 << 16, budget / max(per_key, 1e-12)))).bit_length() - 1)
    while m > (1 << 16) and m * per_key * (m.bit_length() - 1) / 18.0 > budget:
        m >>= 1
    sample = I.generate(wl["dist"], m, 0, wl["bits"])
    for _ in range(args.warmup):
        O.sort_keys(wl["kt"], sample)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.sort_keys(wl["kt"], sample)
    dt = time.perf_counter() - t0
    value = args.steps * m / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "keys/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": wl["dtype"], "data": "synthetic",
        "config": {"workload": wl["desc"], "sample_keys_per_step": m},
        "cpu_baseline": {"value": value, "unit": "keys/s", "cores": 1, "kind": "oracle",
                         "sample": f"{m} keys of the same workload per step (first {m} keys of the "
                                   f"seeded input), numpy stable sort, one thread", **_cpu_info()},
        "e2e": {"value": value, "unit": "keys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _u64_order(t):
    """int64 view of unsigned keys -> int64 whose signed order is the unsigned order."""
    import torch
    return t ^ torch.tensor(-(1 << 63), dtype=torch.int64, device=t.device)


def _check_sorted(src, dst, bits, offsets=None):
    """Output sorted (inside every segment) and a permutation of the input (an
    order-independent hash, per segment when there are segments)."""
    import torch
    from paper_1410_6754_gb300.inputs import _mix_t
    if bits == 64:
        o, oi = _u64_order(dst), src
    else:
        o, oi = dst.to(torch.int64) & 0xFFFFFFFF, src.to(torch.int64) & 0xFFFFFFFF
    if offsets is None:
        return bool((o[1:] >= o[:-1]).all()) and bool(_mix_t(oi).sum() == _mix_t(o if bits != 64 else dst).sum())
    lens = offsets[1:] - offsets[:-1]
    seg = torch.repeat_interleave(torch.arange(lens.numel(), device=dst.device), lens)
    ok = bool(((o[1:] >= o[:-1]) | (seg[1:] != seg[:-1])).all())
    z = torch.zeros(lens.numel(), dtype=torch.int64, device=dst.device)
    hs = z.clone().index_add_(0, seg, _mix_t(oi))
    hd = z.clone().index_add_(0, seg, _mix_t(o if bits != 64 else dst))
    return ok and bool(torch.equal(hs, hd))


def _plain_per_segment(src, offsets, kw):
    """Keys/s of sorting every segment with its own plain call (the comparison for the
    batched segmented sort)."""
    import torch
    import paper_1410_6754_gb300 as ams
    off = offsets.cpu().tolist()
    dst = torch.empty_like(src)
    skw = {k: v for k, v in kw.items() if k != "offsets"}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(len(off) - 1):
        lo, hi = off[s], off[s + 1]
        if hi > lo:
            ams.sort_keys_into(src[lo:hi], dst[lo:hi], **skw)
    torch.cuda.synchronize()
    return (off[-1] - off[0]) / (time.perf_counter() - t0)


def _cpu_info():
    """Host cores and CPU model (for the CPU baseline line)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                k = ln.split(":")[0].strip().lower()
                if k in ("model name", "cpu model", "hardware") and ":" in ln:
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for ln in out.splitlines():
                if ln.lower().startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model or "unknown"}


def _timed(fn, reps, warm=2):
    """Median ms of fn() over `reps` runs (CUDA events on the current stream, after
    `warm` untimed runs)."""
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return statistics.median(times)


def run_configs(peak):
    """ms per sort of every configuration of the evaluation besides the headline
    (device-resident inputs, out of place, median of 5 after 2 warm-ups), each output
    checked (sorted and a permutation of its input)."""
    import numpy as np
    import torch

    import paper_1410_6754_gb300 as ams
    from paper_1410_6754_gb300 import inputs as I
    out = {}
    ctx = ams.Context()

    def keys_case(name, dist, n, bits, kt, levels, buckets, b, a):
        src = I.generate(dist, n, 0, bits, device="cuda")
        dst = torch.empty_like(src)
        kw = dict(levels=levels, buckets=buckets, seed=0, a=a, b=b, kt=kt)
        ms = _timed(lambda: ctx.sort(src, dst, **kw), 5)
        ctx.sync()
        ok = _check_sorted(src, dst, bits)
        w = bits // 8
        alg = (levels + 1) * 2 * n * w
        out[name] = {"ms": ms, "keys_per_s": n / (ms * 1e-3), "ok": ok,
                     "step_roofline_frac": alg / (ms * 1e-3) / 1e9 / peak}
        del src, dst

    def pairs_case(name, keys_np, kt, levels, buckets):
        n = len(keys_np)
        dt = torch.int64 if keys_np.dtype == np.uint64 else (torch.float32 if kt == 2 else torch.int32)
        kin = torch.from_numpy(keys_np.view(np.int64) if keys_np.dtype == np.uint64 else keys_np).cuda()
        vin = torch.arange(n, dtype=torch.int64, device="cuda")
        kout, vout = torch.empty_like(kin), torch.empty_like(vin)
        kw = dict(levels=levels, buckets=buckets, seed=0, kt=kt)
        ms = _timed(lambda: ctx.sort(kin, kout, vin, vout, **kw), 5)
        ctx.sync()
        if kt == 2:
            bits = kout.view(torch.int32).to(torch.int64) & 0xFFFFFFFF
            t = torch.where(bits >> 31 == 1, bits ^ 0xFFFFFFFF, bits | 0x80000000)
            same = torch.equal(kout.view(torch.int32), kin.view(torch.int32)[vout])
        else:
            t = _u64_order(kout)
            same = torch.equal(kout, kin[vout])
        asc = bool(((t[1:] > t[:-1]) | ((t[1:] == t[:-1]) & (vout[1:] > vout[:-1]))).all())
        w = (8 if kt == 1 else 4) + 8
        alg = (levels + 1) * 2 * n * w
        out[name] = {"ms": ms, "pairs_per_s": n / (ms * 1e-3), "ok": bool(same and asc),
                     "step_roofline_frac": alg / (ms * 1e-3) / 1e9 / peak}
        del kin, vin, kout, vout

    keys_case("single_level_u32_2e20_uniform_r256_a16", "uniform", 1 << 20, 32, 0, 1, [256], 1, 16)
    for dist in I.DISTRIBUTIONS:
        keys_case(f"two_level_u64_2e28_{dist}_r256x256_b4", dist, 1 << 28, 64, 1, 2, [256, 256], 4, 0)
    pairs_case("pairs_u64_dup1024_2e27_3lvl_r256", I.dup_keys_u64(1 << 27, 2), 1, 3, [256, 256, 256])
    pairs_case("pairs_f32_normal_zeros_2e27_3lvl_r256", I.normal_f32(1 << 27, 3), 2, 3, [256, 256, 256])
    ctx.close()
    torch.cuda.empty_cache()
    return out


def run_segmented_sub(reps=3):
    """The batched segmented sort (100,000 uint32 segments, log-uniform lengths rescaled
    to ~2^28 keys, uniform values): one segmented call against one plain call per
    segment."""
    import numpy as np
    import torch

    import paper_1410_6754_gb300 as ams
    from paper_1410_6754_gb300 import inputs as I
    wl = WORKLOADS["segmented_u32"]
    lens = I.segment_lengths(wl["segments"], wl["n"], 4, max_log2=20)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    n = int(off[-1])
    offsets = torch.from_numpy(off).cuda()
    src = I.generate("uniform", n, 0, 32, device="cuda")
    dst = torch.empty_like(src)
    ctx = ams.Context()
    kw = dict(levels=wl["levels"], buckets=wl["buckets"], seed=0, b=wl["b"], kt=0, offsets=offsets)
    ms = _timed(lambda: ctx.sort(src, dst, **kw), reps)
    ctx.sync()
    ok = _check_sorted(src, dst, 32, offsets)
    plain = _plain_per_segment(src, offsets, kw)
    ctx.close()
    del src, dst
    torch.cuda.empty_cache()
    return {"segments": wl["segments"], "keys": n, "ms": ms, "keys_per_s": n / (ms * 1e-3),
            "plain_per_segment_keys_per_s": plain, "ok": ok,
            "plan": f"levels {wl['levels']}, r {wl['buckets']}, b {wl['b']}; segments <= C go to the base case"}


def run_rlm_sub(peak, reps=3):
    """RLM-sort (Section 5) of the same 2^28 uniform uint64 keys: tiles of 8192 keys,
    three levels of 16, 32 and 64 parts (the last level's parts are single tiles; of
    the splits measured, three levels beat two because the first level's selections
    run over all 32,768 tiles), out of place, output checked.  Algorithmic bytes:
    (levels x 2 + 1) passes of read + write (the tile sorts of every level and every
    delivery)."""
    import torch

    import paper_1410_6754_gb300 as ams
    from paper_1410_6754_gb300 import inputs as I
    n, run, parts = 1 << 28, 8192, [16, 32, 64]
    src = I.generate("uniform", n, 0, 64, device="cuda")
    dst = torch.empty_like(src)
    ctx = ams.Context()
    ms = _timed(lambda: ams.rlm_sort(src, dst, run=run, parts=parts, seed=0, kt=1, ctx=ctx), reps)
    ctx.sync()
    ok = _check_sorted(src, dst, 64)
    ctx.close()
    del src, dst
    torch.cuda.empty_cache()
    alg = (2 * len(parts) + 1) * 2 * n * 8
    return {"n": n, "run": run, "parts": parts, "ms": ms, "keys_per_s": n / (ms * 1e-3), "ok": ok,
            "step_roofline_frac": alg / (ms * 1e-3) / 1e9 / peak,
            "definition": "(2 x levels + 1) x (read + write) x n x key bytes"}


def serving_bench(n_requests, streams, tuned, seed=5):
    """Serving loop: a seeded Poisson stream of mixed requests (sizes log-uniform in
    [2^10, 2^26]; key types 50% uint32 / 30% uint64 / 20% float32; uniform or Zipf
    values, float32 normal) run (a) one at a time, in arrival order, on one stream --
    each request starts when it has arrived and the previous one has finished -- and
    (b) through the server (continuous batching over worker streams, 64 GB budget), at
    the same arrival times.  The arrival rate is 1.1x the one-at-a-time capacity
    measured on the same requests back to back.  Latency = completion - arrival (host
    steady clock).  Both runs write separate outputs, which must be equal, sorted and
    permutations of their inputs."""
    import threading

    import numpy as np
    import torch

    import paper_1410_6754_gb300 as ams
    from paper_1410_6754_gb300 import inputs as I

    N = n_requests
    rng = np.random.default_rng(seed)
    sizes = np.floor(2.0 ** rng.uniform(10, 26, N)).astype(np.int64)
    u = rng.random(N)
    kts = np.where(u < 0.5, 0, np.where(u < 0.8, 1, 2))
    zipf = rng.random(N) < 0.5
    pools, outs_one, outs_srv, offs, views = {}, {}, {}, {}, []
    for kt in (0, 1, 2):
        idx = np.nonzero(kts == kt)[0]
        tot = int(sizes[idx].sum())
        bits = 64 if kt == 1 else 32
        if kt == 2:
            base = torch.from_numpy(I.normal_f32(min(tot, 1 << 24), 5).view(np.int32)).cuda()
            reps = -(-tot // base.numel())
            pools[kt] = base.repeat(reps)[:tot].contiguous()
        else:
            a = I.generate("uniform", tot, 5 + kt, bits, device="cuda")
            zf = I.generate("zipf", tot, 7 + kt, bits, device="cuda")
            mask = torch.from_numpy(np.repeat(zipf[idx], sizes[idx])).cuda()
            pools[kt] = torch.where(mask, zf, a)
            del a, zf, mask
        outs_one[kt] = torch.empty_like(pools[kt])
        outs_srv[kt] = torch.empty_like(pools[kt])
        off = 0
        o = [0]
        for i in idx:
            views.append((i, kt, off, int(sizes[i])))
            off += int(sizes[i])
            o.append(off)
        offs[kt] = torch.tensor(o, dtype=torch.int64, device="cuda")
    views.sort()
    req = [(kt, pools[kt][o:o + m], outs_one[kt][o:o + m], outs_srv[kt][o:o + m]) for _, kt, o, m in views]
    plans = []
    t_tune = time.perf_counter()
    for kt, src, _, _ in req:
        if tuned:
            cfg = ams.tune(src.numel(), kt)
            plans.append(dict(levels=cfg["levels"], buckets=cfg["buckets"], b=cfg["b"], a=cfg["a"],
                              cap=cfg["cap"]))
        else:
            plans.append(dict(levels=2, buckets=[64, 64]))
    t_tune = time.perf_counter() - t_tune
    # one-at-a-time service times back to back (warm), for the arrival rate
    for i, (kt, src, dst, _) in enumerate(req[:20]):
        ams.sort_keys_into(src, dst, kt=kt, **plans[i])
    ams.sync()
    service = np.zeros(N)
    for i, (kt, src, dst, _) in enumerate(req):
        t0 = time.perf_counter()
        ams.sort_keys_into(src, dst, kt=kt, **plans[i])
        ams.sync()
        service[i] = time.perf_counter() - t0
    rate = 1.1 * N / service.sum()
    arrivals = np.cumsum(np.random.default_rng(seed + 1).exponential(1.0 / rate, N))
    # (a) one at a time, replayed at the arrival times (measured)
    done_one = np.zeros(N)
    t_start = time.perf_counter()
    for i, (kt, src, dst, _) in enumerate(req):
        due = t_start + arrivals[i]
        while time.perf_counter() < due:
            d = due - time.perf_counter()
            if d > 2e-4:
                time.sleep(d - 1e-4)
        ams.sort_keys_into(src, dst, kt=kt, **plans[i])
        ams.sync()
        done_one[i] = time.perf_counter() - t_start
    lat_one = (done_one - arrivals) * 1e3
    one_tput = sizes.sum() / (done_one.max() - arrivals[0])
    # (b) the server on the same stream of arrivals; its worker contexts are sized for
    # the largest request of the stream first (no allocation inside the timed run)
    srv = ams.Server(hbm_budget_bytes=64 << 30, streams=streams, pack_max_keys=1 << 16)
    need = [ams.request_scratch_bytes(int(sizes[i]), int(kts[i]), **plans[i]) for i in range(N)]
    big = int(np.argmax(need))
    srv.reserve(int(sizes[big]), int(kts[big]), **plans[big])
    tickets = [None] * N
    t_start_ns = time.monotonic_ns()

    def client():
        for i, (kt, src, _, dst) in enumerate(req):
            due = t_start_ns + int(arrivals[i] * 1e9)
            while time.monotonic_ns() < due:
                d = (due - time.monotonic_ns()) / 1e9
                if d > 2e-4:
                    time.sleep(d - 1e-4)
            tickets[i] = srv.submit(src, dst, kt=kt, **plans[i])

    th = threading.Thread(target=client)
    th.start()
    t_done = np.zeros(N)
    for i in range(N):
        while tickets[i] is None:
            time.sleep(1e-5)
        _, t1 = srv.wait(tickets[i])
        t_done[i] = (t1 - t_start_ns) / 1e9
    th.join()
    counters = srv.counters()
    srv.close()
    lat_srv = (t_done - arrivals) * 1e3
    srv_tput = sizes.sum() / (t_done.max() - arrivals[0])
    # results: the server's outputs equal the one-at-a-time outputs, which are sorted
    # per request and hold their request's keys
    same = all(torch.equal(outs_one[kt], outs_srv[kt]) for kt in pools)
    sorted_ok = True
    for kt in pools:
        if kt == 2:
            sorted_ok = sorted_ok and _check_sorted_f32(pools[kt], outs_one[kt], offs[kt])
        else:
            sorted_ok = sorted_ok and _check_sorted(pools[kt], outs_one[kt], 64 if kt == 1 else 32, offs[kt])
    res = {
        "requests": N, "total_keys": int(sizes.sum()), "rate_per_s": float(rate),
        "budget_bytes": 64 << 30, "streams": streams, "pack_max_keys": 1 << 16,
        "plans": "autotuned per size class" if tuned else "2 levels, r = 64 x 64",
        "tune_s": t_tune,
        "server": {"keys_per_s": float(srv_tput), "p50_ms": float(np.percentile(lat_srv, 50)),
                   "p99_ms": float(np.percentile(lat_srv, 99))},
        "one_at_a_time": {"keys_per_s": float(one_tput), "p50_ms": float(np.percentile(lat_one, 50)),
                          "p99_ms": float(np.percentile(lat_one, 99)),
                          "how": "measured: requests replayed at the same arrival times, one sort at a time"},
        "results_equal": bool(same), "results_sorted": bool(sorted_ok),
        "server_counters": counters,
    }
    del pools, outs_one, outs_srv, req
    torch.cuda.empty_cache()
    return res


def _check_sorted_f32(src, dst, offsets):
    """Float keys: every segment of dst is in float order (-0.0 before +0.0) and holds
    the bit patterns of the same segment of src (order-independent hash)."""
    import torch
    from paper_1410_6754_gb300.inputs import _mix_t

    def omap(t):
        b = t.view(torch.int32).to(torch.int64) & 0xFFFFFFFF
        return torch.where(b >> 31 == 1, b ^ 0xFFFFFFFF, b | 0x80000000)
    o, oi = omap(dst), omap(src)
    lens = offsets[1:] - offsets[:-1]
    seg = torch.repeat_interleave(torch.arange(lens.numel(), device=dst.device), lens)
    ok = bool(((o[1:] >= o[:-1]) | (seg[1:] != seg[:-1])).all())
    z = torch.zeros(lens.numel(), dtype=torch.int64, device=dst.device)
    return ok and bool(torch.equal(z.clone().index_add_(0, seg, _mix_t(oi)), z.clone().index_add_(0, seg, _mix_t(o))))


def _e2e_pipelined(ams, host_src, dst, kw, steps, dist, world, n, w):
    """The end-to-end sorts again, pipelined the way a caller with a stream of inputs
    would run them: ams_sort_host_async on two contexts and two streams, one page-locked
    host array per step (each holding the same unsorted input), so that one step's copy
    back overlaps the next step's copy in and sort.  Timed on the host from the first
    enqueue to the end of the last copy back, three repetitions (the median is the
    value; all are listed); two results are checked in each.  The rate of one copy in
    each direction at once is listed beside it: that is what the overlap can reach."""
    import time

    import torch
    ctxs = [ams.Context(), ams.Context()]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    bufs = []
    for _ in range(steps):
        h = torch.empty_like(host_src, pin_memory=True)
        h.copy_(host_src)
        bufs.append(h)
    for i in range(2):  # size both contexts' staging and scratch (outside the timing)
        ams.sort_host_async(bufs[i], **kw, ctx=ctxs[i], stream=streams[i])
        ctxs[i].sync()
    want = dst.cpu()  # the sorted input
    # the host link with one copy in each direction at once (what the overlap can reach)
    half = host_src.numel() // 2
    scratch = torch.empty(half, dtype=dst.dtype, device=dst.device)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(streams[0]):
        scratch.copy_(bufs[0][:half], non_blocking=True)
    with torch.cuda.stream(streams[1]):
        bufs[1][half:].copy_(dst[half:], non_blocking=True)
    torch.cuda.synchronize()
    duplex = 2 * half * host_src.element_size() / (time.perf_counter() - t0) / 1e9
    del scratch
    reps, ok = [], True
    for _ in range(3):
        for h in bufs:  # every step starts from the unsorted input (outside the timing)
            h.copy_(host_src)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(steps):
            ams.sort_host_async(bufs[i], **kw, ctx=ctxs[i % 2], stream=streams[i % 2])
        for c in ctxs:
            c.sync()
        reps.append(max_over_ranks(time.perf_counter() - t0, dist, "cuda"))
        ok = ok and bool(torch.equal(bufs[0], want)) and bool(torch.equal(bufs[-1], want))
    for c in ctxs:
        c.close()
    del bufs
    t = sorted(reps)[1]
    return {"value": world * n * steps / t, "unit": "keys/s", "steps": steps, "contexts": 2, "streams": 2,
            "reps_keys_per_s": [round(world * n * steps / r) for r in reps], "duplex_copy_gbs": round(duplex, 1),
            "h2d_bytes_per_step": n * w, "d2h_bytes_per_step": n * w, "ok": ok,
            "api": "ams_sort_host_async (pinned host buffers, one per step; copies inside the timed region; "
                   "median of 3 repetitions)"}


def run_ams(args, wl):
    import torch
    rank, world, local_rank = _dist_env()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    if rank == 0:
        import __graft_entry__
        __graft_entry__.build()
    if dist:
        dist.barrier()
    import paper_1410_6754_gb300 as ams
    from paper_1410_6754_gb300 import inputs as I

    n, bits = wl["n"], wl["bits"]
    offsets = None
    if wl.get("segments"):
        import numpy as np
        lens = I.segment_lengths(wl["segments"], n, 4, max_log2=20)
        off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        n = int(off[-1])
        offsets = torch.from_numpy(off).cuda()
    src = I.generate(wl["dist"], n, rank, bits, device="cuda")
    dst = torch.empty_like(src)
    ctx = ams.Context()
    kw = dict(levels=wl["levels"], buckets=wl["buckets"], seed=0, a=wl["a"], b=wl["b"], kt=wl["kt"])
    if offsets is not None:
        kw["offsets"] = offsets
    for _ in range(args.warmup):
        ctx.sort(src, dst, **kw)
    ctx.sync()
    if not _check_sorted(src, dst, bits, offsets):
        print(json.dumps({"error": "output check failed"}), flush=True)
        return 1
    ctx.stats()  # reset the launch / event tallies
    torch.cuda.synchronize()
    sampler = ClockSampler(_gpu_index(local_rank))
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    # headline: the sorts alone (no per-kernel events)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        ctx.sort(src, dst, **kw)
    e1.record()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    st_head = ctx.stats()
    ms = max_over_ranks(ms, dist, "cuda")
    value = job_rate(world, args.steps * n, ms * 1e-3)
    # kernel shares: a second timed pass with CUDA events around every kernel (on the
    # stream the kernels are launched on)
    tsteps = max(3, min(args.steps, 20))
    for _ in range(tsteps):
        ctx.sort(src, dst, flags=ams.FLAG_PHASE_TIMERS, **kw)
    ctx.sync()
    st = ctx.stats()

    # dominant kernel: algorithmic bytes per launch / average launch time
    w = bits // 8
    peak, peak_src = _peaks()
    calls_per_step = {k: st["kernel_calls"][k] / max(1, tsteps) for k in st["kernel_calls"]}
    dom = max(KIND_BYTES, key=lambda k: st["kernel_ms"][k])
    avg_ms = st["kernel_ms"][dom] / max(1, st["kernel_calls"][dom])
    bytes_per_launch = KIND_BYTES[dom] * w * st["kernel_elems"][dom] / max(1e-9, calls_per_step[dom])
    achieved = bytes_per_launch / (avg_ms * 1e-3) / 1e9
    step_bytes = (wl["levels"] + 1) * 2 * n * w
    share = {k: round(st["kernel_ms"][k] / max(1e-9, sum(st["kernel_ms"].values())), 4)
             for k in st["kernel_ms"]}

    # end to end through the host-buffer entry point (pinned host memory)
    e2e = None
    if args.e2e_steps > 0 and offsets is None:
        host_src = src.cpu().pin_memory()
        host = torch.empty_like(host_src).pin_memory()
        times = []
        for i in range(args.e2e_steps + 1):
            host.copy_(host_src)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ams.sort_host(host, **kw)
            times.append(time.perf_counter() - t0)
        e2e_s = max_over_ranks(statistics.median(times[1:]), dist, "cuda")
        e2e = {"value": job_rate(world, n, e2e_s), "unit": "keys/s", "h2d_bytes_per_step": n * w,
               "d2h_bytes_per_step": n * w, "steps": args.e2e_steps,
               "api": "ams_sort_host (pinned host buffers, copies inside the timed region)"}
        del host
        if world == 1:  # (8 page-locked copies of the input per rank: one process only)
            e2e["pipelined"] = _e2e_pipelined(ams, host_src, dst, kw, max(args.e2e_steps, 8), dist, world, n, w)
        del host_src

    plain = None
    if offsets is not None and rank == 0:
        plain = _plain_per_segment(src, offsets, kw)
    cpu = None
    if rank == 0 and world == 1 and args.cpu_seconds > 0 and offsets is None:
        import oracle as O
        m = 1 << 23
        sample = src[:m].cpu().numpy().view("uint64" if bits == 64 else "uint32")
        reps, t0 = 0, time.perf_counter()
        while reps < 1 or (time.perf_counter() - t0 < args.cpu_seconds and reps < 8):
            O.sort_keys(wl["kt"], sample)
            reps += 1
        dt = (time.perf_counter() - t0) / reps
        cpu = {"value": m / dt, "unit": "keys/s", "cores": 1, "kind": "oracle",
               "sample": f"first {m} keys of the same input, numpy stable sort, one thread, "
                         f"{reps} repetitions", **_cpu_info()}

    extras = {}
    if rank == 0 and world == 1 and not args.no_extras and wl is WORKLOADS["two_level_u64"]:
        del src, dst
        ctx.close()
        torch.cuda.empty_cache()
        t_ex = time.perf_counter()
        extras["configs"] = run_configs(peak)
        extras["segmented"] = run_segmented_sub()
        extras["rlm"] = run_rlm_sub(peak)
        extras["serving"] = serving_bench(args.requests, args.server_streams, args.tuned)
        extras["extras_wall_s"] = time.perf_counter() - t_ex

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "keys/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": wl["dtype"], "data": "synthetic",
            "config": {"workload": wl["desc"], "n": n, "levels": wl["levels"],
                       "buckets": wl["buckets"], "b": wl["b"], "a": wl["a"] or "ceil(1.6 log10 n)",
                       "parallelism": f"replicas x{world}",
                       "l2": ("input and output exceed L2; no flush" if n * w > (256 << 20)
                              else "input fits L2; no flush (not a bench line)"),
                       **({"segments": wl["segments"], "plain_per_segment_keys_per_s": plain}
                          if offsets is not None else {})},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "traffic": _traffic(dom),
                         "peak_source": f"{peak_src} hbm copy bandwidth",
                         "alg_bytes_per_launch": bytes_per_launch, "avg_launch_ms": avg_ms,
                         "timing": f"per-kernel CUDA events on the launch stream, separate pass of {tsteps} sorts"},
            "step_roofline": {"alg_bytes": step_bytes, "achieved_gbs": step_bytes / (ms / args.steps * 1e-3) / 1e9,
                              "frac": step_bytes / (ms / args.steps * 1e-3) / 1e9 / peak,
                              "definition": "(levels + 1) x (read + write) x n x key bytes per step"},
            "kernel_share": share,
            "kernel_avg_ms": {k: st["kernel_ms"][k] / max(1, st["kernel_calls"][k]) for k in st["kernel_ms"]},
            "e2e": e2e, "cpu_baseline": cpu, "clocks": clocks,
            "gpu_launches": st_head["kernel_launches"],
            **extras,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_serving(args):
    """The serving workload on its own line (see serving_bench)."""
    import __graft_entry__
    __graft_entry__.build()
    r = serving_bench(args.requests, args.server_streams, args.tuned)
    line = {
        "metric": METRIC, "value": r["server"]["keys_per_s"], "unit": "keys/s", "n_gpus": 1,
        "steps": r["requests"], "warmup": 20, "ms_per_step": None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64/f32", "data": "synthetic",
        "config": {"workload": f"serving: {r['requests']} Poisson requests, sizes log-uniform [2^10, 2^26], "
                               "50% u32 / 30% u64 / 20% f32, uniform or Zipf(1.1) values"},
        "serving": r,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ams", choices=["ams", "reference"])
    ap.add_argument("--workload", default="two_level_u64", choices=sorted(WORKLOADS) + ["serving"])
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--requests", type=int, default=400, help="serving: request count")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline only (no configs / segmented / serving sub-objects)")
    ap.add_argument("--server-streams", type=int, default=4, help="serving workload: worker streams")
    ap.add_argument("--tuned", action="store_true", help="serving workload: autotuned plans per size class")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.workload == "serving":
        return run_serving(args)
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, wl)
    return run_ams(args, wl)


if __name__ == "__main__":
    sys.exit(main())
