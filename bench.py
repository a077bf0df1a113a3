#!/usr/bin/env python
"""Benchmark of bulk generation with libxr on GB300.

One step = the whole path over one batch: for each of the 8 generators and
each output type (native word, double) -- seed a base state with SplitMix64(42),
jump-start 2^20 streams (stream i = J^(first + i)(base)), and fill 2^20 x 2^10
outputs.  Every step writes 120 GiB of output.  `value` is generated bytes per
second (GB/s, 1e9) over all ranks with the inputs already on the device;
`e2e` repeats the step through the host-buffer entry point, device-to-host
copies included.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl xr|reference]

Under torchrun every rank is an independent replica over a disjoint range of
stream indices (weak scaling, no collective on the data path).
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

import workloads as W  # noqa: E402

METRIC = "generated GB/s & % of HBM roofline (batched vs plain, 1 GB300); p50/p99 latency"
UNIT = "GB/s"
FILL_SOURCES = ("paper_1805_01407_gb300/csrc/xr_fill_impl.cuh", "paper_1805_01407_gb300/csrc/xr_device.cuh")
FUSED_SOURCES = FILL_SOURCES + ("paper_1805_01407_gb300/csrc/xr_fill_streams.cuh", "paper_1805_01407_gb300/csrc/xr_f2.cuh")
LC_SOURCES = ("paper_1805_01407_gb300/csrc/xr_analysis.cu",)


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["xr", "reference"], default="xr")
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--cpu-seconds", type=float, default=10.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-batched", action="store_true")
    p.add_argument("--no-serve", action="store_true")
    p.add_argument("--no-extra", action="store_true")
    p.add_argument("--no-analysis", action="store_true")
    p.add_argument("--no-jumpstart", action="store_true")
    p.add_argument("--serve-requests", type=int, default=20000)
    p.add_argument("--batched-steps", type=int, default=5)
    p.add_argument("--profile", choices=["fill", "fill-jobs", "streams", "fused", "batch", "lc", "lc-bulk"],
                   default=None,
                   help="run a small case for an ncu capture instead of the benchmark")
    p.add_argument("--profile-variant", default="xoshiro256**")
    p.add_argument("--profile-dtype", default=None)
    p.add_argument("--profile-streams", type=int, default=1 << 16)
    p.add_argument("--profile-launches", type=int, default=3)
    p.add_argument("--profile-max-len", type=int, default=1 << 24,
                   help="batch profile: largest request length")
    return p.parse_args()


def dist_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_first(rank, S):
    """First stream index of a rank: rank r owns streams [r S, (r + 1) S) of
    the same base, so ranks never overlap and need no collective."""
    return rank * S


def max_over_ranks(value, dist, device):
    """Largest value over all ranks (the slowest rank's time)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def jobs():
    return [(v, d) for v in W.CONFIG_BULK["variants"] for d in (W.native_dtype(v), "f64")]


def dtype_bytes(d):
    return 8 if d in ("u64", "f64") else 4  # u32, f32


def state_bytes(v):
    return 32 if v.startswith("xoshiro256") else 16


def workload_config(world):
    c = W.CONFIG_BULK
    S, m = c["S"], c["m"]
    nbytes = sum(S * m * dtype_bytes(d) for _, d in jobs())
    return {
        "workload": "bulk fill: 8 generators (xoshiro256+/++/**, xoroshiro128+/++/**, "
                    "xoshiro128**/++) x {native word, f64}; 2^20 streams x 2^10 outputs per job "
                    "(2^30 values); SplitMix64(42) base; stream i = J^(first+i)(base)",
        "streams": S, "outputs_per_stream": m, "jobs_per_step": len(jobs()),
        "values_per_step": len(jobs()) * S * m, "bytes_per_step": nbytes,
        "values_per_step_all_ranks": world * len(jobs()) * S * m,
        "l2": "each launch writes 4-8 GiB, far larger than the 129 MB L2; no flush needed",
        "parallelism": "replicas over disjoint stream ranges" if world > 1 else "single GPU",
    }, nbytes


# ---------------------------------------------------------------- clocks

CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    """nvidia-smi sampling every 200 ms while the timed region runs."""

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="xr_clocks_", suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + CLOCK_FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu_index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "note": "nvidia-smi unavailable"}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = [n for k, n in enumerate(names) if any(r[5 + k].lower() == "active" for r in rows)]
        power = [num(r[3]) for r in rows if num(r[3]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": num(rows[0][2]), "reasons": reasons, "samples": len(rows),
                "power_w_max": max(power) if power else None}


# ---------------------------------------------------------------- roofline inputs

def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0}, "fallback"


def fill_source_hash(sources=FILL_SOURCES):
    h = hashlib.sha256()
    for p in sources:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes per fill launch from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "fill_traffic.txt")
    try:
        kv = {}
        with open(path) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("source_sha") != fill_source_hash():
            return None
        return {"bytes_per_launch": float(kv["dram_bytes_per_launch_full_size"]),
                "algorithmic_bytes_per_launch": float(kv.get("algorithmic_bytes_per_launch", "nan")),
                "note": kv.get("scaling", "")}
    except (OSError, KeyError, ValueError):
        return None


def recorded_fused_counts():
    """Integer ALU lane operations and shared-memory wavefronts per stream of
    the fused stream-start fill (xoshiro256++, 64 u64 outputs), from the
    committed ncu summary, if taken on the current sources; else None."""
    path = os.path.join(ROOT, "profiles", "fill_streams__xoshiro256pp_2p21x64.txt")
    try:
        kv = {}
        with open(path) as f:
            for line in f:
                if ":" in line and not line.startswith("#") and not line.startswith(" "):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("source_sha") != fill_source_hash(FUSED_SOURCES):
            return None
        return {"alu_lane_ops_per_stream": float(kv["alu_lane_ops_per_stream"]),
                "shared_wavefronts_per_stream": float(kv["shared_wavefronts_per_stream"])}
    except (OSError, KeyError, ValueError):
        return None


def recorded_lc_alu_ops():
    """ALU-pipe lane operations of one Berlekamp-Massey launch of the bulk
    linear-complexity configuration (448 sequences x 2^16 bits), from the
    committed ncu summary, if taken on the current source; else None."""
    path = os.path.join(ROOT, "profiles", "berlekamp_massey__bulk_448x65536.txt")
    try:
        kv = {}
        with open(path) as f:
            for line in f:
                if ":" in line and not line.startswith("#") and not line.startswith(" "):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("source_sha") != fill_source_hash(LC_SOURCES):
            return None
        return float(kv["alu_lane_ops_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


def recorded_alu_ops():
    """ALU-pipe lane operations per value of each fill job, from the committed
    ncu instruction counts (sm__inst_executed_pipe_alu x 32 / values), if they
    were taken on the current kernel source; {} otherwise."""
    path = os.path.join(ROOT, "profiles", "fill_alu_ops__all_generators_2p16x2p10.txt")
    try:
        ops, sha = {}, None
        with open(path) as f:
            for line in f:
                if line.startswith("source_sha:"):
                    sha = line.split(":", 1)[1].strip()
                parts = line.split()
                if len(parts) >= 3 and parts[0] in W.ALL_VARIANTS:
                    ops[(parts[0], parts[1])] = float(parts[2])
        return ops if sha == fill_source_hash() else {}
    except (OSError, ValueError):
        return {}


def write_ceiling(xr, out, stream):
    """The HBM write ceiling measured here: the library's store-only kernel
    (16-byte stores, 2, 4 or 8 CTAs of 512 threads per SM) and
    cudaMemsetAsync over the same buffer, best of 10 each, CUDA events on the
    stream."""
    import torch
    nbytes = out.numel() * out.element_size()

    def best(fn, reps=10):
        fn()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return nbytes / (min(ts) / 1e3) / 1e9

    store = {k: best(lambda: xr.probe_store(out, k, stream=stream)) for k in (2, 4, 8)}
    memset = best(lambda: xr.probe_memset(out, stream=stream))
    rows, row_bytes = W.CONFIG_BULK["S"], W.CONFIG_BULK["m"] * 8
    tiles = {name: best(lambda: xr.probe_tile_store(out, rows, row_bytes, cfg, stream=stream))
             for cfg, name in ((0, "2 warps x 6 tiles"), (1, "1 warp x 8 tiles"), (2, "1 warp x 3 tiles"))}
    peak = max(max(store.values()), memset)
    return {"write_peak_gbs": peak, "store_kernel_gbs": store, "memset_gbs": memset, "bytes": nbytes,
            "tile_store_gbs": tiles,
            "how": "best of 10, CUDA events on the launching stream, over the bench's 8 GiB output buffer; "
                   "tile_store_gbs: the fill's own store pattern (2^20 rows of 8 KiB as 32-row x 128-byte "
                   "TMA tiles) with nothing generated"}


def alu_ceiling(xr, stream):
    """The integer-ALU ceiling measured here: independent lop3 chains on every
    SM (8 CTAs of 256 threads per SM), lane operations per second, best of 5."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    sink = torch.zeros(4, dtype=torch.int32, device="cuda")
    blocks, iters = sms * 8, 1 << 16
    xr.probe_alu(sink, blocks, iters, stream=stream)
    ts = []
    for _ in range(5):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        xr.probe_alu(sink, blocks, iters, stream=stream)
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    lane_ops = blocks * 256 * iters * 16
    return {"alu_lane_ops_per_s": lane_ops / (min(ts) / 1e3), "sms": sms, "ms": min(ts),
            "how": "%d CTAs x 256 threads x %d x 16 lop3, best of 5" % (blocks, iters)}


def job_rooflines(jobs_bytes, write_peak, alu_peak, alu_ops):
    """Per job: the slower of the HBM write bound (write_peak) and the integer
    bound (alu_peak lane operations/s over the job's ALU operations per
    value), in GB/s of output, and which binds."""
    res = {}
    for (v, d), bpv in jobs_bytes.items():
        ops = alu_ops.get((v, d))
        alu_gbs = alu_peak / ops * bpv / 1e9 if ops else None
        bound = "alu" if alu_gbs is not None and alu_gbs < write_peak else "hbm"
        res[(v, d)] = {"alu_lane_ops_per_value": ops, "alu_bound_gbs": alu_gbs,
                       "roofline_gbs": min(write_peak, alu_gbs) if alu_gbs else write_peak, "bound": bound}
    return res


# ---------------------------------------------------------------- oracle timing

def oracle_sample(streams, m, seed):
    """Run the oracle on `streams` streams per job; returns (bytes, seconds)."""
    import oracle as O
    nbytes, t0 = 0, time.perf_counter()
    for v, d in jobs():
        base = O.seed(v, seed)
        raw = O.bulk_fill(v, "jump", base, streams, m)
        if d == "f64":
            O.to_f64(v, raw)
        nbytes += streams * m * dtype_bytes(d)
    return nbytes, time.perf_counter() - t0


def cpu_baseline(seconds):
    m, seed = W.CONFIG_BULK["m"], W.CONFIG_BULK["seed"]
    b, t = oracle_sample(64, m, seed)
    streams = max(64, int(64 * seconds / max(t, 1e-3)))
    b, t = oracle_sample(streams, m, seed)
    return {"value": b / t / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "16 jobs (8 generators x {native, f64}) x %d streams x %d outputs "
                      "(stream i = J^i(SplitMix64(42)) by one jump after another), single-threaded "
                      "plain C oracle, %.1f s" % (streams, m, t),
            "seconds": t, "bytes": b}


def _oracle_worker(task):
    streams, m, seed = task
    return oracle_sample(streams, m, seed)


def cpu_baseline_all_cores(streams):
    """The same oracle sample once per host core, in spawned processes started
    together (one single-threaded oracle each): aggregate bytes / wall time."""
    import multiprocessing as mp
    m, seed = W.CONFIG_BULK["m"], W.CONFIG_BULK["seed"]
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(cores) as pool:
        pool.map(_oracle_worker, [(1, m, seed)] * cores, chunksize=1)  # every process loads the oracle
        t0 = time.perf_counter()
        res = pool.map(_oracle_worker, [(streams, m, seed)] * cores, chunksize=1)
        wall = time.perf_counter() - t0
    b = sum(r[0] for r in res)
    return {"value": b / wall / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d processes, each the single-threaded plain C oracle on 16 jobs x %d streams x %d outputs "
                      "(the cpu_baseline recipe), started together; %.1f s wall" % (cores, streams, m, wall),
            "seconds": wall, "bytes": b}


def extra_cpu_baseline(streams=64):
    """The oracle on the other generators of the paper, the same recipe as the
    extra-generator leg (SplitMix64(42) base, streams J^i, 2^10 outputs each,
    native word and f64) on `streams` streams per job."""
    import oracle as O
    m, seed = W.CONFIG_BULK["m"], W.CONFIG_BULK["seed"]
    nbytes, t0 = 0, time.perf_counter()
    for v in W.EXTRA_VARIANTS:
        raw = O.bulk_fill(v, "jump", O.seed(v, seed), streams, m)
        O.to_f64(v, raw)
        nbytes += streams * m * (dtype_bytes(W.native_dtype(v)) + 8)
    t = time.perf_counter() - t0
    return {"value": nbytes / t / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "9 generators x {native, f64} x %d streams x %d outputs, single-threaded plain C, %.2f s"
                      % (streams, m, t)}


def analysis_cpu_baseline():
    """The oracle on the analysis workloads of run_analysis (same inputs)."""
    import oracle as O
    t0 = time.perf_counter()
    O.zeroland("xoshiro256**", 1000, 4)
    t1 = time.perf_counter()
    L = O.linear_complexity("xoshiro256+", 1, ANALYSIS_LC_SMALL[2], 1)
    t2 = time.perf_counter()
    c = W.CONFIG_LC_BULK
    jobs = W.lc_bulk_jobs(**c)
    sample = jobs[::56]
    for v, b, N in sample:
        O.linear_complexity(v, b, N, c["seed"])
    t3 = time.perf_counter()
    per_job = (t3 - t2) / len(sample)
    return {"kind": "oracle", "cores": 1, "zeroland_ms": (t1 - t0) * 1e3, "lc_small_ms": (t2 - t1) * 1e3,
            "lc_small_value": L, "lc_bulk_ms_estimate": per_job * len(jobs) * 1e3,
            "sample": "zeroland and lc_small: the same calls as the device; lc_bulk: %d of the %d sequences "
                      "(every 56th), scaled to all; single-threaded plain C" % (len(sample), len(jobs))}


# ---------------------------------------------------------------- reference arm

def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    cfg, _ = workload_config(1)
    m, seed = W.CONFIG_BULK["m"], W.CONFIG_BULK["seed"]
    streams = 1024
    for _ in range(args.warmup):
        oracle_sample(streams, m, seed)
    tot_b, tot_t = 0, 0.0
    for _ in range(args.steps):
        b, t = oracle_sample(streams, m, seed)
        tot_b += b
        tot_t += t
    value = tot_b / tot_t / 1e9
    sample = ("each step: 16 jobs (8 generators x {native, f64}) x %d streams x %d outputs, "
              "single-threaded plain C oracle" % (streams, m))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": cfg, "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- libxr arm

def run_xr(args):
    import torch
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1805_01407_gb300 as xr
    from paper_1805_01407_gb300 import build as libbuild
    libbuild.build()

    cfg, bytes_per_step = workload_config(world)
    c = W.CONFIG_BULK
    S, m, seed = c["S"], c["m"], c["seed"]
    first = shard_first(rank, S)
    ctx = xr.Context(local)
    stream = torch.cuda.current_stream()
    # Jobs are pipelined over two streams: the seed and stream starts of job
    # j+1 (side stream, higher priority, double-buffered states) overlap the
    # fill of job j (main stream); fills stay in order on the main stream.
    side = torch.cuda.Stream(priority=-1)
    base = [ctx.empty_states("xoshiro256**", 1) for _ in range(2)]
    states = [ctx.empty_states("xoshiro256**", S) for _ in range(2)]
    out = torch.empty(S * m * 8, dtype=torch.uint8, device="cuda")
    views = {d: out.view(xr.torch_dtype(d)) for d in ("u64", "u32", "f64")}
    J = jobs()
    ready = [torch.cuda.Event() for _ in range(2)]
    freed = [torch.cuda.Event() for _ in range(2)]

    def new_events():
        return [tuple(torch.cuda.Event(enable_timing=True) for _ in range(4)) for _ in J]

    def step(evs=None):
        for j, (v, d) in enumerate(J):
            b = j & 1
            side.wait_event(freed[b])
            if evs:
                evs[j][0].record(side)
            ctx.seed(v, seed, base[b], stream=side)
            ctx.make_streams(v, "jump", base[b], first, S, states[b], stream=side)
            if evs:
                evs[j][1].record(side)
            ready[b].record(side)
            stream.wait_event(ready[b])
            if evs:
                evs[j][2].record(stream)
            ctx.fill(v, states[b], S, m, d, views[d], stream=stream)
            if evs:
                evs[j][3].record(stream)
            freed[b].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    assert ctx.status() == 0

    # the two ceilings of the fill, measured here before the timed region
    wc = write_ceiling(xr, out, stream)
    ac = alu_ceiling(xr, stream)

    step_events = [new_events() for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    n0 = xr.launch_count()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    side.wait_event(t0)
    for k in range(args.steps):
        step(step_events[k])
    stream.wait_stream(side)
    t1.record(stream)
    torch.cuda.synchronize()
    launches = xr.launch_count() - n0
    elapsed_ms = t0.elapsed_time(t1)
    clk = clocks.stop()
    fill_ms = {jd: [step_events[k][j][2].elapsed_time(step_events[k][j][3]) for k in range(args.steps)]
               for j, jd in enumerate(J)}
    mk_ms = {jd: [step_events[k][j][0].elapsed_time(step_events[k][j][1]) for k in range(args.steps)]
             for j, jd in enumerate(J)}
    elapsed_ms = max_over_ranks(elapsed_ms, dist, "cuda")
    status = ctx.status()

    value = world * bytes_per_step * args.steps / (elapsed_ms / 1e3) / 1e9
    peaks, peak_kind = measured_peaks()
    peak = float(peaks["hbm_gbs"])
    fill_bytes = fill_time = 0.0
    per_job = {}
    for (v, d), times in fill_ms.items():
        alg = S * m * dtype_bytes(d) + S * state_bytes(v)
        fill_bytes += alg * len(times)
        fill_time += sum(times) / 1e3
        per_job["%s/%s" % (v, d)] = {"fill_ms": statistics.median(times),
                                     "fill_gbs": alg / (statistics.median(times) / 1e3) / 1e9,
                                     "streams_ms": statistics.median(mk_ms[(v, d)])}
    achieved = fill_bytes / fill_time / 1e9
    traffic = recorded_traffic()
    alu_ops = recorded_alu_ops()
    roofs = job_rooflines({(v, d): (S * m * dtype_bytes(d) + S * state_bytes(v)) / (S * m) for v, d in J},
                          wc["write_peak_gbs"], ac["alu_lane_ops_per_s"], alu_ops)
    for (v, d), r in roofs.items():
        pj = per_job["%s/%s" % (v, d)]
        pj.update(bound=r["bound"], roofline_gbs=r["roofline_gbs"], alu_bound_gbs=r["alu_bound_gbs"],
                  frac_of_roofline=pj["fill_gbs"] / r["roofline_gbs"])
    # the step's roofline: every job's bytes at its own bound
    step_roof = fill_bytes / sum(len(fill_ms[jd]) * (S * m * dtype_bytes(jd[1]) + S * state_bytes(jd[0]))
                                 / (roofs[jd]["roofline_gbs"] * 1e9) for jd in J) / 1e9
    mk_total = sum(sum(t) for t in mk_ms.values()) / args.steps
    fill_total = sum(sum(t) for t in fill_ms.values()) / args.steps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": cfg, "impl": "xr",
        "outputs_per_s": world * cfg["values_per_step"] * args.steps / (elapsed_ms / 1e3),
        "roofline": {"bound": "alu" if all(r["bound"] == "alu" for r in roofs.values()) else "hbm",
                     "kernel": "k_fill_tma (all 16 jobs)", "achieved": achieved,
                     "peak": peak, "peak_kind": "%s hbm_gbs (copy, read+write)" % peak_kind,
                     "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic["bytes_per_launch"] if traffic else None,
                     "traffic_note": traffic["note"] if traffic else None,
                     "algorithmic_bytes_per_launch_u64": S * m * 8 + S * 32,
                     "write_peak_gbs": wc["write_peak_gbs"], "frac_of_write_peak": achieved / wc["write_peak_gbs"],
                     "tile_store_ceiling_gbs": max(wc["tile_store_gbs"].values()),
                     "frac_of_tile_store_ceiling": achieved / max(wc["tile_store_gbs"].values()),
                     "write_ceiling": wc,
                     "alu_peak_lane_ops_per_s": ac["alu_lane_ops_per_s"], "alu_ceiling": ac,
                     "jobs_alu_bound": sorted("%s/%s" % jd for jd, r in roofs.items() if r["bound"] == "alu"),
                     "step_roofline_gbs": step_roof, "frac_of_step_roofline": achieved / step_roof,
                     "alu_ops_source": "profiles/fill_alu_ops__all_generators_2p16x2p10.txt" if alu_ops
                     else "not recorded for the current fill source: ALU bound not applied"},
        "step_breakdown_ms": {"fill": fill_total, "make_streams_overlapped": mk_total,
                              "not_in_fills": elapsed_ms / args.steps - fill_total},
        "per_job": per_job,
        "clocks": clk, "gpu_launches": launches, "status": status,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        line["cpu_baseline_all_cores"] = cpu_baseline_all_cores(
            max(64, line["cpu_baseline"]["bytes"] // (16 * 8 * W.CONFIG_BULK["m"]) // 4))
    if not args.no_batched:
        line["batched"] = run_batched(xr, ctx, args)
    if not args.no_serve:
        line["serving"] = run_serving(xr, ctx, args)
    if not args.no_extra:
        line["extra_generators"] = run_extra(xr, ctx, args, wc, ac)
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            line["extra_generators"]["cpu_baseline"] = extra_cpu_baseline()
    if not args.no_jumpstart:
        line["jumpstart"] = run_jumpstart(xr, ctx, args, wc, ac)
    if not args.no_extra:
        line["layouts_and_types"] = run_layouts(xr, ctx, wc)
    if not args.no_analysis:
        line["analysis"] = run_analysis(xr, ctx, args, ac)
    if not args.no_e2e:
        line["e2e"] = run_e2e(ctx, args, first, bytes_per_step, world, dist)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_batched(xr, ctx, args):
    """Batched uneven requests: 4096 requests (lengths log-uniform in [1, 2^24],
    8 generators, native/double, SplitMix64(r) seeds) in one persistent launch
    captured in a CUDA graph and tuned, against the plain path of one xr_seed +
    xr_fill_seq per request, on the same GPU and output arena."""
    import torch
    specs = W.batch_requests(**W.CONFIG_BATCH)
    seeds = [s for (_, _, _, s) in specs]
    reqs, offs, arena = xr.pack_requests([(v, dt, n, r) for r, (v, dt, n, _) in enumerate(specs)])
    nbytes = sum(n * dtype_bytes(dt) for (_, dt, n, _) in specs)
    b = xr.Batch(ctx, reqs)
    slots = torch.zeros(len(specs) * 32, dtype=torch.uint8, device="cuda")
    out = torch.empty(arena, dtype=torch.uint8, device="cuda")
    d_seeds = torch.tensor(seeds, dtype=torch.int64, device="cuda")
    tune_ms = b.tune(d_seeds, slots, out)
    opt, block = b.get_config()
    stream = torch.cuda.current_stream()
    for _ in range(2):
        b.run(d_seeds, slots, out, use_graph=True)
    torch.cuda.synchronize()
    times = []
    for _ in range(args.batched_steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.run(d_seeds, slots, out, use_graph=True)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    batch_ms = statistics.median(times)
    # plain: one seed + one xr_fill_seq per request, events around each request
    st = ctx.empty_states("xoshiro256**", 1)
    views = {d: out.view(xr.torch_dtype(d)) for d in ("u64", "u32", "f64")}
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in specs]
    plain_ms = []
    for rep in range(2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for r, (v, dt, n, _) in enumerate(specs):
            if rep:
                ev[r][0].record(stream)
            ctx.seed(v, seeds[r], st)
            es = dtype_bytes(dt)
            ctx.fill_seq(v, st, n, dt, views[dt][offs[r] // es: offs[r] // es + n])
            if rep:
                ev[r][1].record(stream)
        e1.record(stream)
        e1.synchronize()
        plain_ms.append(e0.elapsed_time(e1))
    per_req = sorted(ev[r][0].elapsed_time(ev[r][1]) for r in range(len(specs)))
    tasks = b.tasks
    b.close()
    q = lambda p: per_req[min(len(per_req) - 1, int(p * len(per_req)))]
    return {
        "workload": "4096 requests, lengths log-uniform in [1, 2^24] (%.1f GB), 8 generators, "
                    "native/f64, SplitMix64(r) seeds; one persistent launch in a CUDA graph" % (nbytes / 1e9),
        "value": nbytes / (batch_ms / 1e3) / 1e9, "unit": UNIT, "ms": batch_ms,
        "frac_of_measured_peak": nbytes / (batch_ms / 1e3) / 1e9 / measured_peaks()[0]["hbm_gbs"],
        "plain_value": nbytes / (plain_ms[-1] / 1e3) / 1e9, "plain_ms": plain_ms[-1],
        "speedup_vs_plain": plain_ms[-1] / batch_ms,
        "plain_request_ms_p50": q(0.5), "plain_request_ms_p99": q(0.99),
        "tuned": {"outputs_per_row": opt, "block": block, "best_trial_ms": tune_ms},
        "tasks": tasks,
    }


def run_extra(xr, ctx, args, wc, ac):
    """The other generators of the paper at the bulk size (2^20 streams x 2^10
    outputs, SplitMix64(42) base, jump-started): fill GB/s per output type,
    median of 5 launches timed with events on their stream."""
    import torch
    S, m, seed = W.CONFIG_BULK["S"], W.CONFIG_BULK["m"], W.CONFIG_BULK["seed"]
    stream = torch.cuda.current_stream()
    peak = measured_peaks()[0]["hbm_gbs"]
    alu_ops = recorded_alu_ops()
    res = {}
    for v in W.EXTRA_VARIANTS:
        base = ctx.empty_states(v, 1)
        states = ctx.empty_states(v, S)
        ctx.seed(v, seed, base)
        ctx.make_streams(v, "jump", base, 0, S, states)
        for d in (W.native_dtype(v), "f64"):
            out = ctx.empty_output(S * m, d)
            for _ in range(3):  # warm-up (the first job follows the serving leg)
                ctx.fill(v, states, S, m, d, out)
            ts = []
            for _ in range(5):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                ctx.fill(v, states, S, m, d, out)
                b.record(stream)
                b.synchronize()
                ts.append(a.elapsed_time(b))
            ms = statistics.median(ts)
            gbs = S * m * dtype_bytes(d) / (ms / 1e3) / 1e9
            r = job_rooflines({(v, d): dtype_bytes(d)}, wc["write_peak_gbs"], ac["alu_lane_ops_per_s"],
                              alu_ops)[(v, d)]
            res["%s/%s" % (v, d)] = {"fill_gbs": gbs, "fill_ms": ms, "frac_of_measured_peak": gbs / peak,
                                     "bound": r["bound"], "roofline_gbs": r["roofline_gbs"],
                                     "alu_bound_gbs": r["alu_bound_gbs"],
                                     "frac_of_roofline": gbs / r["roofline_gbs"]}
            del out
    torch.cuda.synchronize()
    assert ctx.status() == 0
    return res


def run_layouts(xr, ctx, wc):
    """The other output forms at the bulk size (2^20 streams x 2^10 values,
    SplitMix64(42) base, jump-started): the interleaved layout out[j S + i]
    (coalesced warp stores, no staging) beside stream-major, and float32
    outputs (upper 24 bits), with the 32-bit generator the paper recommends
    for floats (xoshiro128+) and a 64-bit one; fill alone, median of 5,
    events on the stream, against the measured write peak."""
    import torch
    S, m, seed = W.CONFIG_BULK["S"], W.CONFIG_BULK["m"], W.CONFIG_BULK["seed"]
    stream = torch.cuda.current_stream()
    res = {}
    for v, d, layout in (("xoshiro256**", "u64", "stream"), ("xoshiro256**", "u64", "interleaved"),
                         ("xoshiro256**", "f64", "interleaved"), ("xoshiro128+", "f32", "stream"),
                         ("xoshiro128+", "f32", "interleaved"), ("xoshiro256+", "f32", "stream")):
        base = ctx.empty_states(v, 1)
        states = ctx.empty_states(v, S)
        ctx.seed(v, seed, base)
        ctx.make_streams(v, "jump", base, 0, S, states)
        out = ctx.empty_output(S * m, d)
        for _ in range(2):
            ctx.fill(v, states, S, m, d, out, layout=layout)
        ts = []
        for _ in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.fill(v, states, S, m, d, out, layout=layout)
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        ms = statistics.median(ts)
        gbs = S * m * dtype_bytes(d) / (ms / 1e3) / 1e9
        res["%s/%s/%s" % (v, d, layout)] = {"fill_ms": ms, "fill_gbs": gbs,
                                            "frac_of_write_peak": gbs / wc["write_peak_gbs"]}
        del out, states
    torch.cuda.synchronize()
    assert ctx.status() == 0
    return res


# Table 13: xoshiro256+ bit 1 (complexity 32896) and xoroshiro128+ bit 2
# (349632, the largest), each from 2 L + 200 bits of SplitMix64(1).
ANALYSIS_LC_SMALL = ("xoshiro256+", 1, 2 * 32896 + 200)
ANALYSIS_LC_LARGE = ("xoroshiro128+", 2, 2 * 349632 + 200)


def run_analysis(xr, ctx, args, ac=None):
    """The paper's analysis workloads: escaping zeroland (Sec. 8; all one-bit
    states of xoshiro256**, 1000 outputs, windows of 4) timed with events, and
    Berlekamp-Massey linear complexity (Sec. 9.3) of two Table 13 rows timed
    around the blocking call (generation of the bits, the one-CTA
    Berlekamp-Massey, the 8-byte read back)."""
    import torch
    stream = torch.cuda.current_stream()
    ctx.zeroland("xoshiro256**", 1000, 4)
    ts = []
    for _ in range(5):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.zeroland("xoshiro256**", 1000, 4)
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    res = {"zeroland": {"workload": "xoshiro256**, 256 one-bit states x 1000 outputs, windows of 4",
                        "ms": statistics.median(ts)}}
    for key, (v, bit, N) in (("lc_small", ANALYSIS_LC_SMALL), ("lc_large", ANALYSIS_LC_LARGE)):
        st = ctx.empty_states(v, 1)
        ctx.seed(v, 1, st)
        ctx.linear_complexity(v, bit, N, st)
        ts, L = [], None
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            L = ctx.linear_complexity(v, bit, N, st)
            ts.append(time.perf_counter() - t0)
        ms = statistics.median(ts) * 1e3
        res[key] = {"workload": "%s bit %d, %d bits" % (v, bit, N), "value": L, "ms": ms,
                    "ns_per_bit": ms * 1e6 / N}
    c = W.CONFIG_LC_BULK
    jobs = W.lc_bulk_jobs(**c)
    states = torch.zeros(len(jobs) * 128, dtype=torch.uint8, device="cuda")
    for j, (v, _, _) in enumerate(jobs):
        ctx.seed(v, c["seed"], states[j * 128:])
    ctx.linear_complexity_many(jobs, states)
    ts = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        got = ctx.linear_complexity_many(jobs, states)
        ts.append(time.perf_counter() - t0)
    ms = statistics.median(ts) * 1e3
    res["lc_bulk"] = {"workload": "every bit of the 8 bulk generators, %d sequences x %d bits, SplitMix64(%d)"
                                  % (len(jobs), c["N"], c["seed"]),
                      "jobs": len(jobs), "ms": ms, "jobs_per_s": len(jobs) / (ms / 1e3),
                      "bits_per_s": len(jobs) * c["N"] / (ms / 1e3),
                      "lowest_bits": {v: got[[k for k, (vv, b, _) in enumerate(jobs) if vv == v][0]]
                                      for v in c["variants"]}}
    ops = recorded_lc_alu_ops()
    if ops and ac:
        # the Berlekamp-Massey kernel's ALU work at the ALU ceiling measured in
        # this run, against the whole call (bit generation and host side included)
        bound_ms = ops / ac["alu_lane_ops_per_s"] * 1e3
        res["lc_bulk"]["alu_roofline"] = {"bound": "alu", "alu_lane_ops_per_call": ops, "alu_bound_ms": bound_ms,
                                          "frac_of_call": bound_ms / ms,
                                          "source": "profiles/berlekamp_massey__bulk_448x65536.txt"}
    assert ctx.status() == 0
    if not args.no_cpu_baseline:
        res["cpu_baseline"] = analysis_cpu_baseline()
    return res


def run_jumpstart(xr, ctx, args, wc, ac):
    """Jump-start at scale: 2^24 xoshiro256++ streams J^i(s0) and L^i(s0) from
    SplitMix64(42), then 64 u64 outputs each; stream starts and fill timed
    with events on their stream (median of 3), then both pipelined over 16
    chunks on two streams, then fused in one kernel (xr_fill_streams).  A
    stream start is one 256 x 256 F2 matrix-vector product (three power-set
    levels)."""
    import torch
    c = W.CONFIG_JUMPSTART
    v, S, m = c["variant"], c["S"], c["m"]
    stream = torch.cuda.current_stream()
    base = ctx.empty_states(v, 1)
    ctx.seed(v, c["seed"], base)
    states = ctx.empty_states(v, S)
    out = ctx.empty_output(S * m, "u64")

    def timed(fn):
        fn()
        ts = []
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    # Pipelined: the streams in 16 chunks; the starts of chunk c+1 (side stream,
    # higher priority) overlap the fill of chunk c (main stream), through the
    # same public calls with first = c * S / 16.
    chunks = 16
    cs = S // chunks
    sb = len(states) // S
    side = torch.cuda.Stream(priority=-1)
    ready = [torch.cuda.Event() for _ in range(chunks)]

    def pipelined(kind):
        side.wait_stream(stream)
        for k in range(chunks):
            ctx.make_streams(v, kind, base, k * cs, cs, states[k * cs * sb:(k + 1) * cs * sb], stream=side)
            ready[k].record(side)
        for k in range(chunks):
            stream.wait_event(ready[k])
            ctx.fill(v, states[k * cs * sb:(k + 1) * cs * sb], cs, m, "u64", out[k * cs * m:(k + 1) * cs * m],
                     stream=stream)

    res = {"workload": "%s, %d streams x %d u64 outputs, SplitMix64(%d) base" % (v, S, m, c["seed"])}
    for kind in c["kinds"]:
        ms_streams = timed(lambda: ctx.make_streams(v, kind, base, 0, S, states))
        ms_fill = timed(lambda: ctx.fill(v, states, S, m, "u64", out))
        check = int(out.view(torch.int64).sum())
        ms_pipe = timed(lambda: pipelined(kind))
        same = int(out.view(torch.int64).sum()) == check
        out.zero_()
        ms_fused = timed(lambda: ctx.fill_streams(v, kind, base, 0, S, m, "u64", out))
        same_fused = int(out.view(torch.int64).sum()) == check
        res[kind] = {"streams_ms": ms_streams, "streams_per_s": S / (ms_streams / 1e3),
                     "fill_ms": ms_fill, "fill_gbs": S * m * 8 / (ms_fill / 1e3) / 1e9,
                     "fill_frac_of_measured_peak": S * m * 8 / (ms_fill / 1e3) / 1e9 / measured_peaks()[0]["hbm_gbs"],
                     "total_gbs": S * m * 8 / ((ms_streams + ms_fill) / 1e3) / 1e9,
                     "pipelined_ms": ms_pipe, "pipelined_gbs": S * m * 8 / (ms_pipe / 1e3) / 1e9,
                     "pipelined_chunks": chunks, "pipelined_same_output": same,
                     "fused_ms": ms_fused, "fused_gbs": S * m * 8 / (ms_fused / 1e3) / 1e9,
                     "fused_frac_of_measured_peak": S * m * 8 / (ms_fused / 1e3) / 1e9 / measured_peaks()[0]["hbm_gbs"],
                     "fused_same_output": same_fused,
                     "fused_roofline": fused_roofline(S, m, ms_fused, wc, ac)}
    del out, states
    torch.cuda.synchronize()
    assert ctx.status() == 0
    return res


def fused_roofline(S, m, ms, wc, ac):
    """The fused kernel's three bounds for S streams x m u64 outputs: output
    bytes at the measured write peak, its ALU lane operations at the measured
    ALU peak, and its shared-memory wavefronts at one per cycle per SM (max
    SM clock); the slowest binds."""
    import torch
    counts = recorded_fused_counts()
    hbm_ms = S * m * 8 / (wc["write_peak_gbs"] * 1e9) * 1e3
    res = {"hbm_ms": hbm_ms}
    if counts:
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        res["alu_ms"] = S * counts["alu_lane_ops_per_stream"] / ac["alu_lane_ops_per_s"] * 1e3
        res["l1_ms"] = S * counts["shared_wavefronts_per_stream"] / (sms * 2.07e9) * 1e3
        res.update(counts)
    bound = max((v, k[:-3]) for k, v in res.items() if k.endswith("_ms"))
    res.update(bound=bound[1], roofline_ms=bound[0], frac=bound[0] / ms,
               source="profiles/fill_streams__xoshiro256pp_2p21x64.txt" if counts else
               "counts not recorded for the current sources: HBM bound only")
    return res


def run_serving(xr, ctx, args):
    """Serving: 256 clients with device-resident states, Poisson arrivals at
    20k requests/s, sizes log-uniform in [2^10, 2^26] values, u64/f64, 16 GiB
    output budget; continuous batching against plain one-xr_fill_seq-per-request
    under the same trace.  Then the same requests all at once (saturation)."""
    import numpy as np
    c = W.CONFIG_SERVE
    names, seeds = W.serve_clients(c["nclients"])
    arr, cl, n, dt = W.serve_trace(args.serve_requests, **c)
    nbytes = float(sum(int(k) * (8 if d in ("u64", "f64") else 4) for k, d in zip(n, dt)))
    res = {"workload": "256 clients (xoshiro256** / xoroshiro128++), Poisson 20k req/s, sizes log-uniform "
                       "2^10..2^26, u64/f64, 16 GiB budget, %d requests (%.0f GB)" % (len(n), nbytes / 1e9)}
    warm = W.serve_trace(64, **dict(c, trace_seed=99))
    for mode in ("batched", "plain"):
        with xr.Server(ctx, names, seeds, arena_bytes=c["arena_bytes"], mode=mode) as srv:
            srv.replay(np.zeros(64), warm[1], warm[2], warm[3])
            lat, wall = srv.replay(arr, cl, n, dt)
            burst_lat, burst_wall = srv.replay(np.zeros(len(n) // 10), cl[: len(n) // 10], n[: len(n) // 10],
                                               dt[: len(n) // 10])
            st = srv.stats()
        bb = float(sum(int(k) * 8 for k in n[: len(n) // 10]))
        res[mode] = {"value": nbytes / (wall / 1e6) / 1e9, "unit": UNIT, "wall_ms": wall / 1e3,
                     "latency_us_p50": float(np.percentile(lat, 50)), "latency_us_p99": float(np.percentile(lat, 99)),
                     "saturation_value": bb / (burst_wall / 1e6) / 1e9,
                     "saturation_latency_us_p99": float(np.percentile(burst_lat, 99)),
                     "rounds": st["rounds"], "arena_peak_bytes": st["arena_peak"]}
    res["value"] = res["batched"]["value"]
    res["unit"] = UNIT
    res["saturation_frac_of_measured_peak"] = res["batched"]["saturation_value"] / measured_peaks()[0]["hbm_gbs"]
    res["batched_vs_plain_saturation"] = res["batched"]["saturation_value"] / res["plain"]["saturation_value"]
    return res


def run_e2e(ctx, args, first, bytes_per_step, world, dist):
    """The same step through xr_fill_host: each job's base state goes from host
    memory to the device, its outputs come back into one pinned host buffer;
    both copies are inside the timed region (wall clock around blocking calls)."""
    import torch
    c = W.CONFIG_BULK
    S, m, seed = c["S"], c["m"], c["seed"]
    host_base = {}
    for v, _ in jobs():
        if v not in host_base:
            t = ctx.empty_states(v, 1)
            ctx.seed(v, seed, t)
            host_base[v] = ctx.get_state(v, t)
    h_out = torch.empty(S * m * 8, dtype=torch.uint8).pin_memory()
    views = {d: h_out.view({"u64": torch.int64, "u32": torch.int32, "f64": torch.float64}[d])
             for d in ("u64", "u32", "f64")}

    def step():
        for v, d in jobs():
            ctx.fill_host(v, "jump", host_base[v], first, S, m, d, views[d])

    step()  # warm-up: staging buffers are allocated on first use
    link_before = d2h_link_gbs(h_out)
    times = []
    for _ in range(args.e2e_steps):
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step()
        torch.cuda.synchronize()
        times.append(max_over_ranks(time.perf_counter() - t0, dist, "cuda"))
    link_after = d2h_link_gbs(h_out)
    chunks = d2h_chunks_gbs(h_out)
    h2d = sum(len(host_base[v]) for v, _ in jobs())
    per_step = [world * bytes_per_step / t / 1e9 for t in times]
    value = statistics.median(per_step)
    link = statistics.median([link_before, link_after])
    return {"value": value, "unit": UNIT,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": bytes_per_step,
            "steps": args.e2e_steps, "ms_per_step": 1e3 * statistics.median(times),
            "per_step_gbs": per_step, "spread_gbs": [min(per_step), max(per_step)],
            "api": "xr_fill_host (pinned host output, two staging buffers, copy/compute overlap)",
            "bound": {"d2h_link_gbs": link, "d2h_link_before_after_gbs": [link_before, link_after],
                      "frac": value / world / link, "frac_spread": [min(per_step) / world / link,
                                                                    max(per_step) / world / link],
                      "d2h_per_gib_chunk_gbs": chunks,
                      "host_buffer_page_nodes": host_page_nodes(h_out),
                      "staging_chunk_bytes": 256 << 20,
                      "what": "device-to-pinned-host copy bandwidth of this GPU, 1 GiB copies timed with events, "
                              "before and after the end-to-end steps"}}


def host_page_nodes(t, samples=64):
    """NUMA node of `samples` pages spread over a host tensor (move_pages with
    no target nodes only reports where each page is): {node: count}."""
    import ctypes
    import platform
    nr = {"x86_64": 279, "aarch64": 239}.get(platform.machine())  # the move_pages system call
    if nr is None:
        return None
    try:
        libc = ctypes.CDLL(None, use_errno=True)
        page = os.sysconf("SC_PAGE_SIZE")
        base, nbytes = t.data_ptr(), t.numel() * t.element_size()
        addrs = [(base + k * (nbytes // samples)) // page * page for k in range(samples)]
        pages = (ctypes.c_void_p * samples)(*addrs)
        status = (ctypes.c_int * samples)()
        libc.syscall.restype = ctypes.c_long
        if libc.syscall(ctypes.c_long(nr), ctypes.c_int(0), ctypes.c_ulong(samples), pages, None, status,
                        ctypes.c_int(0)) != 0:
            return None
        hist = {}
        for st in status:
            hist[str(st)] = hist.get(str(st), 0) + 1
        return hist
    except (OSError, AttributeError):
        return None


def d2h_chunks_gbs(h_out, chunk=1 << 30):
    """Device-to-host copy rate into each 1 GiB piece of the pinned buffer
    (median of 3 each), to see whether the whole buffer sits behind the same
    link."""
    import torch
    src = torch.empty(chunk, dtype=torch.uint8, device="cuda")
    src.fill_(1)
    stream = torch.cuda.current_stream()
    res = []
    for off in range(0, h_out.numel() - chunk + 1, chunk):
        ts = []
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            h_out[off:off + chunk].copy_(src, non_blocking=True)
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        res.append(chunk / (statistics.median(ts) / 1e3) / 1e9)
    del src
    return res


def d2h_link_gbs(h_out):
    """The bound of any end-to-end number here: plain device-to-host copies of
    1 GiB into the same pinned buffer, median of 5, events on the stream."""
    import torch
    nb = min(1 << 30, h_out.numel())
    src = torch.empty(nb, dtype=torch.uint8, device="cuda")
    src.fill_(1)
    stream = torch.cuda.current_stream()
    h_out[:nb].copy_(src, non_blocking=True)
    ts = []
    for _ in range(5):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        h_out[:nb].copy_(src, non_blocking=True)
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    del src
    return nb / (statistics.median(ts) / 1e3) / 1e9


def run_profile(args):
    """A small case for ncu: one warm-up launch, then --profile-launches launches
    of the profiled kernel (fill: 2^16 streams x 2^10 outputs = 512 MiB of u64,
    larger than L2; streams: jump-start of --profile-streams streams; fused:
    xr_fill_streams of --profile-streams streams x 64 outputs)."""
    import torch
    import paper_1805_01407_gb300 as xr
    from paper_1805_01407_gb300 import build as libbuild
    libbuild.build()
    if args.profile == "batch":
        return run_profile_batch(args)
    if args.profile in ("lc", "lc-bulk"):
        return run_profile_lc(args)
    if args.profile == "fill-jobs":
        return run_profile_fill_jobs(args)
    v = args.profile_variant
    d = args.profile_dtype or W.native_dtype(v)
    S, m = args.profile_streams, W.CONFIG_BULK["m"]
    if args.profile == "fused":  # the jump-start shape: 64 outputs per stream
        m = W.CONFIG_JUMPSTART["m"]
    with xr.Context(0) as ctx:
        base = ctx.empty_states(v, 1)
        ctx.seed(v, W.CONFIG_BULK["seed"], base)
        if args.profile == "fused":
            out = ctx.empty_output(S * m, d)
            for _ in range(1 + args.profile_launches):
                ctx.fill_streams(v, "jump", base, 0, S, m, d, out)
            torch.cuda.synchronize()
            assert ctx.status() == 0
            print("profile case done: %s %s S=%d m=%d" % (args.profile, v, S, m))
            return 0
        states = ctx.empty_states(v, S)
        ctx.make_streams(v, "jump", base, 0, S, states)
        out = ctx.empty_output(S * m, d) if args.profile == "fill" else None
        for _ in range(1 + args.profile_launches):
            if args.profile == "fill":
                ctx.fill(v, states, S, m, d, out)
            else:
                ctx.make_streams(v, "jump", base, 0, S, states)
        torch.cuda.synchronize()
        assert ctx.status() == 0
    print("profile case done: %s %s S=%d m=%d" % (args.profile, v, S, m))
    return 0


def run_profile_fill_jobs(args):
    """One fill launch per generator and output type (every generator x
    {native word, f64}), --profile-streams streams x 2^10 outputs from
    SplitMix64(42) jump-started streams, in the order of W.ALL_VARIANTS: for
    ncu's per-launch instruction counts (ALU operations per value)."""
    import torch
    import paper_1805_01407_gb300 as xr
    S, m = args.profile_streams, W.CONFIG_BULK["m"]
    with xr.Context(0) as ctx:
        out = ctx.empty_output(S * m, "u64")
        order = []
        for v in W.ALL_VARIANTS:
            base = ctx.empty_states(v, 1)
            ctx.seed(v, W.CONFIG_BULK["seed"], base)
            states = ctx.empty_states(v, S)
            ctx.make_streams(v, "jump", base, 0, S, states)
            for d in (W.native_dtype(v), "f64"):
                ctx.fill(v, states, S, m, d, out.view(xr.torch_dtype(d)))
                order.append("%s %s" % (v, d))
        torch.cuda.synchronize()
        assert ctx.status() == 0
    print("profile case done: fill launches in order: " + ", ".join(order))
    return 0


def run_profile_lc(args):
    """Linear complexity for ncu: lc = the largest Table 13 row (one cluster
    of 8 CTAs), lc-bulk = the bulk configuration (448 CTAs); one warm-up
    call, then --profile-launches calls."""
    import torch
    import paper_1805_01407_gb300 as xr
    with xr.Context(0) as ctx:
        if args.profile == "lc":
            v, bit, N = ANALYSIS_LC_LARGE
            st = ctx.empty_states(v, 1)
            ctx.seed(v, 1, st)
            for _ in range(1 + args.profile_launches):
                L = ctx.linear_complexity(v, bit, N, st)
            what = "%s bit %d, %d bits: %d" % (v, bit, N, L)
        else:
            c = W.CONFIG_LC_BULK
            jobs = W.lc_bulk_jobs(**c)
            states = torch.zeros(len(jobs) * 128, dtype=torch.uint8, device="cuda")
            for j, (v, _, _) in enumerate(jobs):
                ctx.seed(v, c["seed"], states[j * 128:])
            for _ in range(1 + args.profile_launches):
                ctx.linear_complexity_many(jobs, states)
            what = "%d sequences x %d bits" % (len(jobs), c["N"])
        assert ctx.status() == 0
    print("profile case done: %s" % what)
    return 0


def run_profile_batch(args):
    """Batched configuration (max length --profile-max-len) run without a graph,
    one warm-up and --profile-launches timed-free runs, for ncu."""
    import torch
    import paper_1805_01407_gb300 as xr
    from paper_1805_01407_gb300 import build as libbuild
    libbuild.build()
    specs = W.batch_requests(nreq=W.CONFIG_BATCH["nreq"], max_len=args.profile_max_len,
                             mix_seed=W.CONFIG_BATCH["mix_seed"])
    with xr.Context(0) as ctx:
        reqs, offs, arena = xr.pack_requests([(v, dt, n, r) for r, (v, dt, n, _) in enumerate(specs)])
        b = xr.Batch(ctx, reqs)
        b.set_config(32, 128)
        slots = torch.zeros(len(specs) * 32, dtype=torch.uint8, device="cuda")
        out = torch.empty(arena, dtype=torch.uint8, device="cuda")
        seeds = torch.tensor([s for (_, _, _, s) in specs], dtype=torch.int64, device="cuda")
        for _ in range(1 + args.profile_launches):
            b.run(seeds, slots, out)
        torch.cuda.synchronize()
        assert ctx.status() == 0
        b.close()
    print("profile case done: batch of %d requests, %.2f GB" % (len(specs), arena / 1e9))
    return 0


if __name__ == "__main__":
    a = parse_args()
    if a.profile:
        sys.exit(run_profile(a))
    sys.exit(run_reference(a) if a.impl == "reference" else run_xr(a))
