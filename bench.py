#!/usr/bin/env python3
"""Benchmark of C-SAW biased neighbour selection on one GB300.

Default workload: weighted random walk (first order, with replacement) on an
RMAT scale-20 graph (edge factor 16, weights uniform in [1, 255]), one walker
per vertex, length 80, edge-weight bias.  Metric: sampled edges per second
(SEPS, C-SAW Sec. VI: sampled edges / kernel time; for walks one step is one
sampled edge).

One "step" is one csaw_walk call over all walkers.  Timing: W warm-up steps,
then K timed steps with CUDA events on the launching stream; L2 is flushed
(a 512 MiB write) before every timed step, outside the events.  `e2e` times
the same call through the C ABI with pinned host buffers (start vertices
copied in, the path matrix copied out) inside the timed region.

--impl reference times the oracle (single-threaded C on the host cores) on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SEPS (sampled edges per second)"
L2_FLUSH_BYTES = 512 << 20


def jdump(obj) -> str:
    """One JSON line; numpy scalars become Python numbers."""
    return json.dumps(obj, default=lambda o: o.item() if hasattr(o, "item") else str(o))


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def source_sha(kernel_src: str) -> str:
    """The kernel's source as compiled: its translation unit and the shared
    header every unit includes."""
    h = hashlib.sha256()
    for f in (kernel_src, "csaw_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2009_09103_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_records(kernel_src: str, workload: str):
    """The committed ncu DRAM records of this workload's kernels in one
    translation unit, if they were taken on its current source."""
    p = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    if not os.path.exists(p):
        return []
    with open(p) as f:
        recs = json.load(f)
    sha = source_sha(kernel_src)
    return [r for r in recs if r.get("source") == kernel_src and r.get("source_sha") == sha
            and r.get("workload") == workload]


def traffic_record(kernel_src: str, workload: str):
    """dram bytes per launch from the committed ncu summary, if it was taken
    on the current source of the kernel's translation unit and this workload."""
    recs = traffic_records(kernel_src, workload)
    return recs[0] if recs else None


def roofline_block(kernel, tr, ms, alg_bytes, sector_bytes=None):
    """DRAM-based roofline of one kernel.  achieved = the DRAM bytes of one
    launch (dram__bytes_read.sum + dram__bytes_write.sum from the ncu record
    taken on this kernel's current source and this workload) over the
    launch's CUDA-event time; peak = the measured HBM copy bandwidth.  The
    method's own bytes -- algorithmic, and counted in 32-byte sectors -- are
    reported beside it as L2-inclusive work: much of it is served by L2."""
    peak, peak_kind = measured_peaks()
    sec = ms / 1e3
    l2inc = {"algorithmic_bytes_per_launch": alg_bytes,
             "algorithmic_gbs": round(alg_bytes / sec / 1e9, 1),
             "algorithmic_over_hbm_peak": round(alg_bytes / sec / 1e9 / peak, 4)}
    if sector_bytes is not None:
        l2inc["sector_bytes_per_launch"] = sector_bytes
        l2inc["sector_over_hbm_peak"] = round(sector_bytes / sec / 1e9 / peak, 4)
    blk = {"bound": "hbm", "kernel": kernel, "peak": peak, "peak_source": peak_kind, "unit": "GB/s"}
    if tr:
        dram = tr["traffic_bytes_per_launch"]
        ach = dram / sec / 1e9
        blk.update({"achieved": round(ach, 1), "frac": round(ach / peak, 4), "traffic": dram,
                    "basis": "DRAM bytes per launch (ncu record of this kernel source) / event time"})
        if tr.get("l2_hit_rate_pct") is not None:
            blk["l2_hit_rate_pct"] = tr["l2_hit_rate_pct"]
        if tr.get("ncu_duration_ns"):
            blk["ncu_duration_ms"] = tr["ncu_duration_ns"] / 1e6
    else:
        blk.update({"achieved": None, "frac": None, "traffic": None,
                    "basis": "no DRAM record taken on the current kernel source"})
    blk["l2_inclusive"] = l2inc
    return blk


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def walk_bytes(torch, off_t, path):
    """Algorithmic bytes of one walk launch (edge-weight bias): per transition
    a->b: 16 (offsets of a) + 4*deg(a) (weights) + 4 (column of the pick); per
    walker 4 (start) and 4*(L+1) (its path row); per dead end 16 (offsets)."""
    p = path.to(torch.int64) & 0xFFFFFFFF
    a, b = p[:, :-1], p[:, 1:]
    real = b != 0xFFFFFFFF
    deg = (off_t[1:] - off_t[:-1])
    n_trans = int(real.sum())
    deg_sum = int(deg[a[real]].sum())
    n_dead = int(((~real) & (a != 0xFFFFFFFF)).sum())
    n, row = path.shape
    return n_trans, 16 * n_trans + 4 * deg_sum + 4 * n_trans + 4 * n + 4 * n * row + 16 * n_dead


def walk_sector_bytes(torch, off_t, path):
    """Sector-granular bytes of one edge-weight walk launch: the distinct
    32-byte sectors each unit must touch.  Per transition a->b: the sectors
    holding off[a] and off[a+1] (16 bytes from byte 8a), those spanned by a's
    weights w[off[a]:off[a+1]] and the one holding the picked column; per dead
    end the sectors of its offsets; per walker 4 (start) and its path row
    4*(L+1), written whole."""
    p = path.to(torch.int64) & 0xFFFFFFFF
    a, b = p[:, :-1], p[:, 1:]
    real = b != 0xFFFFFFFF
    av = a[real]
    beg, end = off_t[av], off_t[av + 1]
    off_sec = (8 * av + 15) // 32 - (8 * av) // 32 + 1
    w_sec = (4 * end - 1) // 32 - (4 * beg) // 32 + 1
    dead = a[(~real) & (a != 0xFFFFFFFF)]
    dead_sec = (8 * dead + 15) // 32 - (8 * dead) // 32 + 1
    n, row = path.shape
    return 32 * (int(off_sec.sum()) + int(w_sec.sum()) + int(av.numel()) + int(dead_sec.sum())) \
        + 4 * n + 4 * n * row


def node2vec_bytes(torch, off_t, path):
    """Algorithmic bytes of one node2vec walk launch: per transition a->b,
    16 (offsets of a) + 8*deg(a) (columns and weights of the row, both needed
    for the biases) and, from the second step on, 16 (offsets of the previous
    vertex t) + 4*deg(t) (its sorted list, read once by the merge that tests
    membership); per walker 4 (start) and 4*(L+1) (its path row); per dead
    end 16 (offsets)."""
    p = path.to(torch.int64) & 0xFFFFFFFF
    a, b = p[:, :-1], p[:, 1:]
    real = b != 0xFFFFFFFF
    deg = (off_t[1:] - off_t[:-1])
    n_trans = int(real.sum())
    deg_sum = int(deg[a[real]].sum())
    with_prev = real[:, 1:]                    # transitions taken at step t >= 1
    prev = p[:, :-2][with_prev]
    n_prev = int(with_prev.sum())
    prev_sum = int(deg[prev].sum())
    n_dead = int(((~real) & (a != 0xFFFFFFFF)).sum())
    n, row = path.shape
    return n_trans, (16 * n_trans + 8 * deg_sum + 16 * n_prev + 4 * prev_sum
                     + 4 * n + 4 * n * row + 16 * n_dead)


def cached_walk_bytes(torch, off_t, path, length):
    """Algorithmic bytes of one walk launch over the cumulative array's
    search aids: per step 32 (the vertex record) + 8 per s2 probe
    (ceil(log2(G + 1)) over the row's G = (end-1)/64 - beg/64 entries) + 32
    (one half of the s1 run) + 32 (the 8-edge group: its weights, or one half
    of its leaf entries) + 4 (picked column) + 4 (path entry); per walker 4
    (start) and 4 * (L + 1) (its path row)."""
    p = path.to(torch.int64) & 0xFFFFFFFF
    a, b = p[:, :-1], p[:, 1:]
    real = b != 0xFFFFFFFF
    n_trans = int(real.sum())
    av = a[real]
    beg, end = off_t[av], off_t[av + 1]
    G = ((end - 1) >> 6) - (beg >> 6)
    probes = int(torch.ceil(torch.log2((G + 1).to(torch.float64))).sum())
    n = path.shape[0]
    return (32 + 32 + 32 + 4 + 4) * n_trans + 8 * probes + 4 * n + 4 * n * (length + 1)


def walk_workload(args):
    from paper_2009_09103_gb300 import inputs
    if args.workload == "node2vec":
        if args.scale == 22:
            return inputs.workload_node2vec_s22()
        g = inputs.rmat_csr(args.scale, 32, 15, args.scale)
        return inputs.WalkWorkload(g, np.arange(g.V, dtype=np.uint32), 40, "node2vec", (1, 2, 4), 3)
    if args.scale == 20:
        return inputs.workload_walk_s20()
    g = inputs.rmat_csr(args.scale, 16, 255, args.scale)
    return inputs.WalkWorkload(g, np.arange(g.V, dtype=np.uint32), 80, "edge_weight", (1, 1, 1), 2)


def walk_config(args, wl):
    g = wl.graph
    if wl.bias == "node2vec":
        return (f"node2vec walk p=2 q=0.5 (integer multipliers 1/2/4): RMAT scale {args.scale}, edge factor "
                f"32, weights uniform [1,15], {g.V:,} walkers (one per vertex), length {wl.length}")
    return (f"weighted random walk: RMAT scale {args.scale}, edge factor 16, weights uniform [1,255], "
            f"{g.V:,} walkers (one per vertex), length {wl.length}, edge-weight bias")


def walk_mode(args, wl):
    """How the main line's walk gets its cumulative bias arrays: "build" (a
    static bias: the call builds the array over all rows, then every step is a
    search of it -- the array's construction is inside every timed step),
    "cached" (--cdf: built once per graph, before timing) or "streaming"
    (--streaming, or node2vec's dynamic bias: every step streams its row)."""
    if args.cdf:
        return "cached"
    if args.streaming or wl.bias == "node2vec":
        return "streaming"
    return "build"


def time_steps(torch, fn, steps, warmup, stream, flush):
    """CUDA-event times (ms) of `steps` calls of fn on `stream` after
    `warmup` untimed ones, with L2 flushed before each."""
    for _ in range(warmup):
        fn()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for i in range(steps):
        flush.fill_(i)
        evs[i][0].record(stream)
        fn()
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def run_walk_bench(args, rank, world):
    import torch
    from paper_2009_09103_gb300 import build, csaw, inputs

    build.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    t0 = time.time()
    wl = walk_workload(args)
    g = wl.graph
    mode = walk_mode(args, wl)
    log(f"[bench] {args.workload} graph: V={g.V} E={g.E} built in {time.time() - t0:.1f}s; mode {mode}")
    G = csaw.Graph(g.off, g.col, g.w)
    if mode == "cached":
        # node2vec reads the edge weights' cumulative array (intersection path)
        G.build_cdf("edge_weight" if wl.bias == "node2vec" else wl.bias)
    stream = torch.cuda.current_stream()
    starts = torch.from_numpy(wl.starts.view(np.int32)).to(dev)
    n = starts.numel()
    path = torch.empty((n, wl.length + 1), dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    seed = wl.rng_seed + rank  # replicas: independent walks per rank
    per_call = mode == "build"

    def step():
        csaw.walk(G, starts, wl.length, wl.bias, seed, wl.n2v_mult, path=path, stream=stream, build_cdf=per_call)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    off_t = torch.from_numpy(g.off.astype(np.int64)).to(dev)
    n_trans, alg_bytes = (node2vec_bytes if wl.bias == "node2vec" else walk_bytes)(torch, off_t, path)
    sector_bytes = walk_sector_bytes(torch, off_t, path) if wl.bias == "edge_weight" else None

    clocks = Clocks(dev.index)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for i in range(args.steps):
        flush.fill_(i)
        evs[i][0].record(stream)
        step()
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    times_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = sum(times_ms)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = n_trans * args.steps * world / (total_ms / 1e3)

    # end to end through the C ABI with pinned host buffers
    h_starts = torch.empty(n, dtype=torch.int32, pin_memory=True)
    h_starts.copy_(starts.cpu())
    h_path = torch.empty((n, wl.length + 1), dtype=torch.int32, pin_memory=True)
    hs = h_starts.numpy().view(np.uint32)
    hp = h_path.numpy().view(np.uint32)

    def e2e_call():
        csaw.walk(G, hs, wl.length, wl.bias, seed, wl.n2v_mult, path=hp, stream=stream, build_cdf=per_call)

    e2e_call()   # warm
    e2e_steps = max(1, min(args.steps, 5))
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_call()
    e2e_s = (time.perf_counter() - t1) / e2e_steps
    e2e_ok = bool(np.array_equal(hp, path.cpu().numpy().view(np.uint32)))
    e2e = {"value": n_trans * world / e2e_s, "unit": "edges/s",
           "h2d_bytes_per_step": 4 * n, "d2h_bytes_per_step": 4 * n * (wl.length + 1),
           "matches_device_run": e2e_ok}

    wl_name = f"{args.workload}_s{args.scale}"
    kernels = {}
    if mode == "streaming":
        kname = "walk_kernel<NODE2VEC>" if wl.bias == "node2vec" else "walk_kernel<EDGE_WEIGHT>"
        roofline = roofline_block(kname, traffic_record("csaw_walk.cu", wl_name), ms_per_step, alg_bytes,
                                  sector_bytes)
    elif wl.bias == "node2vec":
        roofline = roofline_block("walk_kernel<NODE2VEC>", traffic_record("csaw_walk.cu", wl_name + "_cdf"),
                                  ms_per_step, alg_bytes)
    else:
        # the step's phases timed by CUDA events on the step's stream inside
        # the call (the array's construction, then the walk kernels); the
        # paths checked against the graph's prebuilt array
        cb = cached_walk_bytes(torch, off_t, path, wl.length)
        ms_walk = ms_per_step
        if mode == "build":
            ph = []
            for i in range(args.steps):
                flush.fill_(i)
                p_ms = [0.0, 0.0]
                csaw.walk(G, starts, wl.length, wl.bias, seed, wl.n2v_mult, path=path, stream=stream, build_cdf=True,
                          phase_ms=p_ms)
                ph.append(p_ms)
            ms_build = float(np.mean([x[0] for x in ph]))
            ms_walk = float(np.mean([x[1] for x in ph]))
            G.build_cdf(wl.bias)
            path2 = torch.empty_like(path)
            csaw.walk(G, starts, wl.length, wl.bias, seed, wl.n2v_mult, path=path2, stream=stream)
            torch.cuda.synchronize()
            same = bool(torch.equal(path, path2))
            G.drop_cdf(wl.bias)
            kernels = {"walk_cached_kernel_ms": ms_walk,
                       "cumulative_array_build_ms": ms_build,
                       "basis": "CUDA events on the step's stream around each phase inside the call (phase_ms)",
                       "build_algorithmic_bytes": 4 * g.E + 9 * g.E // 8 + 40 * g.V,
                       "identical_paths_graph_array": same}
            recs = traffic_records("csaw_graph.cu", wl_name + "_build")
            if recs and ms_build > 0:
                peak, peak_kind = measured_peaks()
                dram = sum(r["traffic_bytes_per_launch"] for r in recs)
                kernels["build_dram_bytes"] = dram
                kernels["build_dram_gbs"] = round(dram / (ms_build / 1e3) / 1e9, 1)
                kernels["build_dram_frac"] = round(dram / (ms_build / 1e3) / 1e9 / peak, 4)
                kernels["build_kernels"] = sorted(r["kernel"] for r in recs)
        kn = "walk_cached_kernel<WEIGHTS>" if mode == "build" else "walk_cached_kernel<LEAF>"
        roofline = roofline_block(kn, traffic_record("csaw_walk_cdf.cu", wl_name + ("_build" if mode == "build" else "_cdf")),
                                  ms_walk, cb)
    cum = {"build": "built over all rows inside every step (segmented scan over edge tiles into summaries of the "
                    "prefix sums and per-vertex records; each step bisects the summaries and sums one 32-byte "
                    "group of weights)",
           "cached": "cached per edge (built once per graph, before timing)",
           "streaming": "computed per step (streamed over the row)"}[mode]
    result = {
        "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32 biases / u64 prefix sums", "data": "synthetic (seeded RMAT)",
        "config": {"workload": walk_config(args, wl),
                   "parallelism": "replicas" if world > 1 else "1 GPU",
                   "l2": "flushed (512 MiB write) before every timed step",
                   "cumulative_array": cum,
                   "sampled_edges_per_step": n_trans},
        "gpu_launches": args.steps * (4 if mode == "build" else 1),
        "roofline": roofline,
        "e2e": e2e,
    }
    if kernels:
        result["kernels"] = kernels
    if clk:
        result["clocks"] = clk
    if mode == "build" and not args.no_variant:
        # The per-visit streaming walk (each step streams its row's biases):
        # the same paths, timed the same way.
        path3 = torch.empty_like(path)
        t_s = time_steps(torch, lambda: csaw.walk(G, starts, wl.length, wl.bias, seed, wl.n2v_mult,
                                                  path=path3, stream=stream),
                         args.steps, args.warmup, stream, flush)
        ms3 = sum(t_s) / len(t_s)
        result["streaming_per_visit"] = {
            "value": n_trans * world / (ms3 / 1e3), "unit": "edges/s", "ms_per_step": ms3,
            "kernel": "walk_kernel", "identical_paths": bool(torch.equal(path, path3)),
            "roofline": roofline_block("walk_kernel<EDGE_WEIGHT>", traffic_record("csaw_walk.cu", wl_name), ms3,
                                       alg_bytes, sector_bytes)}
        result["gpu_launches_streaming"] = args.steps
    G.close()
    return result, (g, wl, n_trans)


def oracle_walk_sample(g, wl, budget_s: float):
    """Time the oracle on walker subsets until about budget_s of CPU work."""
    import oracle
    oracle.build()
    n = len(wl.starts)
    # uniformly spaced walkers: the same mix of start degrees as the full run
    m = 256
    total_t, total_e, used = 0.0, 0, 0
    while total_t < budget_s and used < n:
        ids = np.linspace(0, n - 1, num=m, dtype=np.int64) + used % 7
        ids = np.unique(np.clip(ids, 0, n - 1))
        t0 = time.perf_counter()
        p = oracle.walk(g, wl.starts[ids], wl.length, wl.bias, wl.rng_seed, mult=wl.n2v_mult,
                        walker_ids=ids.astype(np.uint64))
        total_t += time.perf_counter() - t0
        total_e += int((p[:, 1:] != 0xFFFFFFFF).sum())
        used += len(ids)
        m = min(4 * m, 65536)
    return total_e / total_t, used, total_t


def oracle_walk_all_cores(g, wl, budget_s: float, threads: int):
    """The single-threaded oracle run as `threads` concurrent copies over
    disjoint walker shards (ctypes releases the GIL during each call)."""
    import concurrent.futures as cf
    import oracle
    oracle.build()
    n = len(wl.starts)

    def shard(t):
        done_e, used, t0 = 0, 0, time.perf_counter()
        m = 64
        while time.perf_counter() - t0 < budget_s:
            ids = (np.arange(m, dtype=np.int64) * threads + t + used * threads) % n
            p = oracle.walk(g, wl.starts[ids], wl.length, wl.bias, wl.rng_seed, mult=wl.n2v_mult,
                            walker_ids=ids.astype(np.uint64))
            done_e += int((p[:, 1:] != 0xFFFFFFFF).sum())
            used += m
            m = min(2 * m, 4096)
        return done_e, used
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        res = list(ex.map(shard, range(threads)))
    wall = time.perf_counter() - t0
    edges = sum(r[0] for r in res)
    return edges / wall, sum(r[1] for r in res), wall


def run_reference(args, rank, world):
    """The oracle, as it stands, on the host cores, on bounded samples."""
    if rank != 0:
        return None
    wl = walk_workload(args)
    g = wl.graph
    per_step = args.ref_seconds or max(2.0, min(20.0, 60.0 / max(1, args.steps)))
    vals = []
    used_total = 0
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle_walk_all_cores(g, wl, 0.3, cores)
    for _ in range(args.steps):
        v, used, _ = oracle_walk_all_cores(g, wl, per_step, cores)
        vals.append(v)
        used_total += used
    value = statistics.mean(vals)
    sample = (f"{used_total // max(1, args.steps)} walkers per step in {cores} disjoint shards (one "
              f"copy of the single-threaded oracle per core), full length {wl.length}")
    return {
        "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32 biases / u64 prefix sums", "data": "synthetic (seeded RMAT)",
        "impl": "reference",
        "config": {"workload": walk_config(args, wl)},
        "cpu_baseline": {"value": value, "unit": "edges/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


# --------------------------------------------------------------------------
# Batched sampling (config: RMAT s24, 4096 instances): C-SAW's layered
# neighbour sampling as one batched plan replayed as a CUDA graph, against one
# plain csaw_sample call per instance; SEPS = sampled edges / GPU time.

def sample_frontier_bytes(res, g, fanout, bias):
    """Algorithmic bytes of the selection kernels of one run: per frontier
    vertex v of degree d, 16 (offsets) + 4d (weights, or columns) + 4d
    (degree gathers, neighbour-degree bias) + 8 per pick (edge written)."""
    deg = np.diff(g.off).astype(np.int64)
    n_inst = res.n_instances
    total = 0
    for lvl in range(res.depth):
        a, b = int(res.edge_offsets[lvl * n_inst]), int(res.edge_offsets[(lvl + 1) * n_inst])
        src = res.src[a:b]
        # distinct (instance, source) pairs are the frontier vertices that emitted edges
        inst = np.repeat(np.arange(n_inst), np.diff(res.edge_offsets[lvl * n_inst:(lvl + 1) * n_inst + 1]).astype(np.int64))
        key = (inst.astype(np.int64) << 32) | src.astype(np.int64)
        first = np.ones(len(key), dtype=bool)
        first[1:] = key[1:] != key[:-1]
        d = deg[src[first].astype(np.int64)]
        per_row = 4 * d * (2 if bias == "neighbor_degree" else 1)
        total += int((16 + per_row).sum()) + 8 * (b - a)
    return total


def time_gpu(torch, fn, reps=1, flush=None):
    """Mean ms of fn() over reps, CUDA events on the current stream; with
    flush, a buffer larger than L2 is written before each rep (outside the
    events)."""
    st = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    torch.cuda.synchronize()
    for i in range(reps):
        if flush is not None:
            flush.fill_(i)
        evs[i][0].record(st)
        fn()
        evs[i][1].record(st)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs) / reps


BATCHED_DESC = ("batched layered sampling: RMAT scale 24, edge factor 16, 4096 instances of log-uniform "
                "[64,8192) distinct seeds, depth 2, fanout [25,10], neighbour-degree bias")


def batched_leg(torch, csaw, wl, G, cdf, steps, warmup, plain_instances, flush):
    """The batched plan (one CUDA graph over all instances and layers) against
    one plain csaw_sample call per instance (each alone at its own index) on
    the same graph; returns SEPS and times of both."""
    if cdf:
        G.build_cdf(wl.bias)
    n_inst = len(wl.inst_offsets) - 1
    plan = csaw.SamplePlan(G, n_inst, len(wl.seeds), wl.fanout, wl.bias)
    ds = torch.from_numpy(wl.seeds.view(np.int32)).cuda()
    dio = torch.from_numpy(wl.inst_offsets.view(np.int64)).cuda()
    for _ in range(warmup):
        plan.run(ds, dio, wl.rng_seed)
    ms_plan = time_gpu(torch, lambda: plan.run(ds, dio, wl.rng_seed), steps, flush)
    res = plan.result()
    info = plan.info()
    plan.close()
    edges = int(res.n_edges)
    n_plain = min(n_inst, plain_instances)
    pick = np.unique(np.linspace(0, n_inst - 1, n_plain).astype(np.int64))
    calls = []
    for i in pick:
        sub = np.zeros(n_inst + 1, dtype=np.uint64)
        sub[i + 1:] = wl.inst_offsets[i + 1] - wl.inst_offsets[i]
        calls.append((wl.seeds[wl.inst_offsets[i]:wl.inst_offsets[i + 1]].copy(), sub))

    def plain():
        for s_, io_ in calls:
            csaw.sample(G, s_, io_, wl.fanout, wl.bias, wl.rng_seed, to_host=False)
    plain_edges = sum(int(res.edge_offsets[l * n_inst + i + 1] - res.edge_offsets[l * n_inst + i])
                      for i in pick for l in range(len(wl.fanout)))
    if calls:   # warm-up call: the allocator pool and the kernels' first use
        csaw.sample(G, calls[0][0], calls[0][1], wl.fanout, wl.bias, wl.rng_seed, to_host=False)
    ms_plain = time_gpu(torch, plain, 1, flush)
    if cdf:
        G.drop_cdf(wl.bias)
    seps_b = edges / (ms_plan / 1e3)
    seps_p = plain_edges / (ms_plain / 1e3) if plain_edges and ms_plain > 0 else None
    return res, {
        "batched_plan": {"ms_per_run": ms_plan, "seps": seps_b, "sampled_edges": edges, "runs_timed": steps,
                         "select_blocks": info["select_blocks"], "theta_warp": info["theta_warp"],
                         "plan_device_bytes": info["device_bytes"]},
        "plain_one_call_per_instance": {
            "instances_timed": int(len(pick)), "instances_total": n_inst,
            "subset": "all instances" if len(pick) == n_inst else
                      f"{len(pick)} instances uniformly spaced over the {n_inst}",
            "ms": ms_plain, "sampled_edges": plain_edges, "seps": seps_p,
            "timing": "one csaw_sample call per instance (host seeds in, edges left on the device), "
                      "CUDA events around the whole sequence"},
        "batched_over_plain_seps": seps_b / seps_p if seps_p else None,
    }


def batched_workload(args, inputs):
    if args.workload == "sample_s12":
        wl = inputs.workload_sample_s12()
        desc = ("layered biased neighbour sampling: RMAT scale 12, edge factor 16, weights uniform "
                "[1,100], 256 uniform seeds as one instance, depth 2, fanout [10,5], edge-weight bias")
    elif args.scale in (None, 24) and args.instances == 4096:
        wl, desc = inputs.workload_batched_s24(), BATCHED_DESC
    else:
        g0 = inputs.rmat_csr(args.scale, 16, 255, args.scale)
        sizes = inputs.loguniform_sizes(args.instances, 6.0, 7.0, args.scale, stream=4)
        sd, io = inputs.distinct_seeds(sizes, g0.V, args.scale, stream=4)
        wl = inputs.SampleWorkload(g0, sd, io, [25, 10], "neighbor_degree", 4)
        desc = (f"batched layered sampling: RMAT scale {args.scale}, edge factor 16, {args.instances} instances "
                "of log-uniform [64,8192) distinct seeds, depth 2, fanout [25,10], neighbour-degree bias")
    return wl, desc


def batched_block(args):
    """Both forms of the batched comparison (streamed and cached cumulative
    arrays) on the RMAT s24 workload; the block the default run carries."""
    import torch
    from paper_2009_09103_gb300 import csaw, inputs
    t0 = time.time()
    wl, desc = inputs.workload_batched_s24(), BATCHED_DESC
    g = wl.graph
    log(f"[bench] batched: V={g.V} E={g.E} seeds={len(wl.seeds)} built in {time.time() - t0:.1f}s")
    G = csaw.Graph(g.off, g.col, g.w)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    res, streamed = batched_leg(torch, csaw, wl, G, False, args.batched_steps, 1, args.plain_instances, flush)
    _, cached = batched_leg(torch, csaw, wl, G, True, args.batched_steps, 1, args.plain_instances, flush)
    clk = clocks.stop()
    G.close()
    alg = sample_frontier_bytes(res, g, wl.fanout, wl.bias)
    out = {"workload": desc, "sampled_edges_per_run": int(res.n_edges),
           "l2": "flushed (512 MiB write) before every timed run",
           "streamed_cumulative_array": streamed, "cached_cumulative_array": cached,
           "selection_algorithmic_bytes_per_run": alg,
           "selection_algorithmic_gbs_streamed": alg / (streamed["batched_plan"]["ms_per_run"] / 1e3) / 1e9}
    # the plan's kernels run inside one CUDA graph, so their DRAM rates come
    # from the ncu record alone (bytes over ncu's serialised kernel time)
    peak, peak_kind = measured_peaks()
    kd = []
    for r in traffic_records("csaw_sample.cu", "batched_s24"):
        gbs = r["traffic_bytes_per_launch"] / (r["ncu_duration_ns"] / 1e9) / 1e9
        kd.append({"kernel": r["kernel"], "dram_bytes_per_launch": r["traffic_bytes_per_launch"],
                   "ncu_ms_per_launch": r["ncu_duration_ns"] / 1e6, "dram_gbs": round(gbs, 1),
                   "frac_of_hbm_peak": round(gbs / peak, 4), "peak_gbs": peak, "peak_source": peak_kind})
    if kd:
        out["kernels_dram_streamed"] = kd
    if clk:
        out["clocks"] = clk
    return out


def run_sample_bench(args):
    import torch
    from paper_2009_09103_gb300 import build, csaw, inputs
    build.build()
    torch.cuda.set_device(0)
    t0 = time.time()
    wl, desc = batched_workload(args, inputs)
    g = wl.graph
    log(f"[bench] {args.workload}: V={g.V} E={g.E} seeds={len(wl.seeds)} built in {time.time() - t0:.1f}s")
    G = csaw.Graph(g.off, g.col, g.w)
    if args.autotune:
        tuning = csaw.autotune_select(G, wl.seeds, wl.inst_offsets, wl.fanout, wl.bias, wl.rng_seed)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    ref = csaw.sample(G, wl.seeds, wl.inst_offsets, wl.fanout, wl.bias, wl.rng_seed)
    res, legs = batched_leg(torch, csaw, wl, G, args.cdf, args.steps, args.warmup, args.plain_instances, flush)
    plan_ok = bool(np.array_equal(res.dst, ref.dst) and np.array_equal(res.edge_offsets, ref.edge_offsets))
    ms_call = time_gpu(torch, lambda: csaw.sample(G, wl.seeds, wl.inst_offsets, wl.fanout, wl.bias,
                                                  wl.rng_seed, to_host=False), args.steps, flush)
    edges = int(ref.n_edges)
    alg = sample_frontier_bytes(ref, g, wl.fanout, wl.bias)
    peak, peak_kind = measured_peaks()
    ms_plan = legs["batched_plan"]["ms_per_run"]
    out = {
        "metric": METRIC, "value": edges / (ms_plan / 1e3), "unit": "edges/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_plan, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32 biases / u64 prefix sums",
        "data": "synthetic (seeded RMAT)",
        "config": {"workload": desc, "sampled_edges_per_step": edges, "instances": len(wl.inst_offsets) - 1,
                   "cumulative_array": "cached per edge" if args.cdf else "computed per selection",
                   "l2": "flushed (512 MiB write) before every timed run"},
        **legs,
        "plan_matches_sample": plan_ok,
        "batched_call": {"ms": ms_call, "seps": edges / (ms_call / 1e3)},
        "selection_bytes_per_run": alg,
        "gbs_over_whole_run": alg / (ms_plan / 1e3) / 1e9, "peak_gbs": peak, "peak_source": peak_kind,
    }
    if args.autotune:
        out["tuning"] = tuning
    G.close()
    if args.cpu_baseline_seconds > 0:
        import oracle
        oracle.build()
        n_inst = len(wl.inst_offsets) - 1
        done, used, t_used = 0, 0, 0.0
        for i in np.argsort(np.diff(wl.inst_offsets).astype(np.int64), kind="stable"):
            sub = np.zeros(n_inst + 1, dtype=np.uint64)
            sub[i + 1:] = wl.inst_offsets[i + 1] - wl.inst_offsets[i]
            t = time.perf_counter()
            r = oracle.sample(g, wl.seeds[wl.inst_offsets[i]:wl.inst_offsets[i + 1]], sub, wl.fanout, wl.bias,
                              wl.rng_seed)
            t_used += time.perf_counter() - t
            done += int(r["edge_off"][-1])
            used += 1
            if t_used > args.cpu_baseline_seconds:
                break
        out["cpu_baseline"] = {"value": done / t_used, "unit": "edges/s", "cores": 1, "kind": "oracle",
                               "sample": f"{used} instances (smallest first), full depth, {t_used:.1f} s"}
    return out


# --------------------------------------------------------------------------
# Multi-dimensional random walk (frontier sampling), not the default line.

def run_mdrw_bench(args):
    import torch
    from paper_2009_09103_gb300 import build, csaw, inputs
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    t0 = time.time()
    wl = inputs.workload_mdrw_s20()
    g = wl.graph
    n, m = wl.pools.shape
    log(f"[bench] mdrw graph: V={g.V} E={g.E} pools {n}x{m} built in {time.time() - t0:.1f}s")
    G = csaw.Graph(g.off, g.col, g.w)
    stream = torch.cuda.current_stream()
    pools = torch.from_numpy(wl.pools.view(np.int32)).to(dev)
    src = torch.empty((n, wl.steps), dtype=torch.int32, device=dev)
    dst = torch.empty_like(src)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    def step():
        csaw.mdrw(G, pools, wl.steps, wl.rng_seed, src=src, dst=dst, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    n_edges = int((src != -1).sum())
    clocks = Clocks(dev.index)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    torch.cuda.synchronize()
    clocks.start()
    for i in range(args.steps):
        flush.fill_(i)
        evs[i][0].record(stream)
        step()
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    # end to end through the C ABI with pinned host buffers (copies inside the call)
    h_pools = torch.empty((n, m), dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
    h_pools[:] = wl.pools
    h_src = torch.empty((n, wl.steps), dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
    h_dst = torch.empty((n, wl.steps), dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
    csaw.mdrw(G, h_pools, wl.steps, wl.rng_seed, src=h_src, dst=h_dst)
    t1 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 3))
    for _ in range(e2e_steps):
        csaw.mdrw(G, h_pools, wl.steps, wl.rng_seed, src=h_src, dst=h_dst)
    e2e_s = (time.perf_counter() - t1) / e2e_steps
    same = bool(np.array_equal(h_src, src.cpu().numpy().view(np.uint32)) and
                np.array_equal(h_dst, dst.cpu().numpy().view(np.uint32)))
    G.close()
    # per step: 16 (offsets of v) + 4 (the picked column) + 4 (degree of u) +
    # 8 (the sampled edge); per instance: 4 per pool slot read
    alg = 32 * n_edges + 4 * n * m
    tr = traffic_record("csaw_mdrw.cu", "mdrw_s20")
    res = {
        "metric": METRIC, "value": n_edges / (ms / 1e3), "unit": "edges/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32 degrees / u64 prefix sums",
        "data": "synthetic (seeded RMAT)",
        "config": {"workload": f"multi-dimensional random walk: RMAT scale 20, edge factor 16, {n} instances, "
                               f"pools of {m} vertices with edges (uniform), {wl.steps} steps; VertexBias = "
                               "degree, EdgeBias = 1",
                   "l2": "flushed (512 MiB write) before every timed step", "sampled_edges_per_step": n_edges},
        "gpu_launches": args.steps,
        "roofline": roofline_block("mdrw_kernel", tr, ms, alg),
        "e2e": {"value": n_edges / e2e_s, "unit": "edges/s", "h2d_bytes_per_step": 4 * n * m,
                "d2h_bytes_per_step": 8 * n * wl.steps, "matches_device_run": same},
    }
    if clk:
        res["clocks"] = clk
    if args.cpu_baseline_seconds > 0:
        import oracle
        oracle.build()
        done, used, t_used = 0, 0, 0.0
        for i in np.linspace(0, n - 1, n).astype(np.int64):
            t = time.perf_counter()
            rs, _ = oracle.mdrw(g, wl.pools[i:i + 1], wl.steps, wl.rng_seed,
                                instance_ids=np.array([i], dtype=np.uint64))
            t_used += time.perf_counter() - t
            done += int((rs != 0xFFFFFFFF).sum())
            used += 1
            if t_used > args.cpu_baseline_seconds:
                break
        res["cpu_baseline"] = {"value": done / t_used, "unit": "edges/s", "cores": 1, "kind": "oracle",
                               "sample": f"{used} instances in order, all {wl.steps} steps, {t_used:.1f} s"}
    return res


# --------------------------------------------------------------------------
# Layer sampling, not the default line.

def run_layer_bench(args):
    import torch
    from paper_2009_09103_gb300 import build, csaw, inputs
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    t0 = time.time()
    wl = inputs.workload_layer_s20()
    g = wl.graph
    n_inst = len(wl.inst_offsets) - 1
    log(f"[bench] layer graph: V={g.V} E={g.E} instances={n_inst} built in {time.time() - t0:.1f}s")
    G = csaw.Graph(g.off, g.col, g.w)
    if args.cdf:
        G.build_cdf(wl.bias)
    ds = torch.from_numpy(wl.seeds.view(np.int32)).to(dev)
    dio = torch.from_numpy(wl.inst_offsets.view(np.int64)).to(dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    def step():
        return csaw.layer_sample(G, ds, dio, wl.fanout, wl.bias, wl.rng_seed, stream=stream, to_host=False)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(dev.index)
    clocks.start()
    evs = []
    for i in range(args.steps):
        flush.fill_(i)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = step()
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    edges = int(res.n_edges)
    # end to end: host seeds in, edges copied out, through the C ABI
    t1 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 3))
    for _ in range(e2e_steps):
        ref = csaw.layer_sample(G, wl.seeds, wl.inst_offsets, wl.fanout, wl.bias, wl.rng_seed)
    e2e_s = (time.perf_counter() - t1) / e2e_steps
    G.close()
    # per frontier vertex: 16 (offsets) + 4 per pool entry (its bias, read
    # for the totals); per pick: 8 (the sampled edge).  Frontiers follow
    # Update: the next one is the new picked vertices.
    deg = np.diff(g.off).astype(np.int64)
    front = [np.unique(wl.seeds[int(wl.inst_offsets[i]):int(wl.inst_offsets[i + 1])]) for i in range(n_inst)]
    visited = [set(f.tolist()) for f in front]
    eo = ref.edge_offsets.astype(np.int64)
    alg = 8 * edges
    for l in range(len(wl.fanout)):
        alg += sum(16 * len(f) + 4 * int(deg[f.astype(np.int64)].sum()) for f in front)
        nxt = []
        for i in range(n_inst):
            new = sorted(set(ref.dst[eo[l * n_inst + i]:eo[l * n_inst + i + 1]].tolist()) - visited[i])
            visited[i].update(new)
            nxt.append(np.array(new, dtype=np.int64))
        front = nxt
    tr = traffic_record("csaw_sample.cu", "layer_s20" + ("_cdf" if args.cdf else ""))
    out = {
        "metric": METRIC, "value": edges / (ms / 1e3), "unit": "edges/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32 biases / u64 prefix sums",
        "data": "synthetic (seeded RMAT)",
        "config": {"workload": f"layer sampling: RMAT scale 20, edge factor 16, {n_inst} instances of 64 seeds, "
                               f"depth 2, {wl.fanout} picks per instance and layer, edge-weight bias",
                   "l2": "flushed (512 MiB write) before every timed step", "sampled_edges_per_step": edges,
                   "cumulative_array": "cached per edge" if args.cdf else "computed per selection"},
        "roofline": roofline_block("layer_select_kernel", tr, ms, alg),
        "e2e": {"value": edges / e2e_s, "unit": "edges/s", "h2d_bytes_per_step": 4 * len(wl.seeds) + 8 * (n_inst + 1),
                "d2h_bytes_per_step": 8 * edges},
    }
    if clk:
        out["clocks"] = clk
    if args.cpu_baseline_seconds > 0:
        import oracle
        oracle.build()
        done, used, t_used = 0, 0, 0.0
        for i in range(n_inst):
            sub = np.zeros(n_inst + 1, dtype=np.uint64)
            sub[i + 1:] = wl.inst_offsets[i + 1] - wl.inst_offsets[i]
            t = time.perf_counter()
            r = oracle.sample(g, wl.seeds[int(wl.inst_offsets[i]):int(wl.inst_offsets[i + 1])], sub, wl.fanout,
                              wl.bias, wl.rng_seed, layer=True)
            t_used += time.perf_counter() - t
            done += int(r["edge_off"][-1])
            used += 1
            if t_used > args.cpu_baseline_seconds:
                break
        out["cpu_baseline"] = {"value": done / t_used, "unit": "edges/s", "cores": 1, "kind": "oracle",
                               "sample": f"{used} instances, full depth, {t_used:.1f} s single-threaded"}
    return out


# --------------------------------------------------------------------------
# Out-of-memory walks (graph in host memory), not the default line.

def run_oom_bench(args):
    """Walks and layered sampling over an RMAT graph kept in host memory,
    streamed through a device budget of a quarter of the graph, with one
    partition slot (no overlap) and with two slots (the next partition loaded
    while the current one is sampled), host arrays pageable or page-locked
    for the call."""
    import torch
    from paper_2009_09103_gb300 import build, csaw, inputs
    build.build()
    torch.cuda.set_device(0)
    scale = args.scale or 22
    t0 = time.time()
    g = inputs.rmat_csr(scale, 16, 255, scale)
    graph_bytes = 8 * (g.V + 1) + 16 * g.E   # offsets, columns, weights and prefix sums
    budget = graph_bytes // 4
    starts = np.arange(0, g.V, 4, dtype=np.uint32)
    L = 40
    sizes = inputs.loguniform_sizes(1024, 6.0, 4.0, scale, stream=7)
    seeds, io = inputs.distinct_seeds(sizes, g.V, scale, stream=7)
    fan = [25, 10]
    log(f"[bench] oom graph s{scale}: V={g.V} E={g.E} built in {time.time() - t0:.1f}s; budget {budget >> 20} MiB")
    G = csaw.Graph(g.off, g.col, g.w)
    ref_path = csaw.walk(G, starts, L, "edge_weight", 7)
    ref_s = csaw.sample(G, seeds, io, fan, "edge_weight", 9)
    t = time.perf_counter()
    csaw.walk(G, starts, L, "edge_weight", 7)
    t_walk_mem = time.perf_counter() - t
    t = time.perf_counter()
    csaw.sample(G, seeds, io, fan, "edge_weight", 9)
    t_sample_mem = time.perf_counter() - t
    G.close()
    walk_edges = int((ref_path[:, 1:] != 0xFFFFFFFF).sum())
    sample_edges = int(ref_s.n_edges)

    def timed(fn, reps):
        fn()   # warm-up
        ts, out = [], None
        for _ in range(reps):
            t1 = time.perf_counter()
            out = fn()
            ts.append(time.perf_counter() - t1)
        return float(np.median(ts)), out

    reps = max(1, min(args.steps, 3))
    walks, samples = {}, {}
    for slots, pin in ((1, False), (2, False), (2, True)):
        name = f"slots{slots}_{'pinned' if pin else 'pageable'}"
        sec, (path, st) = timed(lambda: csaw.walk_oom(g.off, g.col, g.w, starts, L, "edge_weight", 7,
                                                      budget_bytes=budget, slots=slots, pin_host=pin), reps)
        walks[name] = {"seconds": sec, "seps": walk_edges / sec, "identical_to_in_memory": bool(np.array_equal(path, ref_path)),
                       **st, "link_gbs": st["bytes_loaded"] / sec / 1e9}
        sec, (res, st) = timed(lambda: csaw.sample_oom(g.off, g.col, g.w, seeds, io, fan, "edge_weight", 9,
                                                       budget_bytes=budget, slots=slots, pin_host=pin), reps)
        samples[name] = {"seconds": sec, "seps": sample_edges / sec,
                         "identical_to_in_memory": bool(np.array_equal(res.dst, ref_s.dst) and
                                                        np.array_equal(res.edge_offsets, ref_s.edge_offsets)),
                         **st, "link_gbs": st["bytes_loaded"] / sec / 1e9}
        log(f"[bench] oom {name}: walk {walks[name]['seconds']:.3f}s, sample {samples[name]['seconds']:.3f}s")
    # the host CSR read in place (coherent host access): no partition copies
    sec, (path, st) = timed(lambda: csaw.walk_oom(g.off, g.col, g.w, starts, L, "edge_weight", 7,
                                                  budget_bytes=budget, slots=2, direct=True), reps)
    walks["direct"] = {"seconds": sec, "seps": walk_edges / sec,
                       "identical_to_in_memory": bool(np.array_equal(path, ref_path)), **st,
                       "host_reads": "summaries built on the device from the host weights; each step reads one "
                                     "32-byte group of weights and the picked column from host memory"}
    log(f"[bench] oom direct (mode {st['direct']}): walk {sec:.3f}s")
    best = min(walks.values(), key=lambda r: r["seconds"])
    return {
        "metric": METRIC, "value": best["seps"], "unit": "edges/s", "n_gpus": 1, "steps": reps,
        "warmup": 1, "ms_per_step": 1e3 * best["seconds"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32 biases / u64 prefix sums", "data": "synthetic (seeded RMAT)",
        "config": {"workload": f"out-of-memory walks and sampling: RMAT scale {scale}, edge factor 16 in host memory, "
                               f"device budget per slot a quarter of the graph ({budget >> 20} MiB); {len(starts)} "
                               f"walkers of length {L}; {len(sizes)} sampling instances of log-uniform [64,1024) "
                               f"seeds, fanout {fan}; edge-weight bias",
                   "timing": "wall clock of the whole call (host CSR in, result out), median",
                   "walk_edges": walk_edges, "sample_edges": sample_edges},
        "walks": walks, "sampling": samples,
        "in_memory_seconds": {"walk": t_walk_mem, "sample": t_sample_mem},
    }


# --------------------------------------------------------------------------
# Attempts per pick (the iterations per pick of Sec. VI / Fig. 10): repeated
# sampling against updated sampling from the first pick (attempt cap 0, the
# exact form of bipartite region search), counted by the library built with
# the selection counters.

def run_attempts_bench(args):
    os.environ["CSAW_LIB_VARIANT"] = "stats"
    import torch
    from paper_2009_09103_gb300 import build, csaw, inputs
    build.build()
    torch.cuda.set_device(0)
    cases = []
    s12 = inputs.workload_sample_s12()
    cases.append(("RMAT s12, 256 seeds, fanout [10,5]", s12.graph, s12.seeds, s12.inst_offsets, [10, 5]))
    b24 = inputs.workload_batched_s24()
    cases.append(("RMAT s24, 4096 instances, fanout [25,10]", b24.graph, b24.seeds, b24.inst_offsets, [25, 10]))
    rows = []
    for name, g, seeds, io, fan in cases:
        G = csaw.Graph(g.off, g.col, g.w)
        for bias in ("neighbor_degree", "edge_weight"):
            out = {"workload": name, "bias": bias}
            for label, cap in (("repeated", 1024), ("updated_from_first_pick", 0)):
                csaw.selection_stats(reset=True)
                res = csaw.sample(G, seeds, io, fan, bias, 4, attempt_cap=cap, to_host=False)
                c = csaw.selection_stats(reset=True)
                picks = max(1, c["drawn_picks"])
                out[label] = {**c, "sampled_edges": int(res.n_edges),
                              "draws_per_pick": c["draws_consumed"] / picks,
                              "evaluated_per_pick": c["draws_evaluated"] / picks}
                del res
            out["reduction_draws_per_pick"] = (out["repeated"]["draws_per_pick"] /
                                               out["updated_from_first_pick"]["draws_per_pick"])
            rows.append(out)
            log(f"[bench] attempts {name} {bias}: repeated {out['repeated']['draws_per_pick']:.3f} per pick, "
                f"updated {out['updated_from_first_pick']['draws_per_pick']:.3f}; "
                f"x{out['reduction_draws_per_pick']:.2f}")
        G.close()
    return {"metric": "draws per pick (iterations per pick)", "value": rows[0]["reduction_draws_per_pick"],
            "unit": "ratio", "higher_is_better": True, "n_gpus": 1, "data": "synthetic (seeded RMAT)",
            "library": "built with -DCSAW_STATS (counters; not for timing)", "rows": rows}


# --------------------------------------------------------------------------
# Serving (config: RMAT s26 resident): open-loop Poisson arrivals of a 50/50
# mix of sampling and walk requests into csaw_server, against the same
# requests run one after another with plain calls.

def req_edges(r, res):
    return int(res.sample.n_edges) if r[0] == "sample" else int((res.path[:, 1:] != 0xFFFFFFFF).sum())


def served_leg(csaw, G, reqs, loads, slots, budget):
    """Serial plain service times, then the server at each load point.
    Serial plain is a FIFO queue of one request at a time whose service times
    are each request's measured wall time as a plain host call (csaw_sample /
    csaw_walk with host inputs and host results) run alone."""
    import threading
    import torch
    for r in reqs[: min(8, len(reqs))]:   # warm-up
        if r[0] == "sample":
            csaw.sample(G, r[1], r[2], r[3], "edge_weight", r[4])
        else:
            csaw.walk(G, r[1], r[2], "edge_weight", r[3])
    torch.cuda.synchronize()
    svc, edges = [], []
    for r in reqs:
        t = time.perf_counter()
        if r[0] == "sample":
            res = csaw.sample(G, r[1], r[2], r[3], "edge_weight", r[4])
            edges.append(int(res.n_edges))
        else:
            p = csaw.walk(G, r[1], r[2], "edge_weight", r[3])
            edges.append(int((p[:, 1:] != 0xFFFFFFFF).sum()))
        svc.append(time.perf_counter() - t)
    svc = np.array(svc)
    total_edges = int(sum(edges))
    serial_capacity = len(reqs) / svc.sum()
    points = []
    for frac in loads:
        lam = frac * serial_capacity
        rng = np.random.default_rng(int(frac * 1000))
        arrivals = np.cumsum(rng.exponential(1.0 / lam, size=len(reqs)))
        fin = np.zeros(len(reqs))
        prev = 0.0
        for i in range(len(reqs)):
            start = max(arrivals[i], prev)
            fin[i] = start + svc[i]
            prev = fin[i]
        lat_serial = fin - arrivals
        srv = csaw.Server(G, budget_bytes=budget, slots=slots)
        # warm the server with the largest requests of the mix before the timed arrivals
        big = sorted(range(len(reqs)), key=lambda i: -edges[i])[: 2 * slots]
        warm = []
        for i in big:
            r = reqs[i]
            warm.append(srv.submit_sample(r[1], r[2], r[3], "edge_weight", r[4]) if r[0] == "sample"
                        else srv.submit_walk(r[1], r[2], "edge_weight", r[3]))
        for t in warm:
            srv.poll(t)
        tickets = [None] * len(reqs)
        base = time.perf_counter() + 0.05

        def submitter():
            for i, r in enumerate(reqs):
                delay = base + arrivals[i] - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                if r[0] == "sample":
                    tickets[i] = srv.submit_sample(r[1], r[2], r[3], "edge_weight", r[4])
                else:
                    tickets[i] = srv.submit_walk(r[1], r[2], "edge_weight", r[3])
        th = threading.Thread(target=submitter)
        th.start()
        th.join()
        lat, wait = [], []
        first_sub, last_fin = None, 0
        for i, r in enumerate(reqs):
            res = srv.poll(tickets[i])
            lat.append((res.t_finish_ns - res.t_submit_ns) / 1e9)
            wait.append((res.t_start_ns - res.t_submit_ns) / 1e9)
            first_sub = res.t_submit_ns if first_sub is None else min(first_sub, res.t_submit_ns)
            last_fin = max(last_fin, res.t_finish_ns)
        srv.close()
        span = (last_fin - first_sub) / 1e9
        lat = np.array(lat)
        slow = np.argsort(-lat)[:3]
        worst = [{"kind": reqs[i][0], "size": int(len(reqs[i][1])), "edges": int(edges[i]),
                  "latency_ms": 1e3 * float(lat[i]), "waited_ms": 1e3 * float(wait[i]),
                  "serial_service_ms": 1e3 * float(svc[i])} for i in slow]
        pt = {"load_frac_of_serial_capacity": frac, "arrival_rate_per_s": lam,
              "served": {"seps": total_edges / span, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                         "p99_ms": 1e3 * float(np.percentile(lat, 99)), "slowest": worst},
              "serial_plain": {"seps": total_edges / (fin[-1] - arrivals[0]),
                               "p50_ms": 1e3 * float(np.percentile(lat_serial, 50)),
                               "p99_ms": 1e3 * float(np.percentile(lat_serial, 99))}}
        pt["served_wins_p99"] = bool(pt["served"]["p99_ms"] <= pt["serial_plain"]["p99_ms"])
        pt["served_wins_seps"] = bool(pt["served"]["seps"] >= pt["serial_plain"]["seps"])
        points.append(pt)
        log(f"[bench] load {frac:.2f}: served {pt['served']['seps'] / 1e6:.1f} M SEPS p50/p99 "
            f"{pt['served']['p50_ms']:.1f}/{pt['served']['p99_ms']:.1f} ms; serial "
            f"{pt['serial_plain']['seps'] / 1e6:.1f} M SEPS {pt['serial_plain']['p50_ms']:.1f}/"
            f"{pt['serial_plain']['p99_ms']:.1f} ms")
    return {"serial_plain": {"capacity_req_per_s": serial_capacity, "seps": total_edges / svc.sum(),
                             "service_ms_p50": 1e3 * float(np.percentile(svc, 50)),
                             "service_ms_p99": 1e3 * float(np.percentile(svc, 99))},
            "sampled_edges": total_edges, "points": points}


def serve_desc(scale, n, slots):
    return (f"serving: RMAT scale {scale} edge factor 16 resident; {n} requests, 50/50 layered sampling "
            "(seeds log-uniform [1,16384], depth 1-3, fanout from {5,10,25}) and weighted walks (starts "
            "log-uniform [1,65536], length U[10,80]); Poisson arrivals; 40 GiB admission budget; "
            f"{slots} slots")


def served_block(args, forms=("streamed", "cached")):
    """The serving comparison on the resident graph, with the cumulative
    arrays streamed per selection and cached per edge."""
    import torch
    from paper_2009_09103_gb300 import csaw, inputs
    t0 = time.time()
    scale = args.serve_scale
    g = inputs.rmat_csr(scale, 16, 255, scale)
    log(f"[bench] serve: graph s{scale} V={g.V} E={g.E} built in {time.time() - t0:.1f}s")
    G = csaw.Graph(g.off, g.col, g.w)
    V = g.V
    del g
    reqs = inputs.serving_requests(V, args.requests, 5)
    out = {"workload": serve_desc(scale, len(reqs), args.slots)}
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    for form in forms:
        if form == "cached":
            G.build_cdf("edge_weight")
        out[form + "_cumulative_array"] = served_leg(csaw, G, reqs, args.loads, args.slots, 40 << 30)
        if form == "cached":
            G.drop_cdf("edge_weight")
    clk = clocks.stop()
    G.close()
    if clk:
        out["clocks"] = clk
    return out


def run_serve_bench(args):
    import torch
    from paper_2009_09103_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    args.serve_scale = args.scale or 26
    blk = served_block(args, ("cached",) if args.cdf else ("streamed",))
    leg = blk["cached_cumulative_array" if args.cdf else "streamed_cumulative_array"]
    best = max(leg["points"], key=lambda p: p["served"]["seps"])
    return {
        "metric": METRIC + " and p50/p99 request latency", "value": best["served"]["seps"], "unit": "edges/s",
        "n_gpus": 1, "steps": len(args.loads), "warmup": 1, "ms_per_step": None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32 biases / u64 prefix sums",
        "data": "synthetic (seeded RMAT, seeded request mix)",
        "config": {"workload": blk["workload"] + "; cumulative array "
                   + ("cached per edge" if args.cdf else "computed per selection"),
                   "sampled_edges": leg["sampled_edges"]},
        **leg,
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cpu-baseline-seconds", type=float, default=12.0,
                    help="oracle sample budget; 0 skips the CPU baseline")
    ap.add_argument("--ref-seconds", type=float, default=None,
                    help="--impl reference: oracle seconds per step (default: about a minute in all)")
    ap.add_argument("--workload", default="walk",
                    choices=["walk", "node2vec", "sample_s12", "batched_s24", "serve", "mdrw", "layer", "oom",
                             "attempts"])
    ap.add_argument("--autotune", action="store_true", help="sampling workloads: autotune first")
    ap.add_argument("--no-variant", action="store_true",
                    help="walks: skip the per-visit streaming walk measured after the main line")
    ap.add_argument("--streaming", action="store_true",
                    help="walks: the main line streams each step's row (no cumulative array)")
    ap.add_argument("--cdf", action="store_true",
                    help="build the cached per-edge cumulative array of the static bias first")
    ap.add_argument("--plain-instances", type=int, default=4096,
                    help="batched: instances timed one call each (a uniform subset when fewer than all)")
    ap.add_argument("--batched-steps", type=int, default=2, help="batched block: timed plan runs per form")
    ap.add_argument("--serve-scale", type=int, default=26, help="served block: RMAT scale of the graph")
    ap.add_argument("--no-batched", action="store_true", help="default run: skip the batched block")
    ap.add_argument("--no-served", action="store_true", help="default run: skip the served block")
    ap.add_argument("--instances", type=int, default=4096, help="batched_s24 at another --scale")
    ap.add_argument("--requests", type=int, default=400, help="serve: requests per load point")
    ap.add_argument("--slots", type=int, default=8, help="serve: server slots")
    ap.add_argument("--loads", type=float, nargs="+", default=[0.25, 0.5, 1.0, 1.5, 3.0],
                    help="serve: arrival rates as multiples of the serial capacity")
    ap.add_argument("--scale", type=int, default=None, help="RMAT scale (default: the workload's)")
    args = ap.parse_args()
    if args.scale is None:
        args.scale = {"walk": 20, "node2vec": 22}.get(args.workload)
    rank, world, local = dist_env()
    if args.workload in ("sample_s12", "batched_s24", "serve", "mdrw", "layer", "oom", "attempts"):
        res = (run_serve_bench(args) if args.workload == "serve" else
               run_attempts_bench(args) if args.workload == "attempts" else
               run_mdrw_bench(args) if args.workload == "mdrw" else
               run_oom_bench(args) if args.workload == "oom" else
               run_layer_bench(args) if args.workload == "layer" else run_sample_bench(args))
        print(jdump(res), flush=True)
        return

    if args.impl == "reference":
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("gloo")
        res = run_reference(args, rank, world)
        if rank == 0:
            print(jdump(res), flush=True)
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    import torch
    if world > 1:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    result, (g, wl, n_trans) = run_walk_bench(args, rank, world)
    if rank == 0 and world == 1 and args.cpu_baseline_seconds > 0:
        v, used, t = oracle_walk_sample(g, wl, args.cpu_baseline_seconds)
        result["cpu_baseline"] = {"value": v, "unit": "edges/s", "cores": 1, "kind": "oracle",
                                  "sample": f"{used} walkers (uniformly spaced), full length "
                                            f"{wl.length}, {t:.1f} s single-threaded"}
        cores = os.cpu_count() or 1
        v, used, t = oracle_walk_all_cores(g, wl, min(args.cpu_baseline_seconds, 8.0), cores)
        result["cpu_baseline_all_cores"] = {"value": v, "unit": "edges/s", "cores": cores, "kind": "oracle",
                                            "sample": f"{used} walkers in {cores} disjoint shards, one copy "
                                                      f"of the oracle per core, {t:.1f} s"}
    if rank == 0 and world == 1:
        # the batched and served forms against plain one-call-per-request
        # sampling, on their own configurations (RMAT s24 and s26)
        del g, wl
        if not args.no_batched:
            result["batched"] = batched_block(args)
        if not args.no_served:
            result["served"] = served_block(args)
    if rank == 0:
        print(jdump(result), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
