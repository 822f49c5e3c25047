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


def traffic_record(kernel_src: str, workload: str):
    """dram bytes per launch from the committed ncu summary, if it was taken
    on the current source of the kernel's translation unit and this workload."""
    p = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        recs = json.load(f)
    src = open(os.path.join(ROOT, "paper_2009_09103_gb300", "csrc", kernel_src), "rb").read()
    sha = hashlib.sha256(src).hexdigest()[:16]
    for r in recs:
        if r.get("source") == kernel_src and r.get("source_sha") == sha and r.get("workload") == workload:
            return r
    return None


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


def run_walk_bench(args, rank, world):
    import torch
    from paper_2009_09103_gb300 import build, csaw, inputs

    build.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    t0 = time.time()
    wl = walk_workload(args)
    g = wl.graph
    log(f"[bench] {args.workload} graph: V={g.V} E={g.E} built in {time.time() - t0:.1f}s")
    G = csaw.Graph(g.off, g.col, g.w)
    stream = torch.cuda.current_stream()
    starts = torch.from_numpy(wl.starts.view(np.int32)).to(dev)
    n = starts.numel()
    path = torch.empty((n, wl.length + 1), dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    seed = wl.rng_seed + rank  # replicas: independent walks per rank

    def step():
        csaw.walk(G, starts, wl.length, wl.bias, seed, wl.n2v_mult, path=path, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    off_t = torch.from_numpy(g.off.astype(np.int64)).to(dev)
    n_trans, alg_bytes = walk_bytes(torch, off_t, path)

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
    csaw.walk(G, hs, wl.length, wl.bias, seed, wl.n2v_mult, path=hp, stream=stream)   # warm
    e2e_steps = max(1, min(args.steps, 5))
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for _ in range(e2e_steps):
        csaw.walk(G, hs, wl.length, wl.bias, seed, wl.n2v_mult, path=hp, stream=stream)
    e2e_s = (time.perf_counter() - t1) / e2e_steps
    e2e_ok = bool(np.array_equal(hp, path.cpu().numpy().view(np.uint32)))
    e2e = {"value": n_trans * world / e2e_s, "unit": "edges/s",
           "h2d_bytes_per_step": 4 * n, "d2h_bytes_per_step": 4 * n * (wl.length + 1),
           "matches_device_run": e2e_ok}

    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / (ms_per_step / 1e3) / 1e9
    tr = traffic_record("csaw_walk.cu", f"{args.workload}_s{args.scale}")
    kname = "walk_kernel<NODE2VEC>" if wl.bias == "node2vec" else "walk_kernel<EDGE_WEIGHT>"
    roofline = {"bound": "hbm", "kernel": kname, "achieved": round(achieved, 1),
                "peak": peak, "peak_source": peak_kind, "unit": "GB/s",
                "frac": round(achieved / peak, 4),
                "traffic": tr["traffic_bytes_per_launch"] if tr else None,
                "algorithmic_bytes_per_launch": alg_bytes}
    result = {
        "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32 biases / u64 prefix sums", "data": "synthetic (seeded RMAT)",
        "config": {"workload": walk_config(args, wl),
                   "parallelism": "replicas" if world > 1 else "1 GPU",
                   "l2": "flushed (512 MiB write) before every timed step",
                   "sampled_edges_per_step": n_trans},
        "gpu_launches": args.steps,
        "roofline": roofline,
        "e2e": e2e,
    }
    if clk:
        result["clocks"] = clk
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


def run_reference(args, rank, world):
    """The oracle, as it stands, on the host cores, on bounded samples."""
    if rank != 0:
        return None
    wl = walk_workload(args)
    g = wl.graph
    per_step = max(2.0, min(20.0, 60.0 / max(1, args.steps)))
    vals = []
    used_total = 0
    for _ in range(args.warmup):
        oracle_walk_sample(g, wl, 0.5)
    for _ in range(args.steps):
        v, used, _ = oracle_walk_sample(g, wl, per_step)
        vals.append(v)
        used_total += used
    value = statistics.mean(vals)
    sample = (f"{used_total // max(1, args.steps)} walkers per step (uniformly spaced over the "
              f"{len(wl.starts):,}), full length {wl.length}, single-threaded oracle")
    return {
        "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32 biases / u64 prefix sums", "data": "synthetic (seeded RMAT)",
        "impl": "reference",
        "config": {"workload": walk_config(args, wl)},
        "cpu_baseline": {"value": value, "unit": "edges/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cpu-baseline-seconds", type=float, default=12.0,
                    help="oracle sample budget; 0 skips the CPU baseline")
    ap.add_argument("--workload", default="walk", choices=["walk", "node2vec"])
    ap.add_argument("--scale", type=int, default=None, help="RMAT scale (default: the workload's)")
    args = ap.parse_args()
    if args.scale is None:
        args.scale = {"walk": 20, "node2vec": 22}[args.workload]
    rank, world, local = dist_env()

    if args.impl == "reference":
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("gloo")
        res = run_reference(args, rank, world)
        if rank == 0:
            print(json.dumps(res), flush=True)
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
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
