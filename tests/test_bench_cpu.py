"""bench.py's multi-process contract on CPU: launched by torchrun with two
ranks (gloo), the reference arm runs on rank 0 alone and prints one JSON line."""
import json
import os
import subprocess
import sys

import pytest

from conftest import ROOT


@pytest.mark.slow
def test_reference_arm_two_ranks_gloo():
    env = dict(os.environ, MASTER_ADDR="127.0.0.1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", "--master-port=29631", os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--ref-seconds", "0.5",
           "--scale", "14"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2
    assert out["cpu_baseline"]["kind"] == "oracle" and out["cpu_baseline"]["cores"] == (os.cpu_count() or 1)
    assert out["value"] > 0 and out["e2e"]["h2d_bytes_per_step"] == 0


def _bench_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_walk_byte_models_match_a_direct_count():
    """The roofline numerators, counted transition by transition."""
    torch = pytest.importorskip("torch")
    import numpy as np
    bench = _bench_module()
    NONE = 0xFFFFFFFF
    rng = np.random.default_rng(3)
    deg = rng.integers(0, 9, size=40)
    deg[[5, 17, 23]] = [300, 1000, 65]   # rows spanning several 64-edge blocks
    off = np.zeros(41, dtype=np.int64)
    off[1:] = np.cumsum(deg)
    n, L = 30, 7
    path = np.full((n, L + 1), NONE, dtype=np.uint32)
    for i in range(n):
        v = int(rng.integers(0, 40))
        path[i, 0] = v
        for t in range(L):
            if deg[v] == 0 or rng.random() < 0.1:
                break
            v = int(rng.integers(0, 40))
            path[i, t + 1] = v
    ew = n2v = 0
    n_trans = 0
    for i in range(n):
        ew += 4 + 4 * (L + 1)
        n2v += 4 + 4 * (L + 1)
        for t in range(L):
            a, b = path[i, t], path[i, t + 1]
            if a == NONE:
                break
            if b == NONE:
                ew += 16
                n2v += 16
                break
            n_trans += 1
            ew += 16 + 4 * deg[a] + 4
            n2v += 16 + 8 * deg[a]
            if t >= 1:
                n2v += 16 + 4 * deg[path[i, t - 1]]
    off_t = torch.from_numpy(off)
    path_t = torch.from_numpy(path.view(np.int32))
    assert bench.walk_bytes(torch, off_t, path_t) == (n_trans, ew)
    assert bench.node2vec_bytes(torch, off_t, path_t) == (n_trans, n2v)

    # the summary search: per step 32 (record) + 8 per s2 probe over the row's
    # G = (end-1)/64 - beg/64 entries + 32 + 32 + 4 + 4, per walker 4 + 4 (L + 1)
    import math
    cw = 0
    for i in range(n):
        cw += 4 + 4 * (L + 1)
        for t in range(L):
            a, b = path[i, t], path[i, t + 1]
            if a == NONE or b == NONE:
                break
            beg, end = int(off[a]), int(off[a + 1])
            G = ((end - 1) >> 6) - (beg >> 6)
            cw += 32 + 8 * math.ceil(math.log2(G + 1)) + 32 + 32 + 4 + 4
    assert bench.cached_walk_bytes(torch, off_t, path_t, L) == cw


def test_walk_sector_bytes_match_a_direct_count():
    """Distinct 32-byte sectors per transition, counted address by address."""
    torch = pytest.importorskip("torch")
    import numpy as np
    bench = _bench_module()
    NONE = 0xFFFFFFFF
    rng = np.random.default_rng(5)
    deg = rng.integers(0, 40, size=60)
    off = np.zeros(61, dtype=np.int64)
    off[1:] = np.cumsum(deg)
    n, L = 25, 9
    path = np.full((n, L + 1), NONE, dtype=np.uint32)
    for i in range(n):
        v = int(rng.integers(0, 60))
        path[i, 0] = v
        for t in range(L):
            if deg[v] == 0 or rng.random() < 0.1:
                break
            v = int(rng.integers(0, 60))
            path[i, t + 1] = v
    total = 0
    for i in range(n):
        total += 4 + 4 * (L + 1)
        for t in range(L):
            a, b = int(path[i, t]), int(path[i, t + 1])
            if a == NONE:
                break
            sectors = {(8 * a + k) // 32 for k in range(16)}
            if b == NONE:
                total += 32 * len(sectors)
                break
            wsec = {(4 * e + k) // 32 for e in range(off[a], off[a + 1]) for k in range(4)}
            total += 32 * (len(sectors) + len(wsec) + 1)
    assert bench.walk_sector_bytes(torch, torch.from_numpy(off), torch.from_numpy(path.view(np.int32))) == total


def test_roofline_block_is_dram_based():
    """frac is the DRAM fraction: ncu DRAM bytes per launch / event time /
    measured HBM peak; the method's L2-inclusive bytes are reported apart."""
    bench = _bench_module()
    peak, _ = bench.measured_peaks()
    tr = {"traffic_bytes_per_launch": 45_000_000_000, "ncu_duration_ns": 39_000_000, "l2_hit_rate_pct": 91.0}
    blk = bench.roofline_block("k", tr, 40.0, 460_000_000_000, 463_000_000_000)
    assert blk["bound"] == "hbm" and blk["traffic"] == tr["traffic_bytes_per_launch"]
    assert abs(blk["achieved"] - 45e9 / 0.040 / 1e9) < 0.1
    assert abs(blk["frac"] - blk["achieved"] / peak) < 1e-4 and blk["frac"] < 1.2
    assert blk["l2_inclusive"]["algorithmic_bytes_per_launch"] == 460_000_000_000
    assert blk["l2_inclusive"]["sector_bytes_per_launch"] == 463_000_000_000
    assert blk["l2_hit_rate_pct"] == 91.0
    none = bench.roofline_block("k", None, 40.0, 1000)
    assert none["frac"] is None and none["traffic"] is None
