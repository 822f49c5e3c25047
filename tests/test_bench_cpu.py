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
