"""The attempts-per-pick counters (library built with -DCSAW_STATS): the
draws the GPU selections consume equal the oracle's, for repeated sampling
and for updated sampling from the first pick (attempt cap 0)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from conftest import ROOT
from paper_2009_09103_gb300 import inputs

pytestmark = pytest.mark.gpu

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, ROOT)
from paper_2009_09103_gb300 import csaw, inputs
out = {}
for name, scale, fan, bias, cap, cached in CASES:
    g = inputs.rmat_csr(scale, 16, 100, scale)
    sizes = inputs.loguniform_sizes(40, 2.0, 6.0, scale)
    seeds, io = inputs.distinct_seeds(sizes, g.V, scale)
    G = csaw.Graph(g.off, g.col, g.w)
    if cached:
        G.build_cdf(bias)
    csaw.selection_stats(reset=True)
    csaw.sample(G, seeds, io, fan, bias, 7, attempt_cap=cap)
    out[name] = csaw.selection_stats(reset=True)
    G.close()
print(json.dumps(out))
"""

CASES = [("nd_repeated", 12, [25, 10], "neighbor_degree", 1024, False),
         ("nd_updated", 12, [25, 10], "neighbor_degree", 0, False),
         ("ew_cap5", 13, [10, 5], "edge_weight", 5, False),
         ("ew_cached", 13, [10, 5], "edge_weight", 1024, True),
         ("ew_hubs", 14, [300, 3], "edge_weight", 1024, False)]


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_09103_gb300 import build
    build.build()


def test_gpu_draws_consumed_equal_the_oracle(gpu):
    env = dict(os.environ, CSAW_LIB_VARIANT="stats")
    code = f"ROOT = {ROOT!r}\nCASES = {CASES!r}\n" + CHILD
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    got = json.loads(r.stdout.strip().splitlines()[-1])
    for name, scale, fan, bias, cap, _ in CASES:
        g = inputs.rmat_csr(scale, 16, 100, scale)
        sizes = inputs.loguniform_sizes(40, 2.0, 6.0, scale)
        seeds, io = inputs.distinct_seeds(sizes, g.V, scale)
        oracle.stats(reset=True)
        oracle.sample(g, seeds, io, fan, bias, 7, attempt_cap=cap)
        attempts, picks = oracle.stats(reset=True)
        c = got[name]
        assert (c["draws_consumed"], c["drawn_picks"]) == (attempts, picks), name
        assert c["draws_evaluated"] >= c["draws_consumed"]
        if cap == 0:
            assert c["draws_consumed"] == c["drawn_picks"] == c["updated_picks"]


def test_default_library_has_no_counters(gpu):
    from paper_2009_09103_gb300 import csaw
    if os.environ.get("CSAW_LIB_VARIANT") == "stats":
        pytest.skip("the counters build is loaded")
    with pytest.raises(csaw.CsawError) as e:
        csaw.selection_stats()
    assert e.value.status == csaw.ERR_INVALID
