"""Selection by updated sampling from the first pick (attempt cap 0: one
draw per pick, the exact form of bipartite region search, Sec. IV-B and
Theorem 2) and partial caps, against the oracle run with the same cap."""
import numpy as np
import pytest

import oracle
from paper_2009_09103_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def csaw():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_09103_gb300 import build
    build.build()
    from paper_2009_09103_gb300 import csaw as c
    return c


def star(d, seed):
    rng = np.random.default_rng(seed)
    edges = [(0, j + 1) for j in range(d)] + [(j + 1, 0) for j in range(d)]
    return inputs.csr_from_edges(d + 1, edges, list(rng.integers(1, 1000, size=d)) + [1] * d)


@pytest.mark.parametrize("cap", [0, 1, 5, 33])
@pytest.mark.parametrize("cached", [False, True])
def test_attempt_caps_match_oracle(csaw, cap, cached):
    cases = [(inputs.rmat_csr(12, 16, 100, 12), [10, 5], "edge_weight"),
             (inputs.rmat_csr(12, 16, 100, 12), [25, 10], "neighbor_degree"),
             (star(20000, 1), [40], "edge_weight"),
             (star(3000, 2), [300], "edge_weight")]
    for g, fanout, bias in cases:
        G = csaw.Graph(g.off, g.col, g.w)
        if cached:
            G.build_cdf(bias)
        if g.V > 10000:
            seeds = np.zeros(4, dtype=np.uint32)
            io = np.arange(5, dtype=np.uint64)
        else:
            seeds = inputs.uniform_vertices(300, g.V, 1)
            io = np.array([0, 100, 300], dtype=np.uint64)
        res = csaw.sample(G, seeds, io, fanout, bias, 7, attempt_cap=cap)
        ref = oracle.sample(g, seeds, io, fanout, bias, 7, attempt_cap=cap)
        assert np.array_equal(res.dst, ref["dst"]) and np.array_equal(res.edge_offsets, ref["edge_off"]), \
            (g.V, fanout, bias)
        plan = csaw.SamplePlan(G, len(io) - 1, len(seeds), fanout, bias, attempt_cap=cap)
        plan.run(seeds, io, 7)
        assert np.array_equal(plan.result().dst, ref["dst"])
        plan.close()
        G.close()


def test_exclusion_mode_differs_but_keeps_distinctness(csaw):
    g = inputs.rmat_csr(12, 16, 100, 12)
    G = csaw.Graph(g.off, g.col, g.w)
    seeds = inputs.uniform_vertices(256, g.V, 1)
    io = np.array([0, 256], dtype=np.uint64)
    a = csaw.sample(G, seeds, io, [10], "edge_weight", 1)
    b = csaw.sample(G, seeds, io, [10], "edge_weight", 1, attempt_cap=0)
    assert a.n_edges == b.n_edges and not np.array_equal(a.dst, b.dst)
    # picks of one source (consecutive equal src) are distinct neighbours
    cut = np.flatnonzero(np.diff(b.src.astype(np.int64)) != 0) + 1
    for seg_dst, seg_src in zip(np.split(b.dst, cut), np.split(b.src, cut)):
        v = int(seg_src[0])
        assert len(np.unique(seg_dst)) == len(seg_dst)
        assert set(seg_dst.tolist()) <= set(g.col[g.off[v]:g.off[v + 1]].tolist())
    G.close()
