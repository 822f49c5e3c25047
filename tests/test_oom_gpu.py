"""Out-of-memory walks (graph in host memory, streamed by partition) on the
GPU: the paths equal csaw_walk's and the oracle's."""
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


@pytest.mark.parametrize("bias", ["uniform", "edge_weight"])
@pytest.mark.parametrize("budget", [1 << 30, 1 << 18, "smallest"])
def test_oom_walk_equals_in_memory_walk(csaw, bias, budget):
    g = inputs.rmat_csr(12, 16, 100, 12)
    g.w[::7] = 0   # zero weights: dead ends where a row has no positive weight
    if budget == "smallest":   # just above the largest row: tens of partitions
        budget = 16 * int(np.diff(g.off).max()) + 1024
    starts = np.concatenate([np.arange(g.V, dtype=np.uint32), inputs.uniform_vertices(2000, g.V, 3)])
    path, st = csaw.walk_oom(g.off, g.col, g.w, starts, 30, bias, 41, budget_bytes=budget)
    G = csaw.Graph(g.off, g.col, g.w)
    ref = csaw.walk(G, starts, 30, bias, 41)
    G.close()
    assert np.array_equal(path, ref)
    assert np.array_equal(path, oracle.walk(g, starts, 30, bias, 41))
    if budget < 1 << 18:
        assert st["partitions"] > (20 if bias == "edge_weight" else 5) and st["loads"] >= st["partitions"]
    if budget == 1 << 30:
        assert st["partitions"] == 1


def test_oom_walk_hub_rows_and_errors(csaw):
    rng = np.random.default_rng(3)
    d = 30000
    edges = [(0, j + 1) for j in range(d)] + [(j + 1, 0) for j in range(d)]
    w = list(rng.integers(1, 2**20, size=d)) + [1] * d
    g = inputs.csr_from_edges(d + 1, edges, w)
    starts = np.concatenate([np.zeros(64, dtype=np.uint32), inputs.uniform_vertices(64, g.V, 2)])
    path, st = csaw.walk_oom(g.off, g.col, g.w, starts, 20, "edge_weight", 5, budget_bytes=16 * d + 4096)
    assert np.array_equal(path, oracle.walk(g, starts, 20, "edge_weight", 5))
    assert st["partitions"] >= 2
    with pytest.raises(csaw.CsawError):   # the hub's row does not fit
        csaw.walk_oom(g.off, g.col, g.w, starts, 5, "edge_weight", 5, budget_bytes=16 * d - 1)
    with pytest.raises(csaw.CsawError):
        csaw.walk_oom(g.off, g.col, g.w, np.array([g.V], dtype=np.uint32), 5, "edge_weight", 5)
    with pytest.raises(csaw.CsawError):
        csaw.walk_oom(g.off, g.col, g.w, starts, 5, "neighbor_degree", 5)
