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


@pytest.mark.parametrize("slots,pin", [(2, False), (3, True), (1, False)])
def test_oom_walk_slots_and_prefetch(csaw, slots, pin):
    """Several partition slots, the next busiest partition loaded while a
    round runs, and page-locked host arrays: the same paths."""
    g = inputs.rmat_csr(13, 16, 100, 13)
    budget = 16 * int(np.diff(g.off).max()) + 4096
    starts = inputs.uniform_vertices(5000, g.V, 9)
    path, st = csaw.walk_oom(g.off, g.col, g.w, starts, 25, "edge_weight", 17, budget_bytes=budget,
                             slots=slots, pin_host=pin)
    assert np.array_equal(path, oracle.walk(g, starts, 25, "edge_weight", 17))
    assert st["partitions"] > 5
    if slots > 1:
        assert st["reuses"] > 0


@pytest.mark.parametrize("bias", ["uniform", "edge_weight"])
def test_oom_walk_direct_reads_host_arrays(csaw, bias):
    """Direct mode: the device reads the host CSR in place (summaries and
    records of the weights built on the device from the host weights); the
    paths equal the oracle's, zero weights and dead ends included."""
    g = inputs.rmat_csr(13, 16, 100, 13)
    g.w[::7] = 0
    starts = np.concatenate([np.arange(g.V, dtype=np.uint32), inputs.uniform_vertices(3000, g.V, 5)])
    path, st = csaw.walk_oom(g.off, g.col, g.w, starts, 30, bias, 41, budget_bytes=1 << 26, direct=True)
    assert np.array_equal(path, oracle.walk(g, starts, 30, bias, 41))
    if st["direct"] == 0:
        pytest.skip("this device does not read pageable host memory")
    assert st["loads"] == 0 and st["bytes_loaded"] == 0
    # summaries that do not fit the budget: the call partitions instead
    path2, st2 = csaw.walk_oom(g.off, g.col, g.w, starts, 30, bias, 41, budget_bytes=16 * int(np.diff(g.off).max()) + 4096,
                               slots=1, direct=True)
    assert np.array_equal(path2, path)
    if bias == "edge_weight":
        assert st2["direct"] == 0 and st2["partitions"] > 1


def test_oom_walk_direct_hub_and_bad_columns(csaw):
    rng = np.random.default_rng(4)
    d = 30000
    edges = [(0, j + 1) for j in range(d)] + [(j + 1, 0) for j in range(d)]
    w = list(rng.integers(1, 2**20, size=d)) + [1] * d
    g = inputs.csr_from_edges(d + 1, edges, w)
    starts = np.concatenate([np.zeros(64, dtype=np.uint32), inputs.uniform_vertices(64, g.V, 2)])
    path, st = csaw.walk_oom(g.off, g.col, g.w, starts, 20, "edge_weight", 5, budget_bytes=1 << 24, direct=True)
    assert np.array_equal(path, oracle.walk(g, starts, 20, "edge_weight", 5))
    col = g.col.copy()
    col[len(col) // 3] = g.V + 9
    with pytest.raises(csaw.CsawError) as e:
        csaw.walk_oom(g.off, col, g.w, starts, 5, "edge_weight", 5, budget_bytes=1 << 24, direct=True)
    assert e.value.status == csaw.ERR_INVALID


def _sample_cases():
    g = inputs.rmat_csr(12, 16, 100, 12)
    sizes = inputs.loguniform_sizes(30, 0.0, 7.0, 4)
    seeds, io = inputs.distinct_seeds(sizes, g.V, 4)
    return g, seeds, io


@pytest.mark.parametrize("bias,fanout", [("edge_weight", [10, 5]), ("neighbor_degree", [25, 10]),
                                         ("uniform", [3, 3, 3]), ("edge_weight", [0xFFFFFFFF, 2]),
                                         ("edge_weight", [300, 2])])
@pytest.mark.parametrize("budget", ["whole", "several", "smallest"])
def test_oom_sampling_equals_in_memory_sampling(csaw, bias, fanout, budget):
    """Layered sampling over a host-resident graph, one partition at a time
    (busiest first), equals csaw_sample and the oracle at any partition count."""
    g, seeds, io = _sample_cases()
    big = 16 * int(np.diff(g.off).max()) + 1024
    b = {"whole": 1 << 30, "several": 16 * g.E // 4 + big, "smallest": big}[budget]
    res, st = csaw.sample_oom(g.off, g.col, g.w, seeds, io, fanout, bias, 23, budget_bytes=b, slots=2)
    ref = oracle.sample(g, seeds, io, fanout, bias, 23)
    assert np.array_equal(res.edge_offsets, ref["edge_off"])
    assert np.array_equal(res.src, ref["src"]) and np.array_equal(res.dst, ref["dst"])
    assert np.array_equal(res.frontier_sizes, ref["fsize"][: len(fanout) * (len(io) - 1)])
    G = csaw.Graph(g.off, g.col, g.w)
    mem = csaw.sample(G, seeds, io, fanout, bias, 23)
    G.close()
    assert np.array_equal(res.dst, mem.dst)
    if budget == "smallest":
        assert st["partitions"] > 5 and st["loads"] >= len(fanout)
    if budget == "whole":
        assert st["partitions"] == 1


def test_oom_sampling_slots_pinning_and_errors(csaw):
    g, seeds, io = _sample_cases()
    big = 16 * int(np.diff(g.off).max()) + 1024
    ref = oracle.sample(g, seeds, io, [25, 10], "neighbor_degree", 4)
    for slots, pin in ((1, False), (3, True), (8, False)):
        res, st = csaw.sample_oom(g.off, g.col, g.w, seeds, io, [25, 10], "neighbor_degree", 4, budget_bytes=big,
                                  slots=slots, pin_host=pin)
        assert np.array_equal(res.dst, ref["dst"]) and np.array_equal(res.edge_offsets, ref["edge_off"])
    w0 = g.w.copy()
    w0[5] = 0
    with pytest.raises(csaw.CsawError) as e:   # a zero bias is refused
        csaw.sample_oom(g.off, g.col, w0, seeds, io, [5], "edge_weight", 1, budget_bytes=big)
    assert e.value.status == csaw.ERR_INVALID
    with pytest.raises(csaw.CsawError) as e:   # a row larger than the budget
        csaw.sample_oom(g.off, g.col, g.w, seeds, io, [5], "edge_weight", 1, budget_bytes=big // 2)
    assert e.value.status == csaw.ERR_NOMEM
    with pytest.raises(csaw.CsawError) as e:
        csaw.sample_oom(g.off, g.col, g.w, seeds, io, [5], "node2vec", 1, budget_bytes=big)
    assert e.value.status == csaw.ERR_INVALID


def test_oom_bad_columns_are_refused(csaw):
    """Columns are checked on the device as partitions arrive: a column that
    is not a vertex fails the call (no walker is left outside every
    partition, no kernel reads out of range)."""
    g, seeds, io = _sample_cases()
    col = g.col.copy()
    col[len(col) // 2] = g.V + 5
    big = 16 * int(np.diff(g.off).max()) + 1024
    starts = inputs.uniform_vertices(3000, g.V, 1)
    for slots in (1, 2):
        with pytest.raises(csaw.CsawError) as e:
            csaw.walk_oom(g.off, col, g.w, starts, 20, "edge_weight", 3, budget_bytes=big, slots=slots)
        assert e.value.status == csaw.ERR_INVALID
        with pytest.raises(csaw.CsawError) as e:
            csaw.sample_oom(g.off, col, g.w, np.arange(g.V, dtype=np.uint32),
                            np.array([0, g.V], dtype=np.uint64), [3], "edge_weight", 1, budget_bytes=big, slots=slots)
        assert e.value.status == csaw.ERR_INVALID
    # neighbour degree: an edge into a vertex without neighbours
    gd = inputs.csr_from_edges(5, [(0, 1), (0, 2), (1, 0), (2, 3), (3, 4)])   # vertex 4 has no neighbours
    with pytest.raises(csaw.CsawError) as e:
        csaw.sample_oom(gd.off, gd.col, gd.w, np.array([0, 2], dtype=np.uint32), np.array([0, 2], dtype=np.uint64),
                        [1], "neighbor_degree", 1, budget_bytes=1 << 20)
    assert e.value.status == csaw.ERR_INVALID
