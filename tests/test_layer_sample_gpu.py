"""Layer sampling on the GPU through the C ABI, bit-exact against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2009_09103_gb300 import inputs

pytestmark = pytest.mark.gpu
FANOUT_ALL = 0xFFFFFFFF


@pytest.fixture(scope="module")
def csaw():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_09103_gb300 import build
    build.build()
    from paper_2009_09103_gb300 import csaw as c
    return c


def same(r, ref):
    assert np.array_equal(r.edge_offsets, ref["edge_off"])
    assert np.array_equal(r.frontier_sizes, ref["fsize"][:len(r.frontier_sizes)])
    assert np.array_equal(r.src, ref["src"]) and np.array_equal(r.dst, ref["dst"])


def graphs():
    g8 = inputs.rmat_csr(8, 8, 40, 1)
    g12 = inputs.rmat_csr(12, 16, 100, 12)
    gz = inputs.CSRGraph(g12.off, g12.col, g12.w.copy())
    gz.w[::3] = 0   # zero biases: never picked, the take-all rule counts positives
    return {"rmat_s8": g8, "rmat_s12": g12, "rmat_s12_zero_w": gz}


@pytest.mark.parametrize("gname", ["rmat_s8", "rmat_s12", "rmat_s12_zero_w"])
@pytest.mark.parametrize("bias", ["uniform", "edge_weight", "neighbor_degree"])
@pytest.mark.parametrize("sizes", [[5, 40], [64, 300, 7], [FANOUT_ALL, 3]])
def test_layer_sample_bit_exact(csaw, gname, bias, sizes):
    g = graphs()[gname]
    n_inst = 60
    sz = inputs.loguniform_sizes(n_inst, 0.0, 6.0, 5)
    seeds, io = inputs.distinct_seeds(sz, g.V, 5)
    io[8] = io[7]   # instance 7 empty (instance 8 takes both seed lists)
    G = csaw.Graph(g.off, g.col, g.w)
    r = csaw.layer_sample(G, seeds, io, sizes, bias, 31)
    G.close()
    same(r, oracle.sample(g, seeds, io, sizes, bias, 31, layer=True))


@pytest.mark.parametrize("cap", [0, 1, 33])
def test_layer_sample_updated_sampling(csaw, cap):
    # small attempt caps force the updated-sampling (exclusion) path
    g = graphs()["rmat_s12"]
    sz = inputs.loguniform_sizes(30, 2.0, 4.0, 9)
    seeds, io = inputs.distinct_seeds(sz, g.V, 9)
    G = csaw.Graph(g.off, g.col, g.w)
    r = csaw.layer_sample(G, seeds, io, [200, 50], "edge_weight", 3, attempt_cap=cap)
    G.close()
    same(r, oracle.sample(g, seeds, io, [200, 50], "edge_weight", 3, attempt_cap=cap, layer=True))


def test_layer_sample_hub_rows_and_cached_array(csaw):
    rng = np.random.default_rng(3)
    d = 20000
    edges = [(0, j + 1) for j in range(d)] + [(j + 1, 0) for j in range(d)] + [(1, 2), (2, 1)]
    w = list(rng.integers(1, 1000, size=d)) + [1] * d + [5, 5]
    g = inputs.csr_from_edges(d + 1, edges, w)
    seeds = np.array([0, 5, 0, 1, 2, 7], dtype=np.uint32)
    io = np.array([0, 2, 4, 6], dtype=np.uint64)
    G = csaw.Graph(g.off, g.col, g.w)
    ref = oracle.sample(g, seeds, io, [500, 100], "edge_weight", 8, layer=True)
    same(csaw.layer_sample(G, seeds, io, [500, 100], "edge_weight", 8), ref)
    G.build_cdf("edge_weight")   # row positions by binary search of the cached array
    same(csaw.layer_sample(G, seeds, io, [500, 100], "edge_weight", 8), ref)
    G.close()


def test_layer_sample_device_inputs(csaw):
    import torch
    g = graphs()["rmat_s12"]
    sz = inputs.loguniform_sizes(20, 1.0, 5.0, 2)
    seeds, io = inputs.distinct_seeds(sz, g.V, 2)
    G = csaw.Graph(g.off, g.col, g.w)
    r = csaw.layer_sample(G, torch.from_numpy(seeds.view(np.int32)).cuda(),
                          torch.from_numpy(io.view(np.int64)).cuda(), [30, 30], "neighbor_degree", 4)
    G.close()
    same(r, oracle.sample(g, seeds, io, [30, 30], "neighbor_degree", 4, layer=True))


def test_layer_sample_row_beyond_the_chunk_table(csaw):
    # vertex 0: 2.2 M neighbours (more chunks than a warp's table holds, so
    # its picks scan the row); vertex 1: 10,000 (in the table)
    d0, d1 = 2_200_000, 10_000
    V = d0 + 2
    leaves = np.arange(2, V, dtype=np.uint32)
    deg = np.ones(V, dtype=np.int64)
    deg[0], deg[1] = d0, d1
    deg[2:2 + d1] = 2
    off = np.zeros(V + 1, dtype=np.uint64)
    off[1:] = np.cumsum(deg)
    col = np.empty(int(off[-1]), dtype=np.uint32)
    col[0:d0] = leaves
    col[d0:d0 + d1] = leaves[:d1]
    rest = col[d0 + d1:]
    rest[:2 * d1] = np.tile(np.array([0, 1], dtype=np.uint32), d1)
    rest[2 * d1:] = 0
    w = np.random.default_rng(4).integers(1, 500, size=len(col)).astype(np.uint32)
    g = inputs.CSRGraph(off, col, w)
    seeds = np.array([0, 1, 1, 0], dtype=np.uint32)
    io = np.array([0, 2, 3, 4], dtype=np.uint64)
    G = csaw.Graph(g.off, g.col, g.w)
    r = csaw.layer_sample(G, seeds, io, [300, 20], "edge_weight", 12)
    G.close()
    same(r, oracle.sample(g, seeds, io, [300, 20], "edge_weight", 12, layer=True))
