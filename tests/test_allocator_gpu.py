"""csaw_graph_set_allocator: the library's device memory through the caller's
allocator (here PyTorch's caching allocator), with results unchanged."""
import numpy as np
import pytest

from paper_2009_09103_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_09103_gb300 import build
    build.build()
    from paper_2009_09103_gb300 import csaw
    return torch, csaw


def test_torch_allocator_covers_the_library(env):
    torch, csaw = env
    g = inputs.rmat_csr(14, 16, 100, 14)
    sizes = inputs.loguniform_sizes(40, 2.0, 6.0, 3)
    seeds, io = inputs.distinct_seeds(sizes, g.V, 3)
    starts = inputs.uniform_vertices(4000, g.V, 8)
    G = csaw.Graph(g.off, g.col, g.w)
    ref_s = csaw.sample(G, seeds, io, [25, 10], "neighbor_degree", 5)
    ref_w = csaw.walk(G, starts, 30, "edge_weight", 6)
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    seen = {"n": 0, "covered": True}

    def on_alloc(ptr, nbytes):
        # the block the library just took counts in torch's allocated memory
        seen["n"] += 1
        seen["covered"] &= ptr is not None and torch.cuda.memory_allocated() - base >= nbytes

    G.use_torch_allocator(on_alloc)
    res = csaw.sample(G, seeds, io, [25, 10], "neighbor_degree", 5, to_host=False)
    torch.cuda.synchronize()
    held = torch.cuda.memory_allocated() - base
    assert seen["n"] > 0 and seen["covered"]
    # the result's device edges stay allocated (through torch) until released
    n_edges = int(res.n_edges)
    assert held >= 8 * n_edges
    src = np.concatenate([t.cpu().numpy().view(np.uint32) for t in res.src])
    dst = np.concatenate([t.cpu().numpy().view(np.uint32) for t in res.dst])
    assert np.array_equal(src, ref_s.src) and np.array_equal(dst, ref_s.dst)
    del res
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base
    n0 = seen["n"]
    w = csaw.walk(G, starts, 30, "edge_weight", 6)
    assert np.array_equal(w, ref_w) and seen["n"] > n0
    # plans and cached arrays made afterwards come from the same allocator
    n1 = seen["n"]
    plan = csaw.SamplePlan(G, len(io) - 1, len(seeds), [25, 10], "neighbor_degree")
    assert seen["n"] > n1
    plan.run(seeds, io, 5)
    got = plan.result()
    assert np.array_equal(got.dst, ref_s.dst) and np.array_equal(got.edge_offsets, ref_s.edge_offsets)
    plan.close()
    G.build_cdf("edge_weight")
    assert np.array_equal(csaw.walk(G, starts, 30, "edge_weight", 6), ref_w)
    G.drop_cdf("edge_weight")
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base
    G.use_own_allocator()
    n2 = seen["n"]
    assert np.array_equal(csaw.walk(G, starts, 30, "edge_weight", 6), ref_w)
    assert seen["n"] == n2
    G.close()


def test_torch_allocator_in_the_server(env):
    """Server slots run on their own threads; their buffers come from the
    graph's allocator too, and results stay those of the requests alone."""
    torch, csaw = env
    g = inputs.rmat_csr(12, 16, 100, 12)
    G = csaw.Graph(g.off, g.col, g.w)
    seeds = inputs.uniform_vertices(300, g.V, 2)
    io = np.array([0, 300], dtype=np.uint64)
    starts = inputs.uniform_vertices(500, g.V, 3)
    ref_s = csaw.sample(G, seeds, io, [5, 5], "edge_weight", 1)
    ref_w = csaw.walk(G, starts, 20, "edge_weight", 2)
    count = {"n": 0}
    G.use_torch_allocator(lambda p, n: count.__setitem__("n", count["n"] + 1))
    srv = csaw.Server(G, budget_bytes=1 << 30, slots=2)
    t1 = srv.submit_sample(seeds, io, [5, 5], "edge_weight", 1)
    t2 = srv.submit_walk(starts, 20, "edge_weight", 2)
    r1, r2 = srv.poll(t1), srv.poll(t2)
    srv.close()
    assert count["n"] > 0
    assert np.array_equal(r1.sample.dst, ref_s.dst) and np.array_equal(r2.path, ref_w)
    G.close()


def test_set_allocator_rejects_half_a_pair(env):
    torch, csaw = env
    g = inputs.rmat_csr(8, 8, 40, 1)
    G = csaw.Graph(g.off, g.col, g.w)
    st = csaw.lib().csaw_graph_set_allocator(G.handle, csaw.ALLOC_FN(lambda n, s, c: None), csaw.FREE_FN(), None)
    assert st == csaw.ERR_INVALID
    G.close()
