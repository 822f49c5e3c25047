"""Cached cumulative bias arrays (static biases): walks and sampling read the
per-edge prefix sums instead of streaming each row, with identical picks."""
import numpy as np
import pytest

import oracle
from paper_2009_09103_gb300 import inputs

pytestmark = pytest.mark.gpu
ALL = 0xFFFFFFFF


@pytest.fixture(scope="module")
def csaw():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_09103_gb300 import build
    build.build()
    from paper_2009_09103_gb300 import csaw as c
    return c


def star(d, seed, wmax=1000):
    rng = np.random.default_rng(seed)
    edges = [(0, j + 1) for j in range(d)] + [(j + 1, 0) for j in range(d)]
    return inputs.csr_from_edges(d + 1, edges, list(rng.integers(1, wmax, size=d)) + [1] * d)


@pytest.mark.parametrize("bias", ["edge_weight", "neighbor_degree"])
def test_cached_walks_match_oracle(csaw, bias):
    for g in (inputs.rmat_csr(12, 16, 100, 12), inputs.rmat_csr(8, 8, 40, 1), star(70001, 3), ragged(3)):
        G = csaw.Graph(g.off, g.col, g.w)
        G.build_cdf(bias)
        starts = np.concatenate([np.arange(min(g.V, 5000), dtype=np.uint32),
                                 inputs.uniform_vertices(300, g.V, 3)])
        got = csaw.walk(G, starts, 20, bias, 77)
        assert np.array_equal(got, oracle.walk(g, starts, 20, bias, 77))
        G.close()


def ragged(seed, V=7000, wmax=2**20):
    """Rows of degree 0, 1, a few and a few hundred, and rows that straddle
    the 2048-edge scan tiles; the edge count is not a multiple of 8."""
    rng = np.random.default_rng(seed)
    kind = rng.integers(0, 10, size=V)
    deg = np.where(kind < 3, 0, np.where(kind < 6, 1, np.where(kind < 9, rng.integers(2, 30, size=V),
                                                               rng.integers(100, 700, size=V))))
    deg[[5, 17, V - 100]] = [2047, 2049, min(6500, V - 1)]
    if int(deg.sum()) % 8 == 0:
        deg[6] += 1
    cols = [np.sort(rng.choice(V, size=int(d), replace=False)) for d in deg]
    off = np.concatenate([[0], np.cumsum(deg)]).astype(np.uint64)
    col = np.concatenate(cols).astype(np.uint32)
    w = rng.integers(1, wmax, size=len(col)).astype(np.uint32)
    return inputs.CSRGraph(off, col, w)


@pytest.mark.parametrize("bias", ["edge_weight", "neighbor_degree"])
def test_walk_with_cumulative_array_built_per_call(csaw, bias):
    """build_cdf: the call builds the kind's cumulative array and its summary
    (segmented scan over edge tiles) and walks over it; paths equal the
    oracle's and those of the streaming walk, on graphs with empty rows, rows
    across tile boundaries, a 70,001-neighbour hub and tiny edge counts.
    Neighbour degree with an edge into a vertex without neighbours keeps the
    streaming path (the option is ignored) and stays exact."""
    tiny = inputs.csr_from_edges(4, [(0, 1), (0, 2), (0, 3), (1, 0), (2, 0), (2, 3), (3, 2)],
                                 [3, 1, 4, 1, 5, 9, 2])
    for g in (ragged(1), ragged(2, V=3000, wmax=7), inputs.rmat_csr(12, 16, 100, 12), star(70001, 3), tiny):
        G = csaw.Graph(g.off, g.col, g.w)
        starts = np.concatenate([np.arange(min(g.V, 7000), dtype=np.uint32), inputs.uniform_vertices(500, g.V, 4)])
        got = csaw.walk(G, starts, 24, bias, 31, build_cdf=True)
        assert np.array_equal(got, oracle.walk(g, starts, 24, bias, 31)), (g.V, g.E)
        assert np.array_equal(got, csaw.walk(G, starts, 24, bias, 31))
        G.close()


def test_walk_build_per_call_equals_cached_on_device(csaw):
    """Device inputs: the per-call array gives the paths of the graph's
    cached array, which the option then leaves in use."""
    import torch
    g = inputs.rmat_csr(14, 16, 255, 14)
    G = csaw.Graph(g.off, g.col, g.w)
    s = torch.from_numpy(np.arange(g.V, dtype=np.uint32).view(np.int32)).cuda()
    a = csaw.walk(G, s, 40, "edge_weight", 9, build_cdf=True)
    G.build_cdf("edge_weight")
    b = csaw.walk(G, s, 40, "edge_weight", 9, build_cdf=True)
    c = csaw.walk(G, s, 40, "edge_weight", 9)
    torch.cuda.synchronize()
    assert bool(torch.equal(a, b)) and bool(torch.equal(b, c))
    pick = inputs.uniform_vertices(400, g.V, 2).astype(np.int64)
    ref = oracle.walk(g, pick.astype(np.uint32), 40, "edge_weight", 9, walker_ids=pick.astype(np.uint64))
    assert np.array_equal(a[torch.from_numpy(pick).cuda()].cpu().numpy().view(np.uint32), ref)
    G.close()


@pytest.mark.parametrize("n,build", [(600_000, True), (1_100_003, False), (262_145, True)])
def test_host_walk_in_chunks_with_overlapped_copies(csaw, n, build):
    """Host inputs and outputs over a cumulative array: the walkers run in
    chunks (each chunk's rows copied out while the next walks), every walker
    keeping its own draws -- the paths equal the device call's and the
    oracle's, ragged last chunk included."""
    import torch
    g = inputs.rmat_csr(14, 16, 255, 14)
    G = csaw.Graph(g.off, g.col, g.w)
    if not build:
        G.build_cdf("edge_weight")
    starts = inputs.uniform_vertices(n, g.V, 6)
    host = csaw.walk(G, starts, 10, "edge_weight", 21, build_cdf=build)
    dev = csaw.walk(G, torch.from_numpy(starts.view(np.int32)).cuda(), 10, "edge_weight", 21, build_cdf=build)
    assert np.array_equal(host, dev.cpu().numpy().view(np.uint32))
    pick = np.unique(np.concatenate([np.arange(0, n, 9973), [n - 1, n // 2, 262_143, 262_144]])).astype(np.int64)
    pick = pick[pick < n]
    ref = oracle.walk(g, starts[pick], 10, "edge_weight", 21, walker_ids=pick.astype(np.uint64))
    assert np.array_equal(host[pick], ref)
    # page-locked host rows
    pinned = torch.empty((n, 11), dtype=torch.int32, pin_memory=True)
    got = csaw.walk(G, starts, 10, "edge_weight", 21, build_cdf=build, path=pinned.numpy().view(np.uint32))
    assert np.array_equal(got, host)
    bad = starts.copy()
    bad[n // 3] = g.V   # checked on the host while the chunks walk
    with pytest.raises(csaw.CsawError) as e:
        csaw.walk(G, bad, 10, "edge_weight", 21, build_cdf=build)
    assert e.value.status == csaw.ERR_INVALID
    G.close()


def test_walk_phase_times(csaw):
    """phase_ms: device times of the array's construction and of the walk,
    measured by events inside the call; the paths are unchanged."""
    import torch
    g = inputs.rmat_csr(14, 16, 255, 14)
    G = csaw.Graph(g.off, g.col, g.w)
    s = torch.from_numpy(np.arange(g.V, dtype=np.uint32).view(np.int32)).cuda()
    ref = csaw.walk(G, s, 30, "edge_weight", 4, build_cdf=True)
    ph = [0.0, 0.0]
    got = csaw.walk(G, s, 30, "edge_weight", 4, build_cdf=True, phase_ms=ph)
    assert bool(torch.equal(got, ref)) and ph[0] > 0 and ph[1] > 0
    host_ph = [0.0, 0.0]
    host = csaw.walk(G, np.arange(g.V, dtype=np.uint32), 30, "edge_weight", 4, build_cdf=True, phase_ms=host_ph)
    assert np.array_equal(host, ref.cpu().numpy().view(np.uint32)) and host_ph[0] > 0 and host_ph[1] > 0
    st_ph = [0.0, 0.0]   # streaming: nothing is built
    csaw.walk(G, s, 30, "edge_weight", 4, phase_ms=st_ph)
    assert st_ph[0] < ph[0] and st_ph[1] > 0
    G.close()


@pytest.mark.parametrize("bias", ["edge_weight", "uniform"])
def test_cached_walk_tile_boundaries_and_dead_ends(csaw, bias):
    """Path rows are staged 16 entries at a time per walker and written out
    by the warp: lengths around the tile size, ragged warps and walkers that
    stop at a vertex without neighbours."""
    dead = inputs.csr_from_edges(6, [(0, 1), (1, 2), (3, 4), (5, 0), (5, 3)], [2, 3, 5, 1, 7])
    for g in (dead, inputs.rmat_csr(8, 8, 40, 1)):
        G = csaw.Graph(g.off, g.col, g.w)
        if bias != "uniform":
            G.build_cdf(bias)
        for n in (1, 33, 70):
            starts = inputs.uniform_vertices(n, g.V, n)
            for length in (0, 1, 14, 15, 16, 17, 31, 32, 47, 80):
                got = csaw.walk(G, starts, length, bias, 5)
                assert np.array_equal(got, oracle.walk(g, starts, length, bias, 5)), (g.V, n, length)
        G.close()


def test_cached_walk_s20_subset(csaw):
    import torch
    wl = inputs.workload_walk_s20()
    g = wl.graph
    G = csaw.Graph(g.off, g.col, g.w)
    s = torch.from_numpy(wl.starts.view(np.int32)).cuda()
    streamed = csaw.walk(G, s, wl.length, wl.bias, wl.rng_seed)
    G.build_cdf("edge_weight")
    cached = csaw.walk(G, s, wl.length, wl.bias, wl.rng_seed)
    torch.cuda.synchronize()
    assert bool(torch.equal(streamed, cached))
    pick = inputs.uniform_vertices(300, g.V, 12).astype(np.int64)
    ref = oracle.walk(g, wl.starts[pick], wl.length, wl.bias, wl.rng_seed, walker_ids=pick.astype(np.uint64))
    assert np.array_equal(cached[torch.from_numpy(pick).cuda()].cpu().numpy().view(np.uint32), ref)
    G.close()


@pytest.mark.parametrize("bias", ["edge_weight", "neighbor_degree"])
@pytest.mark.parametrize("fanout", [[10, 5], [3, 3, 3], [ALL, 2], [40, 300]])
def test_cached_sampling_matches_oracle(csaw, bias, fanout):
    g = inputs.rmat_csr(12, 16, 100, 12)
    G = csaw.Graph(g.off, g.col, g.w)
    G.build_cdf(bias)
    seeds = inputs.uniform_vertices(300, g.V, 1)
    io = np.array([0, 1, 1, 50, 200, 300], dtype=np.uint64)
    res = csaw.sample(G, seeds, io, fanout, bias, 7)
    ref = oracle.sample(g, seeds, io, fanout, bias, 7)
    assert np.array_equal(res.dst, ref["dst"]) and np.array_equal(res.src, ref["src"])
    assert np.array_equal(res.edge_offsets, ref["edge_off"])
    # a plan created with the cached array gives the same
    plan = csaw.SamplePlan(G, 5, 300, fanout, bias)
    plan.run(seeds, io, 7)
    assert np.array_equal(plan.result().dst, ref["dst"])
    plan.close()
    G.close()


def test_cached_sampling_hubs_and_fallback(csaw):
    # hubs, k around PICK_MAX, and a heavy neighbour forcing updated sampling
    for d, k, heavy in ((70000, 25, False), (9000, 300, False), (3000, 255, False), (40, 25, True),
                        (9000, 30, True)):
        g = star(d, d % 11)
        if heavy:
            w = g.w.copy()
            w[d // 3] = 2**31          # row 0 holds the first d entries (CSR order)
            g = inputs.CSRGraph(g.off, g.col, w)
        G = csaw.Graph(g.off, g.col, g.w)
        G.build_cdf("edge_weight")
        seeds = np.zeros(6, dtype=np.uint32)
        io = np.arange(7, dtype=np.uint64)
        res = csaw.sample(G, seeds, io, [k], "edge_weight", 11)
        ref = oracle.sample(g, seeds, io, [k], "edge_weight", 11)
        assert np.array_equal(res.dst, ref["dst"]), (d, k, heavy)
        G.close()


def test_cached_array_not_used_with_zero_biases(csaw):
    g0 = inputs.rmat_csr(10, 8, 5, 3)
    w = g0.w.copy()
    w[np.random.default_rng(4).random(len(w)) < 0.3] = 0
    g = inputs.CSRGraph(g0.off, g0.col, w)
    G = csaw.Graph(g.off, g.col, g.w)
    G.build_cdf("edge_weight")
    seeds = inputs.uniform_vertices(200, g.V, 9)
    io = np.array([0, 100, 200], dtype=np.uint64)
    res = csaw.sample(G, seeds, io, [3, 2], "edge_weight", 5)
    ref = oracle.sample(g, seeds, io, [3, 2], "edge_weight", 5)
    assert np.array_equal(res.dst, ref["dst"])
    starts = np.arange(g.V, dtype=np.uint32)
    assert np.array_equal(csaw.walk(G, starts, 10, "edge_weight", 2), oracle.walk(g, starts, 10, "edge_weight", 2))
    G.drop_cdf("edge_weight")
    G.close()


def test_build_cdf_errors(csaw):
    g = inputs.rmat_csr(8, 8, 40, 1)
    G = csaw.Graph(g.off, g.col, None)
    with pytest.raises(csaw.CsawError) as e:
        G.build_cdf("edge_weight")
    assert e.value.status == csaw.ERR_INVALID
    with pytest.raises(csaw.CsawError) as e:
        G.build_cdf("node2vec")
    assert e.value.status == csaw.ERR_INVALID
    G.build_cdf("neighbor_degree")
    G.close()


def hubby_graph(seed=5):
    """Hubs joined to each other and to many low-degree vertices: node2vec
    steps alternate hub -> leaf -> hub, the case the intersection path serves."""
    rng = np.random.default_rng(seed)
    n_hub, n_leaf = 6, 20000
    und = set()
    for h in range(n_hub):
        for h2 in range(h + 1, n_hub):
            und.add((h, h2))
        for leaf in rng.choice(n_leaf, size=5000, replace=False):
            und.add((h, n_hub + int(leaf)))
    for _ in range(30000):
        a, b = (int(x) for x in rng.integers(n_hub, n_hub + n_leaf, 2))
        if a != b:
            und.add((min(a, b), max(a, b)))
    und = sorted(und)
    edges = und + [(b, a) for a, b in und]
    w = [int(x) for x in rng.integers(1, 50, size=len(und))]
    return inputs.csr_from_edges(n_hub + n_leaf, edges, w + w)


@pytest.mark.parametrize("mult", [(1, 2, 4), (3, 1, 2), (1, 2**20, 3)])
def test_node2vec_intersection_path_matches_oracle(csaw, mult):
    for g in (hubby_graph(), inputs.rmat_csr(12, 16, 40, 12)):
        G = csaw.Graph(g.off, g.col, g.w)
        G.build_cdf("edge_weight")
        starts = np.concatenate([np.arange(min(g.V, 3000), dtype=np.uint32),
                                 inputs.uniform_vertices(500, g.V, 1)])
        got = csaw.walk(G, starts, 15, "node2vec", 9, mult)
        assert np.array_equal(got, oracle.walk(g, starts, 15, "node2vec", 9, mult=mult))
        G.close()
    # no weights: the weight prefix sums are implicit
    g = hubby_graph(7)
    gu = inputs.CSRGraph(g.off, g.col, np.ones_like(g.w))
    G = csaw.Graph(g.off, g.col, None)
    starts = np.arange(3000, dtype=np.uint32)
    assert np.array_equal(csaw.walk(G, starts, 15, "node2vec", 4, mult),
                          oracle.walk(gu, starts, 15, "node2vec", 4, mult=mult))
    G.close()


def test_node2vec_s22_with_cached_weights(csaw):
    import torch
    wl = inputs.workload_node2vec_s22()
    g = wl.graph
    G = csaw.Graph(g.off, g.col, g.w)
    G.build_cdf("edge_weight")
    s = torch.from_numpy(wl.starts.view(np.int32)).cuda()
    path = csaw.walk(G, s, wl.length, wl.bias, wl.rng_seed, wl.n2v_mult)
    torch.cuda.synchronize()
    deg = np.diff(g.off)
    order = np.argsort(deg, kind="stable")
    pick = np.unique(np.concatenate([order[-60:], inputs.uniform_vertices(200, g.V, 5).astype(np.int64)]))
    ref = oracle.walk(g, wl.starts[pick], wl.length, wl.bias, wl.rng_seed, mult=wl.n2v_mult,
                      walker_ids=pick.astype(np.uint64))
    got = path[torch.from_numpy(pick).cuda()].cpu().numpy().view(np.uint32)
    assert np.array_equal(got, ref)
    G.close()
