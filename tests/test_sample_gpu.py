"""Layered sampling on the GPU through the C ABI, bit-exact against the oracle."""
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


def check_equal(res, ref, n_inst, depth):
    assert int(res.n_edges) == int(ref["edge_off"][-1])
    assert np.array_equal(res.edge_offsets, ref["edge_off"])
    assert np.array_equal(res.frontier_sizes, ref["fsize"][: depth * n_inst])
    assert np.array_equal(res.src, ref["src"])
    assert np.array_equal(res.dst, ref["dst"])


def run_both(csaw, g, seeds, io, fanout, bias, seed, G=None):
    own = G is None
    if own:
        G = csaw.Graph(g.off, g.col, g.w)
    res = csaw.sample(G, seeds, io, fanout, bias, seed)
    ref = oracle.sample(g, seeds, io, fanout, bias, seed)
    if own:
        G.close()
    return res, ref


@pytest.mark.parametrize("bias", ["uniform", "edge_weight", "neighbor_degree"])
@pytest.mark.parametrize("fanout", [[10, 5], [1], [3, 3, 3], [ALL, 2], [40, 300]])
def test_sample_small_rmat(csaw, bias, fanout):
    g = inputs.rmat_csr(12, 16, 100, 12)
    seeds = inputs.uniform_vertices(300, g.V, 1)
    io = np.array([0, 1, 1, 50, 200, 300], dtype=np.uint64)   # includes an empty instance
    res, ref = run_both(csaw, g, seeds, io, fanout, bias, 7)
    check_equal(res, ref, 5, len(fanout))


def test_sample_workload_s12(csaw):
    """RMAT s12 ef16, 256 seeds, depth 2, fanout [10, 5], edge weight, seed 1: full output."""
    wl = inputs.workload_sample_s12()
    res, ref = run_both(csaw, wl.graph, wl.seeds, wl.inst_offsets, wl.fanout, wl.bias, wl.rng_seed)
    check_equal(res, ref, 1, 2)
    assert res.n_edges > 2000


def test_sample_exact_exclusion_fallback(csaw):
    # Centre 0 with one heavy neighbour (weight 2^31) and light ones: after the
    # heavy pick, repeated sampling almost never hits a light one, so the
    # updated-sampling fallback (after 1024 attempts) supplies the rest.
    for d, k in ((6, 4), (40, 25), (300, 200), (9000, 30)):
        w = [1] * d
        w[d // 3] = 2**31
        edges = [(0, j + 1) for j in range(d)] + [(j + 1, 0) for j in range(d)]
        g = inputs.csr_from_edges(d + 1, edges, w + [1] * d)
        seeds = np.zeros(8, dtype=np.uint32)
        io = np.arange(9, dtype=np.uint64)   # 8 instances of the same seed
        res, ref = run_both(csaw, g, seeds, io, [k], "edge_weight", 3)
        check_equal(res, ref, 8, 1)


def test_sample_hub_tiers(csaw):
    # degrees around the warp/CTA split and above the CTA shared-memory limit
    rng = np.random.default_rng(2)
    for d in (255, 256, 257, 2000, 8192, 8193, 70000):
        w = rng.integers(1, 1000, size=d)
        edges = [(0, j + 1) for j in range(d)] + [(j + 1, 0) for j in range(d)]
        g = inputs.csr_from_edges(d + 1, edges, list(w) + [1] * d)
        seeds = np.zeros(6, dtype=np.uint32)
        io = np.arange(7, dtype=np.uint64)
        for k in (1, 25, d - 1 if d <= 8193 else 600):
            res, ref = run_both(csaw, g, seeds, io, [k], "edge_weight", 11)
            check_equal(res, ref, 6, 1)


def test_sample_zero_biases(csaw):
    # zero weights: never picked; "take all" counts positive biases only
    rng = np.random.default_rng(4)
    g0 = inputs.rmat_csr(10, 8, 5, 3)
    w = g0.w.copy()
    w[rng.random(len(w)) < 0.3] = 0
    g = inputs.CSRGraph(g0.off, g0.col, w)
    seeds = inputs.uniform_vertices(200, g.V, 9)
    io = np.array([0, 100, 200], dtype=np.uint64)
    for fan in ([3, 2], [ALL, 1], [20]):
        res, ref = run_both(csaw, g, seeds, io, fan, "edge_weight", 5)
        check_equal(res, ref, 2, len(fan))
    # neighbour-degree bias on a directed graph with sink vertices (degree 0)
    edges = [(0, 1), (0, 2), (0, 3), (0, 4), (1, 2), (2, 0), (3, 4)]
    gd = inputs.csr_from_edges(6, edges)
    res, ref = run_both(csaw, gd, np.array([0, 1, 3, 5], dtype=np.uint32),
                        np.array([0, 4], dtype=np.uint64), [2, 2], "neighbor_degree", 1)
    check_equal(res, ref, 1, 2)


def test_sample_many_instances_and_duplicates(csaw):
    g = inputs.rmat_csr(14, 16, 50, 14)
    sizes = inputs.loguniform_sizes(300, 0.0, 7.0, 5)
    seeds, io = inputs.distinct_seeds(sizes, g.V, 6)
    seeds[::7] = seeds[0]                     # duplicates inside instances
    res, ref = run_both(csaw, g, seeds, io, [25, 10], "neighbor_degree", 4)
    check_equal(res, ref, 300, 2)


def test_sample_device_inputs_match_host(csaw):
    import torch
    g = inputs.rmat_csr(12, 16, 100, 12)
    seeds = inputs.uniform_vertices(500, g.V, 2)
    io = np.array([0, 250, 500], dtype=np.uint64)
    G = csaw.Graph(g.off, g.col, g.w)
    host = csaw.sample(G, seeds, io, [5, 4], "edge_weight", 9)
    ds = torch.from_numpy(seeds.view(np.int32)).cuda()
    dio = torch.from_numpy(io.view(np.int64)).cuda()
    dev = csaw.sample(G, ds, dio, [5, 4], "edge_weight", 9, to_host=False)
    torch.cuda.synchronize()
    src = np.concatenate([t.cpu().numpy().view(np.uint32) for t in dev.src])
    dst = np.concatenate([t.cpu().numpy().view(np.uint32) for t in dev.dst])
    assert np.array_equal(src, host.src) and np.array_equal(dst, host.dst)
    assert np.array_equal(dev.edge_offsets, host.edge_offsets)
    G.close()


def test_sample_errors(csaw):
    g = inputs.rmat_csr(8, 8, 40, 1)
    G = csaw.Graph(g.off, g.col, g.w)
    io = np.array([0, 1], dtype=np.uint64)
    with pytest.raises(csaw.CsawError) as e:
        csaw.sample(G, np.array([g.V], dtype=np.uint32), io, [2], "edge_weight", 1)
    assert e.value.status == csaw.ERR_INVALID
    with pytest.raises(csaw.CsawError) as e:
        csaw.sample(G, np.array([0], dtype=np.uint32), io, [2], "node2vec", 1)
    assert e.value.status == csaw.ERR_INVALID
    with pytest.raises(csaw.CsawError) as e:
        csaw.sample(G, np.array([0], dtype=np.uint32), io, [], "edge_weight", 1)
    assert e.value.status == csaw.ERR_INVALID
    with pytest.raises(csaw.CsawError) as e:
        csaw.sample(G, np.array([0, 1], dtype=np.uint32), np.array([0, 2, 1], dtype=np.uint64), [2],
                    "edge_weight", 1)
    assert e.value.status == csaw.ERR_INVALID
    # no seeds at all is a valid, empty sample
    r = csaw.sample(G, np.zeros(0, dtype=np.uint32), np.array([0, 0], dtype=np.uint64), [3, 3],
                    "edge_weight", 1)
    assert r.n_edges == 0
    G.close()


def instance_subset_oracle(g, seeds, io, pick, fanout, bias, seed):
    """Oracle on chosen instances only, each kept at its own index (the
    others empty); instances are independent, so these rows are exact."""
    n = len(io) - 1
    sizes = np.zeros(n, dtype=np.uint64)
    parts = []
    for i in sorted(pick):
        sizes[i] = io[i + 1] - io[i]
        parts.append(seeds[io[i]:io[i + 1]])
    sub_io = np.zeros(n + 1, dtype=np.uint64)
    sub_io[1:] = np.cumsum(sizes)
    return oracle.sample(g, np.concatenate(parts), sub_io, fanout, bias, seed)


@pytest.fixture(scope="module")
def s24():
    """4096 instances of log-uniform [64, 8192) seeds on RMAT s24 ef16, fanout
    [25, 10], neighbour-degree bias."""
    return inputs.workload_batched_s24()


def s24_pick(wl, g):
    """A stratified instance subset: the smallest and largest instances, the
    instance holding the highest-degree seed, fixed ids and a uniform sample."""
    n = len(wl.inst_offsets) - 1
    sizes = np.diff(wl.inst_offsets).astype(np.int64)
    deg = np.diff(g.off).astype(np.int64)
    hub_seed = int(np.argmax(deg[wl.seeds.astype(np.int64)]))
    hub_inst = int(np.searchsorted(wl.inst_offsets, hub_seed, side="right")) - 1
    rnd = inputs.uniform_vertices(4, n, 41).astype(np.int64)
    return sorted(set([int(np.argmin(sizes)), int(np.argmax(sizes)), hub_inst, 17, 2048, n - 1]
                      + rnd.tolist()))


def check_subset(res, ref, n, pick, depth):
    for lvl in range(depth):
        for i in pick:
            a0, a1 = res.edge_offsets[lvl * n + i], res.edge_offsets[lvl * n + i + 1]
            b0, b1 = ref["edge_off"][lvl * n + i], ref["edge_off"][lvl * n + i + 1]
            assert np.array_equal(res.dst[a0:a1], ref["dst"][b0:b1]), (lvl, i)
            assert np.array_equal(res.src[a0:a1], ref["src"][b0:b1]), (lvl, i)
            assert res.frontier_sizes[lvl * n + i] == ref["fsize"][lvl * n + i]


def test_sample_batched_s24_subset(csaw, s24):
    """The full batched csaw_sample run, checked against the oracle on a
    stratified subset of instances and by invariants."""
    wl = s24
    g = wl.graph
    G = csaw.Graph(g.off, g.col, g.w)
    res = csaw.sample(G, wl.seeds, wl.inst_offsets, wl.fanout, wl.bias, wl.rng_seed)
    n = len(wl.inst_offsets) - 1
    pick = s24_pick(wl, g)
    ref = instance_subset_oracle(g, wl.seeds, wl.inst_offsets, pick, wl.fanout, wl.bias, wl.rng_seed)
    check_subset(res, ref, n, pick, 2)
    # layer 0 frontier sizes are the distinct seeds
    assert np.array_equal(res.frontier_sizes[:n], np.diff(wl.inst_offsets))
    G.close()


def test_sample_plan_batched_s24_subset(csaw, s24):
    """The batched plan (one CUDA graph over all 4096 instances and both
    layers) -- the launch the batched throughput is measured on -- against
    the oracle on a stratified instance subset, and against csaw_sample on
    its whole output."""
    wl = s24
    g = wl.graph
    G = csaw.Graph(g.off, g.col, g.w)
    n = len(wl.inst_offsets) - 1
    plan = csaw.SamplePlan(G, n, len(wl.seeds), wl.fanout, wl.bias)
    plan.run(wl.seeds, wl.inst_offsets, wl.rng_seed)
    res = plan.result()
    pick = s24_pick(wl, g)
    ref = instance_subset_oracle(g, wl.seeds, wl.inst_offsets, pick, wl.fanout, wl.bias, wl.rng_seed)
    check_subset(res, ref, n, pick, 2)
    plan.close()
    whole = csaw.sample(G, wl.seeds, wl.inst_offsets, wl.fanout, wl.bias, wl.rng_seed)
    assert np.array_equal(res.edge_offsets, whole.edge_offsets)
    assert np.array_equal(res.frontier_sizes, whole.frontier_sizes)
    assert np.array_equal(res.src, whole.src) and np.array_equal(res.dst, whole.dst)
    G.close()


def test_sample_plan_batched_s24_cached_subset(csaw, s24):
    """The batched plan over the cached cumulative array (hub items in
    vertex order, summary searches) against the oracle on the stratified
    instance subset."""
    wl = s24
    g = wl.graph
    G = csaw.Graph(g.off, g.col, g.w)
    G.build_cdf(wl.bias)
    n = len(wl.inst_offsets) - 1
    plan = csaw.SamplePlan(G, n, len(wl.seeds), wl.fanout, wl.bias)
    plan.run(wl.seeds, wl.inst_offsets, wl.rng_seed)
    res = plan.result()
    plan.close()
    pick = s24_pick(wl, g)
    ref = instance_subset_oracle(g, wl.seeds, wl.inst_offsets, pick, wl.fanout, wl.bias, wl.rng_seed)
    check_subset(res, ref, n, pick, 2)
    G.close()


def test_sample_shared_hub_arrays(csaw):
    """Hub vertices that recur in many instances' frontiers share one
    cumulative array per layer: degrees around the warp/CTA build split
    (2048) and the shared-memory limit (8192), many instances seeded on the
    same hubs, duplicated hubs inside an instance, both static biases and a
    low warp threshold -- bit-exact against the oracle."""
    rng = np.random.default_rng(12)
    # three stars whose leaves are shared, plus a ring through the leaves
    centres = [(0, 2047), (1, 2049), (2, 9000)]
    n_leaf = 9000
    V = 3 + n_leaf
    edges, w = [], []
    for c, d in centres:
        for j in range(d):
            u = 3 + j
            edges += [(c, u), (u, c)]
            w += [int(rng.integers(1, 300))] * 2
    for j in range(n_leaf):
        a, b = 3 + j, 3 + (j + 1) % n_leaf
        edges += [(a, b), (b, a)]
        w += [int(rng.integers(1, 300))] * 2
    key = {}
    for (a, b), x in zip(edges, w):
        key[(a, b)] = x
    es = sorted(key)
    g = inputs.csr_from_edges(V, es, [key[e] for e in es])
    n_inst = 40
    seeds = np.concatenate([np.concatenate([np.array([0, 1, 2], dtype=np.uint32), inputs.uniform_vertices(5, V, i)])
                            for i in range(n_inst)]).astype(np.uint32)
    io = np.arange(0, 8 * n_inst + 1, 8, dtype=np.uint64)
    G = csaw.Graph(g.off, g.col, g.w)
    for bias in ("edge_weight", "neighbor_degree"):
        for fan in ([25, 10], [3, 40, 2]):
            ref = oracle.sample(g, seeds, io, fan, bias, 5)
            check_equal(csaw.sample(G, seeds, io, fan, bias, 5), ref, n_inst, len(fan))
            csaw.set_select_tuning(G, bias, 32, 0)
            check_equal(csaw.sample(G, seeds, io, fan, bias, 5), ref, n_inst, len(fan))
            plan = csaw.SamplePlan(G, n_inst, len(seeds), fan, bias)
            plan.run(seeds, io, 5)
            check_equal(plan.result(), ref, n_inst, len(fan))
            plan.close()
            csaw.set_select_tuning(G, bias, 0, 0)
        # the cached array: hub items drawn in vertex order from it
        G.build_cdf(bias)
        for fan in ([25, 10], [3, 40, 2]):
            ref = oracle.sample(g, seeds, io, fan, bias, 5)
            check_equal(csaw.sample(G, seeds, io, fan, bias, 5), ref, n_inst, len(fan))
            csaw.set_select_tuning(G, bias, 32, 0)
            plan = csaw.SamplePlan(G, n_inst, len(seeds), fan, bias)
            plan.run(seeds, io, 5)
            check_equal(plan.result(), ref, n_inst, len(fan))
            plan.close()
            csaw.set_select_tuning(G, bias, 0, 0)
        G.drop_cdf(bias)
    G.close()
