"""Walks on the GPU through the C ABI, bit-exact against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2009_09103_gb300 import inputs

pytestmark = pytest.mark.gpu
NONE = 0xFFFFFFFF


@pytest.fixture(scope="module")
def csaw():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_09103_gb300 import build
    build.build()
    from paper_2009_09103_gb300 import csaw as c
    return c


def gpu_walk(csaw, g, starts, length, bias, seed, mult=(1, 1, 1)):
    import torch
    G = csaw.Graph(g.off, g.col, g.w)
    s = torch.from_numpy(np.asarray(starts, dtype=np.uint32).view(np.int32)).cuda()
    path = csaw.walk(G, s, length, bias, seed, mult)
    torch.cuda.synchronize()
    out = path.cpu().numpy().view(np.uint32)
    G.close()
    return out


def small_graphs():
    out = {}
    und = [(0, 1, 1), (0, 2, 1), (1, 2, 1), (0, 3, 3)]
    e = [(a, b) for a, b, _ in und] + [(b, a) for a, b, _ in und]
    out["triangle_pendant"] = inputs.csr_from_edges(4, e, [w for *_, w in und] * 2)
    out["dead_end_zero_w"] = inputs.csr_from_edges(5, [(0, 1), (1, 2), (3, 4)], [1, 1, 0])
    out["rmat_s8"] = inputs.rmat_csr(8, 8, 40, 1)
    out["rmat_s12"] = inputs.rmat_csr(12, 16, 100, 12)
    return out


BIASES = [("uniform", (1, 1, 1)), ("edge_weight", (1, 1, 1)), ("neighbor_degree", (1, 1, 1)),
          ("node2vec", (1, 2, 4)), ("node2vec", (3, 1, 2))]


@pytest.mark.parametrize("gname", ["triangle_pendant", "dead_end_zero_w", "rmat_s8", "rmat_s12"])
@pytest.mark.parametrize("bias,mult", BIASES)
def test_walk_bit_exact_small(csaw, gname, bias, mult):
    g = small_graphs()[gname]
    starts = np.concatenate([np.arange(g.V, dtype=np.uint32),
                             inputs.uniform_vertices(300, g.V, 3)])
    ref = oracle.walk(g, starts, 25, bias, 1234, mult=mult)
    got = gpu_walk(csaw, g, starts, 25, bias, 1234, mult)
    assert np.array_equal(got, ref)


def test_walk_hubs_many_chunks(csaw):
    # A star whose centre has more neighbours than fit in one chunk table slot
    # per round (forces the multi-round-per-chunk path), plus ragged tails.
    rng = np.random.default_rng(7)
    for d in (1, 31, 32, 33, 255, 256, 257, 8191, 70001, 300007):
        edges = [(0, j + 1) for j in range(d)] + [(j + 1, 0) for j in range(d)]
        w = list(rng.integers(1, 2**20, size=d)) + [1] * d
        g = inputs.csr_from_edges(d + 1, edges, w)
        starts = np.zeros(64, dtype=np.uint32)
        for bias in ("edge_weight", "uniform"):
            ref = oracle.walk(g, starts, 3, bias, 99)
            got = gpu_walk(csaw, g, starts, 3, bias, 99)
            assert np.array_equal(got, ref), (d, bias)


def test_walk_host_buffers_match_device(csaw):
    g = inputs.rmat_csr(12, 16, 100, 12)
    starts = inputs.uniform_vertices(5000, g.V, 2)
    G = csaw.Graph(g.off, g.col, g.w)
    host = csaw.walk(G, starts, 30, "edge_weight", 5)
    dev = gpu_walk(csaw, g, starts, 30, "edge_weight", 5)
    assert np.array_equal(host, dev)
    assert np.array_equal(host, oracle.walk(g, starts, 30, "edge_weight", 5))


def test_walk_errors(csaw):
    g = inputs.rmat_csr(8, 8, 40, 1)
    G = csaw.Graph(g.off, g.col, g.w)
    with pytest.raises(csaw.CsawError) as e:
        csaw.walk(G, np.array([g.V], dtype=np.uint32), 3, "edge_weight", 1)
    assert e.value.status == csaw.ERR_INVALID
    with pytest.raises(csaw.CsawError) as e:
        csaw.walk(G, np.array([0], dtype=np.uint32), 3, "node2vec", 1, mult=(1, 2**30, 4))
    assert e.value.status == csaw.ERR_OVERFLOW
    with pytest.raises(csaw.CsawError) as e:
        csaw.walk(G, np.array([0], dtype=np.uint32), 3, csaw.make_bias(9), 1)
    assert e.value.status == csaw.ERR_INVALID
    # malformed CSR: unsorted row
    with pytest.raises(csaw.CsawError) as e:
        csaw.Graph(np.array([0, 2, 2], dtype=np.uint64), np.array([1, 0], dtype=np.uint32))
    assert e.value.status == csaw.ERR_INVALID
    with pytest.raises(csaw.CsawError) as e:
        csaw.Graph(np.array([0, 1, 1], dtype=np.uint64), np.array([5], dtype=np.uint32))
    assert e.value.status == csaw.ERR_INVALID
    # empty walk is fine
    assert csaw.walk(G, np.zeros(0, dtype=np.uint32), 3, "edge_weight", 1).shape == (0, 4)


def _adjacent_all(torch, g, path_t):
    """Every consecutive non-sentinel pair is an edge; sentinels only follow
    dead ends.  Edge keys src<<32|dst are sorted in CSR order."""
    dev = path_t.device
    off = torch.from_numpy(g.off.astype(np.int64)).to(dev)
    col = torch.from_numpy(g.col.astype(np.int64)).to(dev)
    src = torch.repeat_interleave(torch.arange(g.V, device=dev), off[1:] - off[:-1])
    keys = (src << 32) | col
    p = path_t.to(torch.int64) & 0xFFFFFFFF
    a, b = p[:, :-1], p[:, 1:]
    real = b != NONE
    q = ((a << 32) | b)[real]
    pos = torch.searchsorted(keys, q).clamp(max=keys.numel() - 1)
    ok_edges = bool((keys[pos] == q).all())
    # a sentinel after a real vertex only at a dead end (degree 0 for edge weights >= 1)
    stop = (~real) & (a != NONE)
    deg = off[1:] - off[:-1]
    ok_stops = bool((deg[a[stop]] == 0).all())
    after_none = (a == NONE) & real
    return ok_edges, ok_stops, not bool(after_none.any())


def oracle_walk_sharded(g, starts, length, bias, seed, mult=(1, 1, 1)):
    """The whole path matrix from the single-threaded oracle, run as one copy
    per host core over disjoint walker ranges, each walker keyed by its own
    index (walks are independent, so the shards join into the full output)."""
    import concurrent.futures as cf
    import os
    n = len(starts)
    threads = os.cpu_count() or 1
    bounds = np.linspace(0, n, 8 * threads + 1).astype(np.int64)
    out = np.empty((n, length + 1), dtype=np.uint32)

    def run(i):
        a, b = int(bounds[i]), int(bounds[i + 1])
        if b > a:
            out[a:b] = oracle.walk(g, starts[a:b], length, bias, seed, mult=mult,
                                   walker_ids=np.arange(a, b, dtype=np.uint64))
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(run, range(len(bounds) - 1)))
    return out


def test_walk_rmat_s20_full_size(csaw):
    """The weighted-walk workload at full size: RMAT s20 ef16, one walker per
    vertex, length 80, in the launch configuration the benchmark times.  The
    whole 1,048,576 x 81 path matrix is bit-exact against the oracle; the
    invariants hold on all of it."""
    import torch
    wl = inputs.workload_walk_s20()
    g = wl.graph
    G = csaw.Graph(g.off, g.col, g.w)
    s = torch.from_numpy(wl.starts.view(np.int32)).cuda()
    path = csaw.walk(G, s, wl.length, wl.bias, wl.rng_seed)
    torch.cuda.synchronize()
    ok_e, ok_s, ok_n = _adjacent_all(torch, g, path)
    assert ok_e and ok_s and ok_n
    ref = oracle_walk_sharded(g, wl.starts, wl.length, wl.bias, wl.rng_seed)
    got = path.cpu().numpy().view(np.uint32)
    assert got.shape == ref.shape == (g.V, wl.length + 1)
    bad = np.flatnonzero((got != ref).any(axis=1))
    assert len(bad) == 0, f"{len(bad)} walkers differ, first {bad[:5]}"
    G.close()


def test_walk_node2vec_s22_subset(csaw):
    """node2vec p=2, q=0.5 on RMAT s22 ef32 at full size; stratified subset
    bit-exact against the oracle."""
    import torch
    wl = inputs.workload_node2vec_s22()
    g = wl.graph
    G = csaw.Graph(g.off, g.col, g.w)
    s = torch.from_numpy(wl.starts.view(np.int32)).cuda()
    path = csaw.walk(G, s, wl.length, wl.bias, wl.rng_seed, wl.n2v_mult)
    torch.cuda.synchronize()
    ok_e, ok_s, ok_n = _adjacent_all(torch, g, path)
    assert ok_e and ok_s and ok_n
    deg = np.diff(g.off)
    order = np.argsort(deg, kind="stable")
    pick = np.unique(np.concatenate([order[-60:], order[len(order) // 2: len(order) // 2 + 60],
                                     inputs.uniform_vertices(120, g.V, 5).astype(np.int64)]))
    ref = oracle.walk(g, wl.starts[pick], wl.length, wl.bias, wl.rng_seed, mult=wl.n2v_mult,
                      walker_ids=pick.astype(np.uint64))
    got = path[torch.from_numpy(pick).cuda()].cpu().numpy().view(np.uint32)
    assert np.array_equal(got, ref)
    G.close()


@pytest.mark.parametrize("wmax", [2**23 + 5, 2**31])
def test_walk_wide_sums(csaw, wmax):
    """Biases large enough that a 512-neighbour round overflows 32 bits take
    the 64-bit path; results stay bit-exact."""
    rng = np.random.default_rng(wmax % 97)
    g0 = inputs.rmat_csr(11, 16, 50, 5)
    w = rng.integers(wmax // 2, wmax, size=g0.E, dtype=np.uint64).astype(np.uint32)
    g = inputs.CSRGraph(g0.off, g0.col, w)
    starts = np.arange(g.V, dtype=np.uint32)
    assert np.array_equal(gpu_walk(csaw, g, starts, 12, "edge_weight", 3),
                          oracle.walk(g, starts, 12, "edge_weight", 3))
    d = 70001
    edges = [(0, j + 1) for j in range(d)] + [(j + 1, 0) for j in range(d)]
    ws = list(rng.integers(1, wmax, size=d)) + [1] * d
    gs = inputs.csr_from_edges(d + 1, edges, ws)
    z = np.zeros(40, dtype=np.uint32)
    assert np.array_equal(gpu_walk(csaw, gs, z, 3, "edge_weight", 8), oracle.walk(gs, z, 3, "edge_weight", 8))


def test_walk_node2vec_wide_multipliers(csaw):
    g = inputs.rmat_csr(11, 16, 40, 6)
    starts = np.arange(g.V, dtype=np.uint32)
    mult = (1, 2**20, 3)
    assert np.array_equal(gpu_walk(csaw, g, starts, 10, "node2vec", 4, mult),
                          oracle.walk(g, starts, 10, "node2vec", 4, mult=mult))


def test_walk_length_zero_and_one(csaw):
    g = inputs.rmat_csr(10, 8, 50, 3)
    starts = inputs.uniform_vertices(100, g.V, 4)
    for L in (0, 1):
        for bias in ("edge_weight", "uniform", "node2vec"):
            got = gpu_walk(csaw, g, starts, L, bias, 5, (1, 2, 4))
            assert got.shape == (100, L + 1)
            assert np.array_equal(got, oracle.walk(g, starts, L, bias, 5, mult=(1, 2, 4)))


def dense_overlap_graph(seed=11):
    """Three hubs joined by heavy edges; hub 0 is adjacent to 20,000 leaves,
    hubs 1 and 2 to random subsets of them (3,000 and 600).  A node2vec step at
    hub 1 or 2 after hub 0 tests membership against a previous list far denser
    than each 128-neighbour tile, which slides the staged window of N(prev)
    and then falls back to global searches."""
    rng = np.random.default_rng(seed)
    n_hub, n_leaf = 3, 20000
    und = {(0, 1): 10**6, (0, 2): 10**6, (1, 2): 10**6}
    leaves = n_hub + np.arange(n_leaf)
    for h, size in ((0, n_leaf), (1, 3000), (2, 600)):
        for leaf in rng.choice(leaves, size=size, replace=False):
            und[(h, int(leaf))] = int(rng.integers(1, 50))
    for _ in range(20000):
        a, b = (int(x) for x in rng.integers(n_hub, n_hub + n_leaf, 2))
        if a != b:
            und[(min(a, b), max(a, b))] = int(rng.integers(1, 50))
    items = sorted(und.items())
    edges = [e for e, _ in items] + [(b, a) for (a, b), _ in items]
    w = [x for _, x in items]
    return inputs.csr_from_edges(n_hub + n_leaf, edges, w + w)


@pytest.mark.parametrize("mult", [(1, 2, 4), (3, 1, 2), (1, 4000, 3)])   # 10**6 * 4000 < 2**32
def test_walk_node2vec_dense_previous_list(csaw, mult):
    g = dense_overlap_graph()
    starts = np.concatenate([np.repeat(np.arange(3, dtype=np.uint32), 400),
                             inputs.uniform_vertices(800, g.V, 5)])
    got = gpu_walk(csaw, g, starts, 12, "node2vec", 21, mult)
    assert np.array_equal(got, oracle.walk(g, starts, 12, "node2vec", 21, mult=mult))
    gu = inputs.CSRGraph(g.off, g.col, np.ones_like(g.w))
    got = gpu_walk(csaw, inputs.CSRGraph(g.off, g.col, None), starts, 12, "node2vec", 22, mult)
    assert np.array_equal(got, oracle.walk(gu, starts, 12, "node2vec", 22, mult=mult))


Q32_ALWAYS = 0xFFFFFFFF


@pytest.mark.parametrize("mode", ["restart", "jump"])
@pytest.mark.parametrize("bias,mult", [("uniform", (1, 1, 1)), ("edge_weight", (1, 1, 1)),
                                       ("neighbor_degree", (1, 1, 1)), ("node2vec", (1, 2, 4))])
@pytest.mark.parametrize("q32", [0, 1 << 30, 3 << 30, Q32_ALWAYS])
def test_walk_teleport_bit_exact(csaw, mode, bias, mult, q32):
    # random walk with restart / with jump (Sec. II-A); graphs with dead ends
    for g in (small_graphs()["dead_end_zero_w"], small_graphs()["rmat_s12"]):
        starts = np.concatenate([np.arange(min(g.V, 500), dtype=np.uint32),
                                 inputs.uniform_vertices(300, g.V, 3)])
        G = csaw.Graph(g.off, g.col, g.w)
        got = csaw.walk(G, starts, 40, bias, 77, mult, teleport=mode, teleport_q32=q32)
        G.close()
        ref = oracle.walk(g, starts, 40, bias, 77, mult=mult, teleport=mode, teleport_q32=q32)
        assert np.array_equal(got, ref), (mode, bias, q32)


def test_walk_teleport_hubs_and_device_buffers(csaw):
    import torch
    rng = np.random.default_rng(3)
    d = 70001
    edges = [(0, j + 1) for j in range(d)] + [(j + 1, 0) for j in range(d)]
    w = list(rng.integers(1, 2**20, size=d)) + [1] * d
    g = inputs.csr_from_edges(d + 1, edges, w)
    starts = np.concatenate([np.zeros(64, dtype=np.uint32), inputs.uniform_vertices(64, g.V, 2)])
    G = csaw.Graph(g.off, g.col, g.w)
    G.build_cdf("edge_weight")   # a teleporting walk streams even with the cached array
    for mode in ("restart", "jump"):
        got = csaw.walk(G, torch.from_numpy(starts.view(np.int32)).cuda(), 20, "edge_weight", 5,
                        teleport=mode, teleport_q32=1 << 31).cpu().numpy().view(np.uint32)
        ref = oracle.walk(g, starts, 20, "edge_weight", 5, teleport=mode, teleport_q32=1 << 31)
        assert np.array_equal(got, ref), mode
    with pytest.raises(csaw.CsawError):
        csaw.lib()   # the library is loaded
        bad = csaw.WalkOpts(7, 0)
        b = csaw.make_bias("edge_weight")
        csaw._check(csaw.lib().csaw_walk_ex(G.handle, csaw._ptr(starts), len(starts), 3, ctypes_byref(b), 1,
                                             csaw._ptr(np.empty((len(starts), 4), dtype=np.uint32)),
                                             csaw.MEM_HOST, None, ctypes_byref(bad)))
    G.close()


def ctypes_byref(x):
    import ctypes
    return ctypes.byref(x)
