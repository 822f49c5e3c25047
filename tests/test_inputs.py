"""The synthetic input generator: RMAT graphs and seed sets (CPU)."""
import numpy as np

from paper_2009_09103_gb300 import inputs


def _check_csr(g, wmax):
    V = g.V
    off = g.off.astype(np.int64)
    assert off[0] == 0 and off[-1] == g.E and np.all(np.diff(off) >= 0)
    src = np.repeat(np.arange(V, dtype=np.int64), np.diff(off))
    col = g.col.astype(np.int64)
    assert np.all(col < V)
    assert not np.any(src == col), "self-loop"
    # rows strictly ascending (sorted, no duplicates)
    same_row = src[1:] == src[:-1]
    assert np.all(col[1:][same_row] > col[:-1][same_row])
    # symmetric with equal weights both ways
    fwd = src * V + col
    rev = col * V + src
    order = np.argsort(rev)
    assert np.array_equal(np.sort(fwd), rev[order])
    pos = np.searchsorted(fwd, rev)
    assert np.array_equal(g.w[pos], g.w)
    assert g.w.min() >= 1 and g.w.max() <= wmax


def test_rmat_small_is_valid_csr():
    g = inputs.rmat_csr(10, 8, 37, seed=3)
    _check_csr(g, 37)
    deg = np.diff(g.off)
    assert deg.max() > 8 * deg.mean()          # power-law: hubs well above the mean
    assert g.E > 0.7 * 2 * 8 * g.V              # few duplicates at this scale


def test_rmat_deterministic_and_seed_dependent():
    a = inputs.rmat_csr(9, 4, 10, seed=1)
    b = inputs.rmat_csr(9, 4, 10, seed=1, threads=3)
    c = inputs.rmat_csr(9, 4, 10, seed=2)
    assert np.array_equal(a.off, b.off) and np.array_equal(a.col, b.col) and np.array_equal(a.w, b.w)
    assert not np.array_equal(a.col, c.col)


def test_rmat_hubs_are_spread_over_ids():
    g = inputs.rmat_csr(12, 16, 100, seed=12)
    deg = np.diff(g.off)
    top = np.argsort(deg)[-16:]
    assert top.max() > g.V // 4   # the label permutation moved hubs away from low ids


def test_workload_sample_s12_shape():
    wl = inputs.workload_sample_s12()
    _check_csr(wl.graph, 100)
    assert wl.graph.V == 4096 and wl.graph.E <= 131072
    assert len(wl.seeds) == 256 and wl.seeds.max() < 4096
    assert wl.fanout == [10, 5]


def test_seed_sets():
    sizes = inputs.loguniform_sizes(4096, 6.0, 7.0, seed=24, stream=4)
    assert sizes.min() >= 64 and sizes.max() < 8192
    # log-uniform: about half the instances below 2^9.5
    frac = np.mean(sizes < 2 ** 9.5)
    assert 0.45 < frac < 0.55
    seeds, offs = inputs.distinct_seeds(sizes[:50], 1 << 16, seed=1)
    for i in range(50):
        s = seeds[offs[i]:offs[i + 1]]
        assert len(np.unique(s)) == len(s) == sizes[i]
        assert s.max() < (1 << 16)
    u = inputs.uniform_vertices(100000, 1000, seed=9)
    counts = np.bincount(u, minlength=1000)
    assert counts.min() > 50 and counts.max() < 160


def test_parallel_csr_build_equals_serial_build():
    import ctypes
    lib = inputs._load()
    for scale, ef in ((9, 8), (14, 16)):
        V, m = 1 << scale, ef << scale
        src = np.empty(m, np.uint32)
        dst = np.empty(m, np.uint32)
        lib.csaw_gen_rmat_draws(scale, m, 0.57, 0.19, 0.19, 3, 4, inputs._p(src), inputs._p(dst))
        outs = []
        for fn, extra in ((lib.csaw_gen_build_csr, ()), (lib.csaw_gen_build_csr_mt, (7,))):
            off = np.empty(V + 1, np.uint64)
            col = np.empty(2 * m, np.uint32)
            n = ctypes.c_uint64()
            args = [V, m, inputs._p(src), inputs._p(dst), *extra, inputs._p(off), inputs._p(col), ctypes.byref(n)]
            assert fn(*args) == 0
            outs.append((off, col[: n.value]))
        assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_workloads_mdrw_and_layer_s20_shape():
    # MDRW pools and layer-sampling seeds are drawn among vertices with an
    # edge; layer seeds are distinct within an instance; both are seeded
    wm = inputs.workload_mdrw_s20()
    deg = np.diff(wm.graph.off)
    assert wm.pools.shape == (2000, 2000) and wm.steps == 2000
    assert (deg[wm.pools.astype(np.int64)] > 0).all()
    wl = inputs.workload_layer_s20()
    io = wl.inst_offsets.astype(np.int64)
    assert len(io) == 2001 and (np.diff(io) == 64).all() and wl.fanout == [512, 512]
    assert (deg[wl.seeds.astype(np.int64)] > 0).all()
    for i in range(0, 2000, 97):
        assert len(set(wl.seeds[io[i]:io[i + 1]].tolist())) == 64
    assert np.array_equal(inputs.workload_layer_s20().seeds, wl.seeds)


def test_serving_requests_mix():
    """The serving mix alternates sampling and walks with the stated size
    ranges, and is a pure function of its seed."""
    a = inputs.serving_requests(1 << 20, 40, 5)
    b = inputs.serving_requests(1 << 20, 40, 5)
    assert [r[0] for r in a] == ["sample", "walk"] * 20
    for ra, rb in zip(a, b):
        assert ra[0] == rb[0] and np.array_equal(ra[1], rb[1])
    for r in a:
        assert r[1].max() < (1 << 20)
        if r[0] == "sample":
            assert 1 <= len(r[1]) <= 16384 and list(r[2]) == [0, len(r[1])]
            assert 1 <= len(r[3]) <= 3 and set(r[3]) <= {5, 10, 25}
        else:
            assert 1 <= len(r[1]) <= 65536 and 10 <= r[2] <= 80
