"""Multi-dimensional random walk on the GPU through the C ABI, bit-exact
against the oracle."""
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


def graphs():
    und = [(0, 1), (0, 2), (1, 2), (0, 3)]
    e = und + [(b, a) for a, b in und]
    return {
        # vertices 4 and 5 isolated: a pool of only them stops at once
        "triangle_pendant_isolated": inputs.csr_from_edges(6, e),
        "rmat_s8": inputs.rmat_csr(8, 8, 40, 1),
        "rmat_s12": inputs.rmat_csr(12, 16, 100, 12),
    }


def run_both(csaw, g, pools, steps, seed):
    G = csaw.Graph(g.off, g.col, g.w)
    got = csaw.mdrw(G, pools, steps, seed)
    G.close()
    ref = oracle.mdrw(g, pools, steps, seed)
    return got, ref


@pytest.mark.parametrize("gname", ["triangle_pendant_isolated", "rmat_s8", "rmat_s12"])
@pytest.mark.parametrize("pool_size", [1, 3, 32, 33, 100, 2000, 2048, 2049])
def test_mdrw_bit_exact_small(csaw, gname, pool_size):
    g = graphs()[gname]
    n = 64 if pool_size >= 1000 else 200
    pools = inputs.uniform_vertices(n * pool_size, g.V, pool_size).reshape(n, pool_size)
    for steps in (1, 31, 32, 33, 75):
        (s, d), (rs, rd) = run_both(csaw, g, pools, steps, 11 + steps)
        assert np.array_equal(s, rs) and np.array_equal(d, rd), (gname, pool_size, steps)


def test_mdrw_empty_slots_and_dead_pools(csaw):
    g = graphs()["triangle_pendant_isolated"]
    pools = np.array([[NONE, 4, NONE], [4, 5, NONE], [NONE, NONE, 3], [4, NONE, 0]], dtype=np.uint32)
    (s, d), (rs, rd) = run_both(csaw, g, pools, 40, 5)
    assert np.array_equal(s, rs) and np.array_equal(d, rd)
    assert (s[0] == NONE).all() and (s[1] == NONE).all() and (s[2] != NONE).all()


def test_mdrw_steps_zero_and_zero_weights_ignored(csaw):
    g = graphs()["rmat_s8"]
    gz = inputs.CSRGraph(g.off, g.col, np.zeros_like(g.w))   # EdgeBias = 1: weights play no part
    pools = inputs.uniform_vertices(50 * 7, g.V, 3).reshape(50, 7)
    G = csaw.Graph(gz.off, gz.col, gz.w)
    s0, d0 = csaw.mdrw(G, pools, 0, 1)
    assert s0.shape == (50, 0) and d0.shape == (50, 0)
    s, d = csaw.mdrw(G, pools, 50, 2)
    G.close()
    rs, rd = oracle.mdrw(g, pools, 50, 2)
    assert np.array_equal(s, rs) and np.array_equal(d, rd)


def test_mdrw_largest_pool(csaw):
    # 65536 slots: 2048 blocks, 64 per lane in the top-level scan
    g = graphs()["rmat_s12"]
    m = 65536
    pools = inputs.uniform_vertices(2 * m, g.V, 17).reshape(2, m)
    pools[0, ::7] = NONE
    (s, d), (rs, rd) = run_both(csaw, g, pools, 40, 23)
    assert np.array_equal(s, rs) and np.array_equal(d, rd)


def test_mdrw_device_buffers_match_host(csaw):
    import torch
    g = graphs()["rmat_s12"]
    pools = inputs.uniform_vertices(300 * 50, g.V, 4).reshape(300, 50)
    G = csaw.Graph(g.off, g.col, g.w)
    hs, hd = csaw.mdrw(G, pools, 64, 9)
    dp = torch.from_numpy(pools.view(np.int32)).cuda()
    ds, dd = csaw.mdrw(G, dp, 64, 9)
    torch.cuda.synchronize()
    G.close()
    assert np.array_equal(ds.cpu().numpy().view(np.uint32), hs)
    assert np.array_equal(dd.cpu().numpy().view(np.uint32), hd)


def test_mdrw_single_slot_equals_gpu_uniform_walk(csaw):
    g = graphs()["rmat_s12"]
    starts = inputs.uniform_vertices(500, g.V, 6)
    G = csaw.Graph(g.off, g.col, g.w)
    s, d = csaw.mdrw(G, starts[:, None], 40, 31)
    path = csaw.walk(G, starts, 40, "uniform", 31)
    G.close()
    taken = path[:, 1:] != NONE
    assert np.array_equal(s, np.where(taken, path[:, :-1], NONE))
    assert np.array_equal(d, path[:, 1:])


def test_mdrw_errors(csaw):
    g = graphs()["rmat_s8"]
    G = csaw.Graph(g.off, g.col, g.w)
    with pytest.raises(csaw.CsawError):
        csaw.mdrw(G, np.zeros((4, 0), dtype=np.uint32), 5, 1)
    with pytest.raises(csaw.CsawError):
        csaw.mdrw(G, np.zeros((1, 65537), dtype=np.uint32), 5, 1)
    s, d = csaw.mdrw(G, np.zeros((0, 5), dtype=np.uint32), 5, 1)
    assert s.shape == (0, 5)
    G.close()


def test_mdrw_full_size_workload_sampled_rows(csaw):
    # RMAT s20, 2000 instances x 2000-slot pools x 2000 steps (the bench's
    # launch); rows of a stratified subset of instances against the oracle,
    # which takes the instances' own RNG ids.
    import torch
    wl = inputs.workload_mdrw_s20()
    g = wl.graph
    G = csaw.Graph(g.off, g.col, g.w)
    dp = torch.from_numpy(wl.pools.view(np.int32)).cuda()
    s, d = csaw.mdrw(G, dp, wl.steps, wl.rng_seed)
    torch.cuda.synchronize()
    G.close()
    s = s.cpu().numpy().view(np.uint32)
    d = d.cpu().numpy().view(np.uint32)
    pick = np.linspace(0, len(wl.pools) - 1, 6).astype(np.int64)
    rs, rd = oracle.mdrw(g, wl.pools[pick], wl.steps, wl.rng_seed, instance_ids=pick.astype(np.uint64))
    assert np.array_equal(s[pick], rs) and np.array_equal(d[pick], rd)
    # sampled steps of all instances: every emitted edge is a graph edge
    flat = s != NONE
    assert flat.all()   # pools of vertices with edges never stop
    v, u = s[flat].astype(np.int64), d[flat].astype(np.int64)
    for i in np.random.default_rng(0).choice(len(v), size=2000, replace=False):
        row = g.col[int(g.off[v[i]]):int(g.off[v[i] + 1])]
        j = np.searchsorted(row, u[i])
        assert j < len(row) and row[j] == u[i]
