"""Batched sample plans (one CUDA graph over all instances and layers) and
the selection autotuner: results identical to csaw_sample and to the oracle."""
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


def same(a, b):
    assert a.n_edges == b.n_edges
    assert np.array_equal(a.edge_offsets, b.edge_offsets)
    assert np.array_equal(a.frontier_sizes, b.frontier_sizes)
    assert np.array_equal(a.src, b.src) and np.array_equal(a.dst, b.dst)


@pytest.mark.parametrize("bias,fanout", [("edge_weight", [10, 5]), ("neighbor_degree", [25, 10]),
                                         ("uniform", [3, 3, 3]), ("edge_weight", [ALL, 2])])
def test_plan_matches_sample_and_oracle(csaw, bias, fanout):
    g = inputs.rmat_csr(12, 16, 100, 12)
    G = csaw.Graph(g.off, g.col, g.w)
    sizes = inputs.loguniform_sizes(64, 0.0, 6.0, 2)
    seeds, io = inputs.distinct_seeds(sizes, g.V, 2)
    plan = csaw.SamplePlan(G, 64, int(io[-1]) + 100, fanout, bias)
    for seed in (1, 2):   # two runs of the same captured graph
        plan.run(seeds, io, seed)
        got = plan.result()
        same(got, csaw.sample(G, seeds, io, fanout, bias, seed))
        ref = oracle.sample(g, seeds, io, fanout, bias, seed)
        assert np.array_equal(got.dst, ref["dst"]) and np.array_equal(got.edge_offsets, ref["edge_off"])
    # fewer seeds than the plan's budget, with a different split
    io2 = np.array([0] + [5] * 63 + [5], dtype=np.uint64)
    io2[1:64] = np.minimum(np.arange(1, 64), 5)
    plan.run(seeds[:5], io2, 3)
    same(plan.result(), csaw.sample(G, seeds[:5], io2, fanout, bias, 3))
    plan.close()
    G.close()


def test_plan_device_inputs_and_hubs(csaw):
    import torch
    rng = np.random.default_rng(3)
    d = 20000
    edges = [(0, j + 1) for j in range(d)] + [(j + 1, 0) for j in range(d)]
    g = inputs.csr_from_edges(d + 1, edges, list(rng.integers(1, 100, size=d)) + [1] * d)
    G = csaw.Graph(g.off, g.col, g.w)
    seeds = np.array([0, 0, 5, 0, 7, 9], dtype=np.uint32)
    io = np.array([0, 2, 4, 6], dtype=np.uint64)
    plan = csaw.SamplePlan(G, 3, 6, [30, 4], "edge_weight")
    plan.run(torch.from_numpy(seeds.view(np.int32)).cuda(), torch.from_numpy(io.view(np.int64)).cuda(), 8)
    same(plan.result(), csaw.sample(G, seeds, io, [30, 4], "edge_weight", 8))
    plan.close()
    G.close()


def test_plan_rejects_bad_inputs(csaw):
    g = inputs.rmat_csr(8, 8, 40, 1)
    G = csaw.Graph(g.off, g.col, g.w)
    plan = csaw.SamplePlan(G, 1, 4, [2], "edge_weight")
    with pytest.raises(csaw.CsawError) as e:
        plan.run(np.arange(5, dtype=np.uint32), np.array([0, 5], dtype=np.uint64), 1)
    assert e.value.status == csaw.ERR_INVALID
    with pytest.raises(csaw.CsawError) as e:
        plan.run(np.array([g.V], dtype=np.uint32), np.array([0, 1], dtype=np.uint64), 1)
    assert e.value.status == csaw.ERR_INVALID
    with pytest.raises(csaw.CsawError):
        plan.result()    # never ran
    plan.close()
    G.close()


def test_tuning_changes_speed_not_results(csaw):
    g = inputs.rmat_csr(13, 16, 100, 13)
    G = csaw.Graph(g.off, g.col, g.w)
    seeds = inputs.uniform_vertices(2000, g.V, 4)
    io = np.linspace(0, 2000, 41).astype(np.uint64)
    ref = csaw.sample(G, seeds, io, [10, 5], "neighbor_degree", 6)
    for tw in (0, 32, 64, 128, 256):
        for per in (0, 1, 2):
            csaw.set_select_tuning(G, "neighbor_degree", tw, per)
            same(csaw.sample(G, seeds, io, [10, 5], "neighbor_degree", 6), ref)
    best = csaw.autotune_select(G, seeds, io, [10, 5], "neighbor_degree", 6)
    assert best["theta_warp"] in (32, 64, 128, 256) and best["blocks_per_sm"] >= 1
    assert csaw.get_select_tuning(G, "neighbor_degree") == best
    same(csaw.sample(G, seeds, io, [10, 5], "neighbor_degree", 6), ref)
    G.close()


def test_batched_equals_one_call_per_instance(csaw):
    """The batched multi-instance run gives every instance exactly what a
    call with that instance alone (at its own index) gives."""
    g = inputs.rmat_csr(14, 16, 100, 14)
    G = csaw.Graph(g.off, g.col, g.w)
    sizes = inputs.loguniform_sizes(50, 2.0, 5.0, 9)
    seeds, io = inputs.distinct_seeds(sizes, g.V, 9)
    plan = csaw.SamplePlan(G, 50, int(io[-1]), [25, 10], "neighbor_degree")
    plan.run(seeds, io, 4)
    batched = plan.result()
    for i in (0, 7, 49):
        sub = np.zeros(51, dtype=np.uint64)
        sub[i + 1:] = io[i + 1] - io[i]
        alone = csaw.sample(G, seeds[io[i]:io[i + 1]], sub, [25, 10], "neighbor_degree", 4)
        for lvl in range(2):
            a = batched.edge_offsets[lvl * 50 + i], batched.edge_offsets[lvl * 50 + i + 1]
            b = alone.edge_offsets[lvl * 50 + i], alone.edge_offsets[lvl * 50 + i + 1]
            assert np.array_equal(batched.dst[a[0]:a[1]], alone.dst[b[0]:b[1]])
    plan.close()
    G.close()
