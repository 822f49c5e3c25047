"""The request server: admission by memory budget, concurrent slots, and
results identical alone, in the mix and to the oracle."""
import numpy as np
import pytest

import oracle
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
    g = inputs.rmat_csr(16, 16, 100, 16)
    G = csaw.Graph(g.off, g.col, g.w)
    yield csaw, g, G
    G.close()


def mixed_requests(g, n=24, seed=0):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        if i % 2 == 0:
            ns = int(2 ** rng.uniform(0, 10))
            seeds = inputs.uniform_vertices(ns, g.V, 100 + i)
            n_inst = int(rng.integers(1, 4))
            io = np.linspace(0, ns, n_inst + 1).astype(np.uint64)
            depth = int(rng.integers(1, 4))
            fan = [int(x) for x in rng.choice([5, 10, 25], size=depth)]
            reqs.append(("sample", seeds, io, fan, 1000 + i))
        else:
            nw = int(2 ** rng.uniform(0, 12))
            starts = inputs.uniform_vertices(nw, g.V, 200 + i)
            reqs.append(("walk", starts, int(rng.integers(10, 81)), 2000 + i))
    return reqs


def test_results_same_alone_and_in_the_mix(env):
    csaw, g, G = env
    reqs = mixed_requests(g)
    srv = csaw.Server(G, budget_bytes=2 << 30, slots=4)
    tickets = []
    for r in reqs:
        if r[0] == "sample":
            tickets.append(srv.submit_sample(r[1], r[2], r[3], "edge_weight", r[4]))
        else:
            tickets.append(srv.submit_walk(r[1], r[2], "edge_weight", r[3]))
    served = [srv.poll(t) for t in tickets]
    srv.close()
    for r, s in zip(reqs, served):
        if r[0] == "sample":
            alone = csaw.sample(G, r[1], r[2], r[3], "edge_weight", r[4])
            assert np.array_equal(s.sample.dst, alone.dst) and np.array_equal(s.sample.src, alone.src)
            assert np.array_equal(s.sample.edge_offsets, alone.edge_offsets)
            ref = oracle.sample(g, r[1], r[2], r[3], "edge_weight", r[4])
            assert np.array_equal(s.sample.src, ref["src"]) and np.array_equal(s.sample.dst, ref["dst"])
            assert np.array_equal(s.sample.edge_offsets, ref["edge_off"])
            n_inst = len(r[2]) - 1
            assert np.array_equal(s.sample.frontier_sizes, ref["fsize"][: len(r[3]) * n_inst])
        else:
            alone = csaw.walk(G, r[1], r[2], "edge_weight", r[3])
            assert np.array_equal(s.path, alone)
            assert np.array_equal(s.path, oracle.walk(g, r[1], r[2], "edge_weight", r[3]))
        assert s.t_submit_ns <= s.t_admit_ns <= s.t_start_ns <= s.t_finish_ns


def test_requests_overlap_on_the_device(env):
    csaw, g, G = env
    srv = csaw.Server(G, budget_bytes=4 << 30, slots=4, max_batch=1)
    starts = inputs.uniform_vertices(3000, g.V, 3)   # 3000 x 80 steps: small requests
    ts = [srv.submit_walk(starts, 80, "edge_weight", k) for k in range(8)]
    res = [srv.poll(t) for t in ts]
    srv.close()
    # some request started before another finished: slots run concurrently
    spans = sorted((r.t_start_ns, r.t_finish_ns) for r in res)
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))


def test_small_requests_finish_beside_large_ones(env):
    """Small requests submitted behind large ones (more than 2^18 sampled
    edges possible) start in a free slot, run on a high-priority stream
    beside them and finish before the last large one; each result is that
    of the request alone."""
    csaw, g, G = env
    srv = csaw.Server(G, budget_bytes=8 << 30, slots=4, max_batch=1)
    big = inputs.uniform_vertices(1 << 15, g.V, 4)          # 32768 x 80 steps: large
    small = inputs.uniform_vertices(500, g.V, 5)            # 500 x 20 steps: small
    tb = [srv.submit_walk(big, 80, "edge_weight", k) for k in range(3)]
    ts = [srv.submit_walk(small, 20, "edge_weight", 10 + k) for k in range(3)]
    rb = [srv.poll(t) for t in tb]
    rs = [srv.poll(t) for t in ts]
    srv.close()
    assert min(r.t_finish_ns for r in rs) < max(r.t_finish_ns for r in rb)
    for k, r in enumerate(rs):
        assert np.array_equal(r.path, oracle.walk(g, small, 20, "edge_weight", 10 + k))
    for k, r in enumerate(rb[:2]):
        assert np.array_equal(r.path, oracle.walk(g, big, 80, "edge_weight", k))


def test_admission_by_budget(env):
    csaw, g, G = env
    starts = inputs.uniform_vertices(1 << 16, g.V, 5)
    one = 4 * len(starts) + 4 * len(starts) * 81 + 4096
    # the budget holds one such walk at a time: admissions are serialised
    srv = csaw.Server(G, budget_bytes=one + one // 2, slots=4)
    ts = [srv.submit_walk(starts, 80, "edge_weight", k) for k in range(4)]
    res = [srv.poll(t) for t in ts]
    srv.close()
    res.sort(key=lambda r: r.t_admit_ns)
    for a, b in zip(res, res[1:]):
        assert b.t_admit_ns >= a.t_finish_ns
    assert all(r.estimate == one for r in res)
    # a request larger than the whole budget is refused at submission
    srv = csaw.Server(G, budget_bytes=one // 2, slots=1)
    with pytest.raises(csaw.CsawError) as e:
        srv.submit_walk(starts, 80, "edge_weight", 1)
    assert e.value.status == csaw.ERR_NOMEM
    srv.close()


def test_poll_timeout_cancel_and_unknown_ticket(env):
    csaw, g, G = env
    srv = csaw.Server(G, budget_bytes=8 << 30, slots=1)
    big = inputs.uniform_vertices(1 << 18, g.V, 7)
    t1 = srv.submit_walk(big, 80, "edge_weight", 1)
    t2 = srv.submit_walk(big[:100], 10, "edge_weight", 2)
    # the single slot is busy with t1, so t2 cannot have finished yet
    with pytest.raises(csaw.CsawError) as e:
        srv.poll(t2, timeout_us=0)
    assert e.value.status == csaw.ERR_TIMEOUT
    try:
        srv.cancel(t2)
        cancelled = True
    except csaw.CsawError as ex:          # t1 finished and t2 was admitted in between
        assert ex.status == csaw.ERR_INVALID
        cancelled = False
    if cancelled:
        with pytest.raises(csaw.CsawError) as e:
            srv.poll(t2)
        assert e.value.status == csaw.ERR_ABORTED
    else:
        assert srv.poll(t2).status == csaw.OK
    assert srv.poll(t1).status == csaw.OK
    with pytest.raises(csaw.CsawError) as e:
        srv.poll(t1)                       # retired
    assert e.value.status == csaw.ERR_NOT_FOUND
    with pytest.raises(csaw.CsawError) as e:
        srv.poll(12345)
    assert e.value.status == csaw.ERR_NOT_FOUND
    srv.close()


def test_destroy_with_requests_in_flight(env):
    csaw, g, G = env
    srv = csaw.Server(G, budget_bytes=8 << 30, slots=2)
    starts = inputs.uniform_vertices(1 << 16, g.V, 9)
    for k in range(6):
        srv.submit_walk(starts, 40, "edge_weight", k)
    srv.close()          # pending ones are aborted, running ones finish; no hang
    # the graph is still usable afterwards
    assert csaw.walk(G, starts[:10], 5, "edge_weight", 1).shape == (10, 6)


def test_invalid_requests(env):
    csaw, g, G = env
    srv = csaw.Server(G, budget_bytes=1 << 30, slots=1)
    with pytest.raises(csaw.CsawError) as e:
        srv.submit_walk(np.array([g.V], dtype=np.uint32), 5)
    assert e.value.status == csaw.ERR_INVALID
    with pytest.raises(csaw.CsawError) as e:
        srv.submit_sample(np.array([0], dtype=np.uint32), np.array([0, 1], dtype=np.uint64), [2], "node2vec")
    assert e.value.status == csaw.ERR_INVALID
    srv.close()


def test_batches_of_waiting_requests(env):
    """One slot and a burst of requests: the waiting ones run as batches
    (one multi-instance launch per kind and bias) and every result equals its
    request alone and the oracle -- mixed depths, fanouts, instance counts,
    walk lengths, empty requests and node2vec walks."""
    csaw, g, G = env
    rng = np.random.default_rng(5)
    reqs = []
    for i in range(30):
        if i % 3 == 0:
            n_inst = int(rng.integers(0, 4))
            ns = int(rng.integers(0, 300))
            seeds = inputs.uniform_vertices(ns, g.V, 300 + i)
            cuts = np.sort(rng.integers(0, ns + 1, size=max(n_inst - 1, 0)))
            io = np.concatenate([[0], cuts, [ns]]).astype(np.uint64) if n_inst else np.array([0], dtype=np.uint64)
            if n_inst == 0:
                seeds = seeds[:0]
            fan = [int(x) for x in rng.choice([1, 5, 25, 300], size=int(rng.integers(1, 4)))]
            reqs.append(("sample", seeds, io, fan, 40 + i, "edge_weight"))
        elif i % 3 == 1:
            nw = int(rng.integers(0, 2000))
            reqs.append(("walk", inputs.uniform_vertices(nw, g.V, 500 + i), int(rng.integers(0, 50)), 60 + i,
                         "edge_weight", (1, 1, 1)))
        else:
            nw = int(rng.integers(1, 500))
            reqs.append(("walk", inputs.uniform_vertices(nw, g.V, 700 + i), int(rng.integers(1, 30)), 80 + i,
                         "node2vec", (1, 2, 4)))
    srv = csaw.Server(G, budget_bytes=8 << 30, slots=1)
    tickets = []
    for r in reqs:
        if r[0] == "sample":
            tickets.append(srv.submit_sample(r[1], r[2], r[3], r[5], r[4]))
        else:
            tickets.append(srv.submit_walk(r[1], r[2], r[4], r[3], r[5]))
    served = [srv.poll(t) for t in tickets]
    srv.close()
    starts = [s.t_start_ns for s in served]
    assert len(set(starts)) < len(starts), "no two requests ran in one batch"
    for r, s in zip(reqs, served):
        if r[0] == "sample":
            ref = oracle.sample(g, r[1], r[2], r[3], r[5], r[4])
            assert np.array_equal(s.sample.edge_offsets, ref["edge_off"])
            assert np.array_equal(s.sample.src, ref["src"]) and np.array_equal(s.sample.dst, ref["dst"])
            n_inst = len(r[2]) - 1
            assert np.array_equal(s.sample.frontier_sizes, ref["fsize"][: len(r[3]) * n_inst])
        else:
            assert np.array_equal(s.path, oracle.walk(g, r[1], r[2], r[4], r[3], mult=r[5]))


def test_batches_with_cached_arrays(env):
    """Batched walks and sampling over the cached cumulative array (the
    thread-per-walker kernel with per-request rows) equal the oracle."""
    csaw, g, _ = env
    G = csaw.Graph(g.off, g.col, g.w)
    G.build_cdf("edge_weight")
    srv = csaw.Server(G, budget_bytes=8 << 30, slots=1)
    reqs = []
    for i in range(12):
        if i % 2:
            reqs.append(("walk", inputs.uniform_vertices(37 * i + 1, g.V, 900 + i), 3 * i, 11 + i))
        else:
            reqs.append(("sample", inputs.uniform_vertices(20 * i + 1, g.V, 950 + i),
                         np.array([0, 20 * i + 1], dtype=np.uint64), [10, 3], 13 + i))
    tickets = [srv.submit_walk(r[1], r[2], "edge_weight", r[3]) if r[0] == "walk"
               else srv.submit_sample(r[1], r[2], r[3], "edge_weight", r[4]) for r in reqs]
    served = [srv.poll(t) for t in tickets]
    srv.close()
    for r, s in zip(reqs, served):
        if r[0] == "walk":
            assert np.array_equal(s.path, oracle.walk(g, r[1], r[2], "edge_weight", r[3]))
        else:
            ref = oracle.sample(g, r[1], r[2], r[3], "edge_weight", r[4])
            assert np.array_equal(s.sample.dst, ref["dst"]) and np.array_equal(s.sample.edge_offsets, ref["edge_off"])
    G.close()
