"""Pins of the oracle against what the paper and the mathematics fix.

Each test checks the oracle (oracle/csaw_ref.c) against something other than
itself: the paper's worked examples (Fig. 1(b), Fig. 5), Philox known-answer
vectors, exact enumeration of the selection law (Theorem 1 with the integer
mapping), closed forms (stationary law of a weighted walk), special cases that
reduce to a textbook routine (fanout "all" is breadth-first search), and
hand-computed node2vec transition tables (Sec. II-A).
"""
import os

import numpy as np
import pytest
from scipy import stats
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import shortest_path

import oracle
from paper_2009_09103_gb300 import inputs
from conftest import GOLDEN, read_kv

TWO64 = 1 << 64
P_MIN = 1e-4  # chi-square acceptance; inputs are seeded so each test is deterministic


def chi2_pvalue(counts, probs):
    counts = np.asarray(counts, dtype=np.float64)
    probs = np.asarray(probs, dtype=np.float64)
    n = counts.sum()
    exp = probs * n
    # merge bins with small expectation into one
    small = exp < 5
    if small.any():
        counts = np.append(counts[~small], counts[small].sum())
        exp = np.append(exp[~small], exp[small].sum())
        if exp[-1] == 0:
            assert counts[-1] == 0
            counts, exp = counts[:-1], exp[:-1]
    if len(exp) < 2:
        return 1.0
    return stats.chisquare(counts, exp * counts.sum() / exp.sum()).pvalue


# ---------------------------------------------------------------- Philox
def test_philox_known_answer_vectors():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(x, 16) for x in line.split()])
    assert len(rows) == 3
    for r in rows:
        out = oracle.philox4x32_10(r[0:4], r[4:6])
        assert [int(x) for x in out] == r[6:10]


def test_draw_word_layout():
    # key = (lo32(seed), hi32(seed)), counter = (attempt, vertex, layer, instance),
    # r = out1 << 32 | out0
    seed = 0x0123456789ABCDEF
    out = oracle.philox4x32_10([7, 11, 13, 17], [seed & 0xFFFFFFFF, seed >> 32])
    assert oracle.draw(seed, 7, 11, 13, 17) == (int(out[1]) << 32) | int(out[0])


def test_draw_bits_are_uniform():
    # statistical sanity: each of the 64 bits of r is set about half the time
    n = 20000
    r = np.array([oracle.draw(1, a, 5, 0, 0) for a in range(n)], dtype=np.uint64)
    for bit in (0, 17, 31, 32, 50, 63):
        ones = int(((r >> np.uint64(bit)) & np.uint64(1)).sum())
        assert abs(ones - n / 2) < 5 * np.sqrt(n / 4)


# ---------------------------------------------------------------- scaling r -> [0, T)
def test_scale_exact_for_powers_of_two_and_extremes():
    for k in (1, 2, 7, 32, 63):
        for r in (0, 1, 12345678901234567, TWO64 - 1, 1 << 63):
            assert oracle.scale(r, 1 << k) == r >> (64 - k)
    for T in (1, 3, 15, 10**12 + 7, TWO64 - 1):
        assert oracle.scale(0, T) == 0
        assert oracle.scale(TWO64 - 1, T) == T - 1


def test_scale_preimage_sizes():
    # x has exactly ceil((x+1) 2^64 / T) - ceil(x 2^64 / T) preimages: check the
    # boundary draws land on each side of every boundary.
    for T in (3, 15, 1000003):
        for x in (0, 1, T // 2, T - 1):
            lo = -(-x * TWO64 // T)            # smallest r with scale(r) >= x
            assert oracle.scale(lo, T) == x
            if lo > 0:
                assert oracle.scale(lo - 1, T) == x - 1


# ---------------------------------------------------------------- paper examples
NAMES = ["v5", "v7", "v9", "v10", "v11"]


def test_fig1b_inverse_transform_sampling():
    g = read_kv("paper_its_examples.txt")
    b = [int(x) for x in g["biases"]]
    prefix = [int(x) for x in g["prefix_with_leading_zero"]]
    assert list(np.cumsum(b)) == prefix[1:]
    T = prefix[-1]
    assert np.allclose(np.array(prefix) / T, [float(x) for x in g["ctps"]], atol=0.005)
    r = int(float(g["its_draw"][0]) * TWO64)
    assert NAMES[oracle.select_given_draws(b, 1, [r])[0]] == g["its_pick"][0]
    # every x in [0, T) selects the candidate whose interval [S_m, S_m+1) holds x
    for x in range(T):
        r = -(-x * TWO64 // T)
        pick = int(oracle.select_given_draws(b, 1, [r])[0])
        assert prefix[pick] <= x < prefix[pick + 1]


def test_fig5_updated_sampling_and_collision():
    g = read_kv("paper_its_examples.txt")
    b = [int(x) for x in g["biases"]]
    r_v7 = int(float(g["its_draw"][0]) * TWO64)
    r2 = int(float(g["updated_draw"][0]) * TWO64)
    # updated sampling from the second attempt on: v7 then v10
    picks = oracle.select_given_draws(b, 2, [r_v7, r2], attempt_cap=1)
    assert [NAMES[i] for i in picks] == ["v7", g["updated_pick"][0]]
    # the paper's updated prefix sums
    rem = [int(x) for x in g["updated_remaining_biases"]]
    assert [0] + list(np.cumsum(rem)) == [int(x) for x in g["updated_prefix"]]
    # repeated sampling: 0.58 hits v7's region again, so two draws are not enough
    assert oracle.select_given_draws(b, 2, [r_v7, r2], attempt_cap=1024) is None
    r3 = int(0.9 * TWO64)  # 0.9 * 15 = 13.5 -> v11
    picks = oracle.select_given_draws(b, 2, [r_v7, r2, r3], attempt_cap=1024)
    assert [NAMES[i] for i in picks] == ["v7", "v11"]


def _fig1_graph():
    """v8 with neighbours v5, v7, v9, v10, v11 of degrees 3, 6, 2, 2, 2
    (Fig. 1(a) caption); padding vertices 12.. give them those degrees."""
    und = [(8, 5), (8, 7), (8, 9), (8, 10), (8, 11)]
    nxt = 12
    for v, extra in ((5, 2), (7, 5), (9, 1), (10, 1), (11, 1)):
        for _ in range(extra):
            und.append((v, nxt))
            nxt += 1
    edges = und + [(b, a) for a, b in und]
    return inputs.csr_from_edges(nxt, edges)


def test_fig1_neighbour_degree_bias_law():
    g = _fig1_graph()
    assert list(g.col[g.off[8]:g.off[9]]) == [5, 7, 9, 10, 11]
    n = 30000
    counts = {5: 0, 7: 0, 9: 0, 10: 0, 11: 0}
    for inst in range(n):
        counts[int(oracle.select(g, 8, 1, "neighbor_degree", 99, 0, inst)[0])] += 1
    p = chi2_pvalue([counts[v] for v in (5, 7, 9, 10, 11)], np.array([3, 6, 2, 2, 2]) / 15)
    assert p > P_MIN


# ---------------------------------------------------------------- hand-worked two-neighbour case
def test_two_neighbour_weights_1_3():
    b = [1, 3]
    rng = np.random.default_rng(5)
    for top in range(4):
        for _ in range(8):
            low = int(rng.integers(0, 1 << 62))
            r = (top << 62) | low          # x = floor(4 r / 2^64) = top
            assert int(oracle.select_given_draws(b, 1, [r])[0]) == (0 if top == 0 else 1)
    # k >= 2: both, CSR order, no draws used
    assert list(oracle.select_given_draws(b, 2, [])) == [0, 1]
    assert list(oracle.select_given_draws(b, 5, [])) == [0, 1]
    # frequency through the full keyed path: P(nbr 0) = 1/4
    g = inputs.csr_from_edges(3, [(0, 1), (0, 2)], weights=[1, 3])
    n = 40000
    c1 = sum(int(oracle.select(g, 0, 1, "edge_weight", 7, 0, i)[0]) == 2 for i in range(n))  # vertex 2 = nbr 1
    assert chi2_pvalue([n - c1, c1], [0.25, 0.75]) > P_MIN


def test_zero_bias_never_drawn_and_take_all_positive():
    b = [0, 5, 0, 0, 2, 0]
    rng = np.random.default_rng(3)
    draws = [int(x) for x in rng.integers(0, 2**63, size=200, dtype=np.uint64)]
    for k in (1,):
        for r in draws:
            assert int(oracle.select_given_draws(b, k, [r])[0]) in (1, 4)
    # two positive candidates <= k: take them in CSR order
    assert list(oracle.select_given_draws(b, 2, [])) == [1, 4]
    assert list(oracle.select_given_draws(b, oracle.FANOUT_ALL, [])) == [1, 4]
    assert len(oracle.select_given_draws([0, 0, 0], 2, [])) == 0


# ---------------------------------------------------------------- exact selection law by enumeration
def _attempt_probs(b):
    """Exact probability that one attempt lands on each candidate, under
    x = floor(r T / 2^64) with r uniform on [0, 2^64)."""
    S = np.cumsum([0] + list(b)).tolist()
    T = S[-1]
    q = []
    for i in range(len(b)):
        lo = -(-S[i] * TWO64 // T)
        hi = -(-S[i + 1] * TWO64 // T)
        q.append((hi - lo) / TWO64)
    return q


def _tuple_probs(b, k):
    """Law of the ordered k-tuple of first distinct hits (Theorem 1 applied
    repeatedly): prod_t q_jt / (1 - sum_{s<t} q_js)."""
    q = _attempt_probs(b)
    out = {}

    def rec(prefix, p, used):
        if len(prefix) == k:
            out[tuple(prefix)] = p
            return
        for j in range(len(b)):
            if q[j] > 0 and j not in prefix:
                rec(prefix + [j], p * q[j] / (1.0 - used), used + q[j])
    rec([], 1.0, 0.0)
    return out


@pytest.mark.parametrize("b,k,cap", [
    ([1, 3], 1, 1024),
    ([5, 1, 1, 2], 2, 1024),
    ([7, 1, 3, 2, 1], 3, 1024),
    ([2, 9, 1, 4, 4, 1], 3, 1024),
    ([7, 1, 3, 2, 1], 3, 0),       # updated sampling from the first attempt
    ([2, 9, 1, 4, 4, 1], 2, 1),    # switch after one attempt
])
def test_selection_law_matches_enumeration(b, k, cap):
    d = len(b)
    edges = [(0, j + 1) for j in range(d)]
    g = inputs.csr_from_edges(d + 1, edges, weights=b)
    probs = _tuple_probs(b, k)
    keys = sorted(probs)
    index = {t: i for i, t in enumerate(keys)}
    counts = np.zeros(len(keys))
    n = 30000
    for inst in range(n):
        picks = oracle.select(g, 0, k, "edge_weight", 2024, 1, inst, attempt_cap=cap)
        t = tuple(int(u) - 1 for u in picks)
        assert len(set(t)) == k
        counts[index[t]] += 1
    assert chi2_pvalue(counts, [probs[t] for t in keys]) > P_MIN


# ---------------------------------------------------------------- walks
def _ring_with_chords(n=64, seed=1):
    rng = np.random.default_rng(seed)
    und = {}
    for v in range(n):
        und[(v, (v + 1) % n)] = int(rng.integers(1, 10))
    und[(0, 2)] = 5      # a triangle 0-1-2 makes the walk aperiodic
    for _ in range(40):
        a, c = (int(x) for x in rng.integers(0, n, 2))
        if a != c:
            und[(min(a, c), max(a, c))] = int(rng.integers(1, 10))
    edges, ws = [], []
    seen = set()
    for (a, c), w in und.items():
        key = (min(a, c), max(a, c))
        if key in seen:
            continue
        seen.add(key)
        edges += [(a, c), (c, a)]
        ws += [w, w]
    return inputs.csr_from_edges(n, edges, ws)


def test_weighted_walk_stationary_law():
    # A long weighted walk on a connected non-bipartite undirected graph visits
    # v with frequency W(v) / sum W, W(v) = sum of the weights at v.
    g = _ring_with_chords()
    V = g.V
    W = np.array([g.w[g.off[v]:g.off[v + 1]].sum() for v in range(V)], dtype=np.float64)
    pi = W / W.sum()
    starts = inputs.uniform_vertices(8000, V, 5)
    path = oracle.walk(g, starts, 600, "edge_weight", 11)
    visits = np.bincount(path[:, 100:].ravel(), minlength=V) / path[:, 100:].size
    assert 0.5 * np.abs(visits - pi).sum() < 0.01


def test_uniform_walk_on_cycle_is_symmetric():
    n = 16
    edges = [(v, (v + 1) % n) for v in range(n)] + [((v + 1) % n, v) for v in range(n)]
    g = inputs.csr_from_edges(n, edges)
    path = oracle.walk(g, np.zeros(20000, dtype=np.uint32), 1, "uniform", 3)
    right = int((path[:, 1] == 1).sum())
    assert chi2_pvalue([right, 20000 - right], [0.5, 0.5]) > P_MIN
    # equal weights behave as uniform: identical paths (biases scale by a constant)
    g2 = inputs.csr_from_edges(n, edges, weights=[7] * len(edges))
    assert np.array_equal(oracle.walk(g2, np.arange(n), 30, "edge_weight", 9),
                          oracle.walk(g, np.arange(n), 30, "uniform", 9))


def test_walk_dead_end_and_zero_weights():
    # 0 -> 1 -> 2, 2 has no out-edge; 3 -> 4 only with weight 0
    g = inputs.csr_from_edges(5, [(0, 1), (1, 2), (3, 4)], weights=[1, 1, 0])
    p = oracle.walk(g, [0, 3, 2], 4, "edge_weight", 1)
    N = oracle.NONE
    assert p[0].tolist() == [0, 1, 2, N, N]
    assert p[1].tolist() == [3, N, N, N, N]
    assert p[2].tolist() == [2, N, N, N, N]


def test_node2vec_hand_computed_transitions():
    # triangle 0-1-2 plus pendant 3 on 0; w(0,3) = 3, others 1.
    # From 1 the first step is by weight: 0 or 2 with 1/2 each.
    # At 0 having come from 1: u=1 is prev (x1), u=2 is adjacent to 1 (x2),
    # u=3 is not (x4): biases 1*1, 1*2, 3*4 -> (1, 2, 12) / 15.
    # At 2 having come from 1: u=0 adjacent to 1 (x2), u=1 is prev (x1): (2, 1)/3.
    und = [(0, 1, 1), (0, 2, 1), (1, 2, 1), (0, 3, 3)]
    edges = [(a, b) for a, b, _ in und] + [(b, a) for a, b, _ in und]
    ws = [w for *_, w in und] * 2
    g = inputs.csr_from_edges(4, edges, ws)
    n = 30000
    path = oracle.walk(g, np.ones(n, dtype=np.uint32), 2, "node2vec", 17, mult=(1, 2, 4))
    first = path[:, 1]
    assert chi2_pvalue([(first == 0).sum(), (first == 2).sum()], [0.5, 0.5]) > P_MIN
    at0 = path[first == 0, 2]
    assert chi2_pvalue([(at0 == 1).sum(), (at0 == 2).sum(), (at0 == 3).sum()],
                       np.array([1, 2, 12]) / 15) > P_MIN
    at2 = path[first == 2, 2]
    assert chi2_pvalue([(at2 == 0).sum(), (at2 == 1).sum()], np.array([2, 1]) / 3) > P_MIN


def test_node2vec_equal_multipliers_equal_weighted_walk():
    # Scaling every bias by c leaves every pick unchanged:
    # floor(floor(r cT / 2^64) / c) = floor(r T / 2^64) and intervals scale by c.
    g = inputs.rmat_csr(10, 8, 50, 3)
    starts = np.arange(g.V, dtype=np.uint32)
    ref = oracle.walk(g, starts, 12, "edge_weight", 77)
    assert np.array_equal(oracle.walk(g, starts, 12, "node2vec", 77, mult=(1, 1, 1)), ref)
    assert np.array_equal(oracle.walk(g, starts, 12, "node2vec", 77, mult=(2, 2, 2)), ref)
    assert not np.array_equal(oracle.walk(g, starts, 12, "node2vec", 77, mult=(1, 2, 4)), ref)


def test_walk_invariants_and_subset_ids():
    g = inputs.rmat_csr(10, 8, 50, 4)
    starts = inputs.uniform_vertices(500, g.V, 8)
    path = oracle.walk(g, starts, 20, "edge_weight", 5)
    adj = set()
    for v in range(g.V):
        for u in g.col[g.off[v]:g.off[v + 1]]:
            adj.add((v, int(u)))
    for row in path:
        for s in range(20):
            a, c = int(row[s]), int(row[s + 1])
            if a == oracle.NONE:
                assert c == oracle.NONE
            elif c != oracle.NONE:
                assert (a, c) in adj
            else:
                assert g.off[a + 1] == g.off[a]   # sentinel only after a dead end
    # a subset run with explicit walker ids reproduces those rows exactly
    ids = np.array([3, 77, 499], dtype=np.uint64)
    sub = oracle.walk(g, starts[ids.astype(np.int64)], 20, "edge_weight", 5, walker_ids=ids)
    assert np.array_equal(sub, path[ids.astype(np.int64)])


# ---------------------------------------------------------------- layered sampling
def test_fanout_all_is_breadth_first_search():
    # With every neighbour taken, the frontier of layer l is BFS level l and
    # the emitted edges are all edges leaving levels 0 .. depth-1.
    g = inputs.rmat_csr(9, 4, 10, 6)
    V = g.V
    A = csr_matrix((np.ones(g.E), g.col.astype(np.int64), g.off.astype(np.int64)), shape=(V, V))
    seed_v = int(np.argmax(np.diff(g.off)))
    dist = shortest_path(A, unweighted=True, indices=[seed_v])[0]
    depth = 3
    out = oracle.sample(g, [seed_v], [0, 1], [oracle.FANOUT_ALL] * depth, "edge_weight", 1)
    for lvl in range(depth + 1):
        assert out["fsize"][lvl] == int((dist == lvl).sum())
    for lvl in range(depth):
        lo, hi = out["edge_off"][lvl], out["edge_off"][lvl + 1]
        src = out["src"][lo:hi]
        expect = np.flatnonzero(dist == lvl)
        assert np.array_equal(np.unique(src), expect)
        assert hi - lo == int(np.diff(g.off)[expect].sum())


def test_sampling_invariants_small_workload():
    wl = inputs.workload_sample_s12()
    g = wl.graph
    out = oracle.sample(g, wl.seeds, wl.inst_offsets, wl.fanout, wl.bias, wl.rng_seed)
    deg = np.diff(g.off)
    visited = set(np.unique(wl.seeds).tolist())
    assert out["fsize"][0] == len(visited)
    frontier = sorted(visited)
    for lvl, k in enumerate(wl.fanout):
        lo, hi = int(out["edge_off"][lvl]), int(out["edge_off"][lvl + 1])
        src, dst = out["src"][lo:hi], out["dst"][lo:hi]
        # sources are the frontier in ascending order, each with min(k, d) picks
        expect_src = np.repeat(np.array(frontier, dtype=np.uint32),
                               np.minimum(k, deg[np.array(frontier, dtype=np.int64)]).astype(np.int64))
        assert np.array_equal(src, expect_src)
        start = 0
        for v in frontier:
            n = int(min(k, deg[v]))
            picks = dst[start:start + n]
            nb = set(g.col[g.off[v]:g.off[v + 1]].tolist())
            assert len(set(picks.tolist())) == n and set(picks.tolist()) <= nb
            start += n
        nxt = sorted(set(dst.tolist()) - visited)
        assert out["fsize"][lvl + 1] == len(nxt)
        visited |= set(nxt)
        frontier = nxt
    assert out["edge_off"][-1] > 2000


def test_sampling_instances_are_independent():
    # An instance's output depends only on its own seeds and index.
    g = inputs.rmat_csr(10, 8, 30, 9)
    seeds = inputs.uniform_vertices(60, g.V, 4)
    io = np.array([0, 20, 40, 60], dtype=np.uint64)
    full = oracle.sample(g, seeds, io, [4, 3], "edge_weight", 5)
    # instance 1 alone, placed at index 1 with an empty instance 0
    solo = oracle.sample(g, seeds[20:40], np.array([0, 0, 20], dtype=np.uint64), [4, 3], "edge_weight", 5)
    for lvl in range(2):
        a = full["edge_off"][lvl * 3 + 1], full["edge_off"][lvl * 3 + 2]
        b = solo["edge_off"][lvl * 2 + 1], solo["edge_off"][lvl * 2 + 2]
        assert np.array_equal(full["dst"][a[0]:a[1]], solo["dst"][b[0]:b[1]])


# --------------------------------------------------------------------------
# Multi-dimensional random walk (frontier sampling, Sec. II-A; Figs. 3-4)

NONE = 0xFFFFFFFF

def test_mdrw_single_slot_pool_is_a_uniform_walk():
    # With one slot the pool pick is forced and the step is a uniform walk
    # step at the same draw counter {0, v, s, instance}.
    g = inputs.rmat_csr(8, 8, 40, 6)
    starts = inputs.uniform_vertices(300, g.V, 2)
    src, dst = oracle.mdrw(g, starts[:, None], 30, 77)
    path = oracle.walk(g, starts, 30, "uniform", 77)
    taken = path[:, 1:] != NONE
    assert (~taken).any() and taken.any()           # dead ends and real steps both occur
    assert np.array_equal(src, np.where(taken, path[:, :-1], NONE))
    assert np.array_equal(dst, path[:, 1:])


def _degree_ladder_graph(degs):
    """Vertices 0..len(degs)-1 with the given degrees, each joined to its own leaves."""
    edges, nxt = [], len(degs)
    for v, d in enumerate(degs):
        for _ in range(d):
            edges += [(v, nxt), (nxt, v)]
            nxt += 1
    return inputs.csr_from_edges(nxt, edges)


def test_mdrw_pool_pick_follows_vertex_degree():
    # VertexBias (Eq. 2) is the degree: the first pick from pool {0,1,2,3} with
    # degrees 1,2,3,4 has probabilities 1:2:3:4; empty slots (NONE) never win.
    g = _degree_ladder_graph([1, 2, 3, 4])
    n = 40000
    pools = np.tile(np.array([0, NONE, 1, 2, 3], dtype=np.uint32), (n, 1))
    src, _ = oracle.mdrw(g, pools, 1, 5)
    counts = np.bincount(src[:, 0], minlength=4)[:4]
    assert counts.sum() == n
    assert stats.chisquare(counts, n * np.array([1, 2, 3, 4]) / 10).pvalue > 1e-6


def test_mdrw_neighbour_pick_is_uniform_whatever_the_weights():
    # EdgeBias = 1 (Sec. III-D case study): the weights play no part.
    d = 8
    edges = [(0, j + 1) for j in range(d)] + [(j + 1, 0) for j in range(d)]
    g = inputs.csr_from_edges(d + 1, edges, [1, 1000, 1, 1, 50, 1, 1, 7] + [1] * d)
    n = 40000
    _, dst = oracle.mdrw(g, np.zeros((n, 1), dtype=np.uint32), 1, 9)
    counts = np.bincount(dst[:, 0], minlength=d + 1)[1:]
    assert counts.sum() == n
    assert stats.chisquare(counts).pvalue > 1e-6


def test_mdrw_update_replaces_the_picked_vertex():
    # Update (Eq. 4): the step's edge (v, u) is a graph edge, v is in the pool,
    # and the next pool is the multiset with one v replaced by u.
    g = inputs.rmat_csr(7, 8, 40, 3)
    adj = set()
    for v in range(g.V):
        for u in g.col[g.off[v]:g.off[v + 1]]:
            adj.add((v, int(u)))
    pools = inputs.uniform_vertices(40 * 6, g.V, 8).reshape(40, 6)
    src, dst = oracle.mdrw(g, pools, 60, 13)
    for i in range(40):
        pool = sorted(int(x) for x in pools[i])
        for s in range(60):
            v, u = int(src[i, s]), int(dst[i, s])
            if v == NONE:
                assert (src[i, s:] == NONE).all() and (dst[i, s:] == NONE).all()
                assert sum(int(g.off[x + 1] - g.off[x]) for x in pool) == 0
                break
            assert (v, u) in adj and v in pool
            pool.remove(v)
            pool = sorted(pool + [u])


def test_mdrw_stops_when_the_pool_has_no_edges():
    g = inputs.csr_from_edges(4, [(0, 1), (1, 0)])   # 2 and 3 isolated
    src, dst = oracle.mdrw(g, np.array([[2, 3, NONE], [2, 0, 3]], dtype=np.uint32), 5, 1)
    assert (src[0] == NONE).all() and (dst[0] == NONE).all()
    assert list(src[1]) == [0, 1, 0, 1, 0] and list(dst[1]) == [1, 0, 1, 0, 1]


def test_mdrw_sampled_edges_are_uniform_in_steady_state():
    # Frontier sampling's stationary law is proportional to the pool's degree
    # sum, under which every directed edge is sampled with equal probability.
    # A connected, non-bipartite, irregular graph; 4-slot pools; after burn-in
    # the sampled edges must be uniform over E.
    und = [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4), (4, 5), (5, 3), (5, 6), (6, 0), (1, 4)]
    edges = und + [(b, a) for a, b in und]
    g = inputs.csr_from_edges(7, edges)
    n, steps, burn = 3000, 120, 40
    pools = inputs.uniform_vertices(n * 4, 7, 21).reshape(n, 4)
    src, dst = oracle.mdrw(g, pools, steps, 3)
    key = {e: i for i, e in enumerate(sorted(edges))}
    s, d = src[:, burn:].ravel(), dst[:, burn:].ravel()
    counts = np.bincount([key[(int(a), int(b))] for a, b in zip(s, d)], minlength=len(edges))
    assert stats.chisquare(counts).pvalue > 1e-6


# --------------------------------------------------------------------------
# Random walk with restart and with jump (Sec. II-A; Update, Eq. 4)

Q32_ALWAYS = 0xFFFFFFFF   # teleport probability 1 - 2^-32


def test_teleport_with_probability_zero_is_the_plain_walk():
    g = inputs.rmat_csr(8, 8, 40, 2)
    deg = np.diff(g.off)
    starts = np.flatnonzero(deg > 0).astype(np.uint32)[:200]   # no dead end is reachable from these
    ref = oracle.walk(g, starts, 30, "edge_weight", 8)
    for mode in ("restart", "jump"):
        assert np.array_equal(oracle.walk(g, starts, 30, "edge_weight", 8, teleport=mode, teleport_q32=0), ref)


def test_teleport_always_restarts_or_jumps_uniformly():
    g = inputs.rmat_csr(6, 8, 40, 2)
    starts = inputs.uniform_vertices(400, g.V, 1)
    p = oracle.walk(g, starts, 25, "node2vec", 4, mult=(1, 2, 4), teleport="restart", teleport_q32=Q32_ALWAYS)
    assert (p == starts[:, None]).all()
    p = oracle.walk(g, starts, 200, "edge_weight", 4, teleport="jump", teleport_q32=Q32_ALWAYS)
    assert (p < g.V).all()
    counts = np.bincount(p[:, 1:].ravel(), minlength=g.V)
    assert counts.sum() == 400 * 200
    assert stats.chisquare(counts).pvalue > 1e-6


def test_restart_walk_law_is_personalized_pagerank():
    # With restart probability c (and a dead end that restarts), the state after
    # enough steps follows pi = c e_s (I - (1-c) P)^-1, P the biased
    # transition matrix with the dead end's row sent to the start.
    und = [(0, 1, 3), (1, 2, 1), (2, 0, 2), (2, 3, 5), (3, 4, 1), (4, 2, 2), (1, 4, 4)]
    edges = [(a, b) for a, b, _ in und] + [(b, a) for a, b, _ in und] + [(3, 5)]   # 5: dead end
    wts = [x for *_, x in und] * 2 + [6]
    g = inputs.csr_from_edges(6, edges, wts)
    V, start, c = 6, 1, 0.25
    P = np.zeros((V, V))
    for (a, b), x in zip(edges, wts):
        P[a, b] += x
    P[5, start] = 1.0
    P /= P.sum(axis=1, keepdims=True)
    e = np.zeros(V)
    e[start] = 1.0
    pi = c * e @ np.linalg.inv(np.eye(V) - (1 - c) * P)
    q32 = int(round(c * 2**32))
    n, L = 40000, 60
    path = oracle.walk(g, np.full(n, start, dtype=np.uint32), L, "edge_weight", 17,
                       teleport="restart", teleport_q32=q32)
    assert (path[:, L] < V).all()   # restart walks never stop
    counts = np.bincount(path[:, L], minlength=V)
    assert stats.chisquare(counts, n * pi).pvalue > 1e-6


# --------------------------------------------------------------------------
# Layer sampling (Sec. II-A; Fig. 2(b) with the whole frontier as the current
# frontier): one pool of all frontier edges per instance and layer

def test_layer_sampling_takes_the_whole_pool_in_order():
    # layer size at least the pool: every edge of the seeds, ascending source
    # then CSR order, and the next frontier is every new neighbour
    g = inputs.rmat_csr(8, 8, 40, 4)
    seeds = np.array([9, 3, 200, 3], dtype=np.uint32)
    io = np.array([0, 4], dtype=np.uint64)
    r = oracle.sample(g, seeds, io, [10**6, 0], "edge_weight", 2, layer=True)
    exp_src, exp_dst = [], []
    for v in (3, 9, 200):
        for u in g.col[g.off[v]:g.off[v + 1]]:
            exp_src.append(v)
            exp_dst.append(int(u))
    n0 = int(r["edge_off"][1])
    assert list(r["src"][:n0]) == exp_src and list(r["dst"][:n0]) == exp_dst
    assert r["fsize"][1] == len(set(exp_dst) - {3, 9, 200})


def test_layer_sampling_pick_follows_edge_bias_over_the_pool():
    # frontier {0, 1}: vertex 0 has edges of weight 1, 2, 3, vertex 1 edges of
    # weight 4 and 10; the first pick of each instance follows the weights
    # over the whole pool (not a vertex first, then a neighbour)
    edges = [(0, 2), (0, 3), (0, 4), (1, 5), (1, 6)]
    wts = [1, 2, 3, 4, 10]
    g = inputs.csr_from_edges(7, edges + [(b, a) for a, b in edges], wts + wts)
    n = 30000
    seeds = np.tile(np.array([0, 1], dtype=np.uint32), n)
    io = np.arange(0, 2 * n + 1, 2, dtype=np.uint64)
    r = oracle.sample(g, seeds, io, [2], "edge_weight", 6, layer=True)
    first = r["dst"][r["edge_off"][:-1].astype(np.int64)]
    counts = np.bincount(first, minlength=7)[2:]
    assert counts.sum() == n
    assert stats.chisquare(counts, n * np.array(wts) / sum(wts)).pvalue > 1e-6


def test_layer_sampling_counts_and_distinct_picks():
    g = inputs.rmat_csr(9, 8, 40, 5)
    g.w[::5] = 0   # zero biases are never picked
    sizes = inputs.loguniform_sizes(40, 0.0, 5.0, 3)
    seeds, io = inputs.distinct_seeds(sizes, g.V, 3)
    r = oracle.sample(g, seeds, io, [25, 60], "edge_weight", 9, layer=True)
    wmap = {}
    for v in range(g.V):
        for j in range(int(g.off[v]), int(g.off[v + 1])):
            wmap[(v, int(g.col[j]))] = int(g.w[j])
    n_inst = len(io) - 1
    F = [sorted(set(int(x) for x in seeds[io[i]:io[i + 1]])) for i in range(n_inst)]
    visited = [set(f) for f in F]
    for l, k in enumerate((25, 60)):
        for i in range(n_inst):
            a, b = int(r["edge_off"][l * n_inst + i]), int(r["edge_off"][l * n_inst + i + 1])
            pairs = list(zip(r["src"][a:b].tolist(), r["dst"][a:b].tolist()))
            npos = sum(1 for v in F[i] for j in range(int(g.off[v]), int(g.off[v + 1])) if g.w[j] > 0)
            assert len(pairs) == min(k, npos) and len(set(pairs)) == len(pairs)
            assert all(wmap.get(p, 0) > 0 and p[0] in F[i] for p in pairs)
            # Update: the next frontier is the new picked vertices
            F[i] = sorted(set(u for _, u in pairs) - visited[i])
            visited[i] |= set(F[i])
            assert r["fsize"][(l + 1) * n_inst + i] == len(F[i])
    assert r["fsize"].shape[0] == 3 * n_inst
