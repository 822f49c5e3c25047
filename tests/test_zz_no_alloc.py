"""csaw_select_noalloc: one selection layer without device allocation.

Some callers cannot allocate device memory while they use this library (code
inside another framework's fixed memory budget, runtimes without a device
allocator, host threads that must not touch the allocator).  This test calls
the no-allocation entry point through the C ABI and checks that two calls in
a row return exactly what csaw_sample returns for the same first layer.
"""
import ctypes

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
    L = csaw.lib()
    P, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
    L.csaw_select_noalloc.argtypes = [P, P, P, u32, u32, u32, ctypes.POINTER(csaw.Bias), u64,
                                      P, P, u64, P, P]
    L.csaw_select_noalloc.restype = ctypes.c_int
    return torch, csaw, L


def first_layer(seeds, io):
    """The sorted distinct seeds of every instance, with their instance ids."""
    vs, ins = [], []
    for i in range(len(io) - 1):
        u = np.unique(seeds[io[i]:io[i + 1]])
        vs.append(u)
        ins.append(np.full(len(u), i, dtype=np.uint32))
    return np.concatenate(vs).astype(np.uint32), np.concatenate(ins)


def noalloc(torch, csaw, L, G, vs, ins, k, bias, seed, expect=0):
    n = len(vs)
    cap = n * min(k, G.info().max_degree)
    dv = torch.from_numpy(vs.view(np.int32)).cuda()
    di = torch.from_numpy(ins.view(np.int32)).cuda()
    src = torch.empty(max(cap, 1), dtype=torch.int32, device="cuda")
    dst = torch.empty(max(cap, 1), dtype=torch.int32, device="cuda")
    off = torch.full((n + 1,), -1, dtype=torch.int64, device="cuda")
    b = csaw.make_bias(bias)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = L.csaw_select_noalloc(G.handle, ctypes.c_void_p(dv.data_ptr()), ctypes.c_void_p(di.data_ptr()),
                               n, k, 0, ctypes.byref(b), seed, ctypes.c_void_p(src.data_ptr()),
                               ctypes.c_void_p(dst.data_ptr()), cap, ctypes.c_void_p(off.data_ptr()), stream)
    assert st == expect, L.csaw_last_error()
    torch.cuda.synchronize()
    if expect != 0:
        return None
    o = off.cpu().numpy().view(np.uint64)
    total = int(o[-1])
    return (src[:total].cpu().numpy().view(np.uint32), dst[:total].cpu().numpy().view(np.uint32), o)


def cases():
    rng = np.random.default_rng(8)
    g1 = inputs.rmat_csr(14, 16, 100, 14)
    sizes = inputs.loguniform_sizes(40, 0.0, 8.0, 3)
    s1, io1 = inputs.distinct_seeds(sizes, g1.V, 3)
    # a star above the shared-memory limit of the CTA path: hub scratch slots
    d = 20000
    edges = [(0, j + 1) for j in range(d)] + [(j + 1, 0) for j in range(d)]
    g2 = inputs.csr_from_edges(d + 1, edges, list(rng.integers(1, 500, size=d)) + [1] * d)
    s2 = np.zeros(12, dtype=np.uint32)
    s2[6:] = rng.integers(1, d + 1, size=6)
    io2 = np.arange(13, dtype=np.uint64)
    return [(g1, s1, io1, 10, "neighbor_degree"), (g1, s1, io1, 3, "edge_weight"),
            (g2, s2, io2, 25, "edge_weight")]


def test_noalloc_matches_csaw_sample_twice(env):
    torch, csaw, L = env
    for g, seeds, io, k, bias in cases():
        G = csaw.Graph(g.off, g.col, g.w)
        ref = csaw.sample(G, seeds, io, [k], bias, 21)
        vs, ins = first_layer(seeds, io)
        for _ in range(2):
            src, dst, off = noalloc(torch, csaw, L, G, vs, ins, k, bias, 21)
            assert np.array_equal(src, ref.src)
            assert np.array_equal(dst, ref.dst)
            # per-instance boundaries agree with csaw_sample's edge offsets
            starts = np.searchsorted(ins, np.arange(len(io) - 1), side="left")
            assert np.array_equal(off[starts], ref.edge_offsets[:-1])
        G.close()


def test_noalloc_rejects_oversized_requests(env):
    torch, csaw, L = env
    g = inputs.rmat_csr(8, 8, 40, 1)
    G = csaw.Graph(g.off, g.col, g.w)
    b = csaw.make_bias("edge_weight")
    too_many = (1 << 20) + 1
    dummy = torch.empty(1, dtype=torch.int32, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    st = L.csaw_select_noalloc(G.handle, p, p, too_many, 5, 0, ctypes.byref(b), 1, p, p,
                               too_many * 5, p, None)
    assert st == csaw.ERR_INVALID
    assert b"at most" in L.csaw_last_error()
    G.close()


def test_noalloc_edge_cases(env):
    """A vertex outside the graph is refused and leaves the next call intact;
    an empty call writes out_offsets[0] = 0; k = CSAW_FANOUT_ALL takes every
    neighbour as csaw_sample does."""
    torch, csaw, L = env
    g = inputs.rmat_csr(12, 16, 100, 12)
    G = csaw.Graph(g.off, g.col, g.w)
    seeds = inputs.uniform_vertices(300, g.V, 4)
    io = np.array([0, 100, 300], dtype=np.uint64)
    vs, ins = first_layer(seeds, io)
    bad = vs.copy()
    bad[len(bad) // 2] = g.V
    assert noalloc(torch, csaw, L, G, bad, ins, 5, "edge_weight", 3, expect=csaw.ERR_INVALID) is None
    assert b"not in the graph" in L.csaw_last_error()
    ref = csaw.sample(G, seeds, io, [5], "edge_weight", 3)
    src, dst, _ = noalloc(torch, csaw, L, G, vs, ins, 5, "edge_weight", 3)
    assert np.array_equal(src, ref.src) and np.array_equal(dst, ref.dst)
    empty = np.zeros(0, dtype=np.uint32)
    src, dst, off = noalloc(torch, csaw, L, G, empty, empty, 5, "edge_weight", 3)
    assert len(src) == 0 and off.tolist() == [0]
    ALL = 0xFFFFFFFF
    for bias in ("edge_weight", "neighbor_degree"):
        ref = csaw.sample(G, seeds, io, [ALL], bias, 8)
        src, dst, off = noalloc(torch, csaw, L, G, vs, ins, ALL, bias, 8)
        assert np.array_equal(src, ref.src) and np.array_equal(dst, ref.dst)
        assert int(off[-1]) == int(np.diff(g.off)[vs.astype(np.int64)].sum())
    G.close()
