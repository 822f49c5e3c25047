"""Seeded synthetic inputs for C-SAW workloads: RMAT graphs and seed sets.

Holds none of the selection arithmetic.  The generator is native C
(``csaw_inputs.c``, SplitMix64 streams keyed per item) so every graph and seed
set is a pure function of its parameters and seed, identical on any machine.
Both the CUDA path's tests and the oracle's tests take their inputs from here.

The workloads follow the sampling and random-walk setups of C-SAW's evaluation
(Sec. VI): RMAT graphs stand in for the SNAP graphs of Table II, which are not
available offline.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csaw_inputs.c")
_LIB_PATH = os.path.join(_HERE, "libcsaw_inputs.so")
_lib = None

RMAT_ABC = (0.57, 0.19, 0.19)


def build(force: bool = False) -> str:
    """Compile the generator with gcc (quick; no GPU needed)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC",
                               "-pthread", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        u32, u64, i32, f64 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_double
        lib.csaw_gen_rmat_draws.argtypes = [u32, u64, f64, f64, f64, u64, i32, P, P]
        lib.csaw_gen_build_csr.argtypes = [u32, u64, P, P, P, P, P]
        lib.csaw_gen_build_csr_mt.argtypes = [u32, u64, P, P, i32, P, P, P]
        lib.csaw_gen_weights_mt.argtypes = [u32, P, P, u32, u64, i32, P]
        lib.csaw_gen_weights.argtypes = [u32, P, P, u32, u64, P]
        lib.csaw_gen_uniform_vertices.argtypes = [u64, u32, u64, u64, P]
        lib.csaw_gen_loguniform_sizes.argtypes = [u32, f64, f64, u64, u64, P]
        lib.csaw_gen_distinct_seeds.argtypes = [u32, P, u32, u64, u64, P]
        for f in ("csaw_gen_rmat_draws", "csaw_gen_build_csr", "csaw_gen_build_csr_mt",
                  "csaw_gen_weights", "csaw_gen_weights_mt",
                  "csaw_gen_uniform_vertices", "csaw_gen_loguniform_sizes", "csaw_gen_distinct_seeds"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


@dataclass
class CSRGraph:
    """Host CSR: off uint64[V+1], col uint32[E] (rows ascending), w uint32[E]."""
    off: np.ndarray
    col: np.ndarray
    w: np.ndarray

    @property
    def V(self) -> int:
        return int(self.off.shape[0] - 1)

    @property
    def E(self) -> int:
        return int(self.col.shape[0])

    def degree(self) -> np.ndarray:
        return np.diff(self.off).astype(np.uint32)


def rmat_csr(scale: int, edge_factor: int, wmax: int, seed: int,
             abc=RMAT_ABC, threads: int | None = None) -> CSRGraph:
    """Symmetrised, deduplicated RMAT graph without self-loops, rows sorted."""
    lib = _load()
    V = 1 << scale
    m = edge_factor * V
    threads = threads or min(32, os.cpu_count() or 1)
    src = np.empty(m, dtype=np.uint32)
    dst = np.empty(m, dtype=np.uint32)
    rc = lib.csaw_gen_rmat_draws(scale, m, abc[0], abc[1], abc[2], seed, threads, _p(src), _p(dst))
    if rc:
        raise ValueError(f"csaw_gen_rmat_draws failed ({rc})")
    off = np.empty(V + 1, dtype=np.uint64)
    col = np.empty(2 * m, dtype=np.uint32)
    ne = ctypes.c_uint64(0)
    rc = lib.csaw_gen_build_csr_mt(V, m, _p(src), _p(dst), threads, _p(off), _p(col), ctypes.byref(ne))
    if rc:
        raise MemoryError(f"csaw_gen_build_csr_mt failed ({rc})")
    del src, dst
    col = col[: ne.value].copy()
    w = np.empty(ne.value, dtype=np.uint32)
    rc = lib.csaw_gen_weights_mt(V, _p(off), _p(col), wmax, seed, threads, _p(w))
    if rc:
        raise ValueError("csaw_gen_weights failed")
    return CSRGraph(off, col, w)


def csr_from_edges(V: int, edges, weights=None) -> CSRGraph:
    """Small hand-built graphs: directed edge list -> CSR with sorted rows."""
    edges = list(edges)
    order = sorted(range(len(edges)), key=lambda i: (edges[i][0], edges[i][1]))
    off = np.zeros(V + 1, dtype=np.uint64)
    for u, _ in edges:
        off[u + 1] += 1
    off = np.cumsum(off).astype(np.uint64)
    col = np.array([edges[i][1] for i in order], dtype=np.uint32)
    if weights is None:
        w = np.ones(len(edges), dtype=np.uint32)
    else:
        w = np.array([weights[i] for i in order], dtype=np.uint32)
    return CSRGraph(off, col, w)


def uniform_vertices(n: int, V: int, seed: int, stream: int = 0) -> np.ndarray:
    lib = _load()
    out = np.empty(n, dtype=np.uint32)
    if lib.csaw_gen_uniform_vertices(n, V, seed, stream, _p(out)):
        raise ValueError("bad V")
    return out


def loguniform_sizes(n_inst: int, lo_exp: float, span: float, seed: int, stream: int = 0) -> np.ndarray:
    """n_i = floor(2^(lo_exp + span*u)), u uniform in [0,1)."""
    lib = _load()
    out = np.empty(n_inst, dtype=np.uint64)
    lib.csaw_gen_loguniform_sizes(n_inst, lo_exp, span, seed, stream, _p(out))
    return out


def distinct_seeds(sizes: np.ndarray, V: int, seed: int, stream: int = 0):
    """Distinct seeds per instance; returns (seeds uint32[sum], inst_offsets uint64[n+1])."""
    lib = _load()
    sizes = np.ascontiguousarray(sizes, dtype=np.uint64)
    out = np.empty(int(sizes.sum()), dtype=np.uint32)
    if lib.csaw_gen_distinct_seeds(len(sizes), _p(sizes), V, seed, stream, _p(out)):
        raise ValueError("instance larger than the vertex set")
    offs = np.zeros(len(sizes) + 1, dtype=np.uint64)
    offs[1:] = np.cumsum(sizes)
    return out, offs


# --------------------------------------------------------------------------
# The five workloads.  Sizes follow the configurations this library is
# measured on; the paper's own evaluation uses SNAP graphs (Table II).

@dataclass
class SampleWorkload:
    graph: CSRGraph
    seeds: np.ndarray
    inst_offsets: np.ndarray
    fanout: list
    bias: str
    rng_seed: int


@dataclass
class WalkWorkload:
    graph: CSRGraph
    starts: np.ndarray
    length: int
    bias: str
    n2v_mult: tuple
    rng_seed: int


def workload_sample_s12(graph_seed: int = 12) -> SampleWorkload:
    """RMAT s12 ef16, w in [1,100]; 256 uniform seeds as one instance; depth 2,
    fanout [10, 5]; edge-weight bias; Philox seed 1."""
    g = rmat_csr(12, 16, 100, graph_seed)
    seeds = uniform_vertices(256, g.V, graph_seed, stream=1)
    return SampleWorkload(g, seeds, np.array([0, 256], dtype=np.uint64), [10, 5], "edge_weight", 1)


def workload_walk_s20(graph_seed: int = 20) -> WalkWorkload:
    """RMAT s20 ef16, w in [1,255]; one walker per vertex, length 80; edge weight."""
    g = rmat_csr(20, 16, 255, graph_seed)
    starts = np.arange(g.V, dtype=np.uint32)
    return WalkWorkload(g, starts, 80, "edge_weight", (1, 1, 1), 2)


def workload_node2vec_s22(graph_seed: int = 22) -> WalkWorkload:
    """RMAT s22 ef32, w in [1,15]; one walker per vertex, length 40; node2vec
    p=2, q=0.5 as integer multipliers (1, 2, 4)."""
    g = rmat_csr(22, 32, 15, graph_seed)
    starts = np.arange(g.V, dtype=np.uint32)
    return WalkWorkload(g, starts, 40, "node2vec", (1, 2, 4), 3)


@dataclass
class MdrwWorkload:
    graph: CSRGraph
    pools: np.ndarray     # uint32[n_instances][pool_size]
    steps: int
    rng_seed: int


def workload_mdrw_s20(graph_seed: int = 20, n_inst: int = 2000, pool_size: int = 2000,
                      steps: int = 2000) -> MdrwWorkload:
    """Multi-dimensional random walk on the weighted-walk graph (RMAT s20 ef16):
    2000 instances, each a pool of 2000 vertices drawn uniformly among those
    with an edge (the frontier size of the paper's evaluation, Sec. VI), 2000
    steps; Philox seed 5."""
    g = rmat_csr(20, 16, 255, graph_seed)
    live = np.flatnonzero(np.diff(g.off) > 0).astype(np.uint32)
    idx = uniform_vertices(n_inst * pool_size, len(live), graph_seed, stream=5)
    return MdrwWorkload(g, live[idx].reshape(n_inst, pool_size), steps, 5)


def workload_layer_s20(graph_seed: int = 20, n_inst: int = 2000, seeds_per_inst: int = 64) -> SampleWorkload:
    """Layer sampling on the weighted-walk graph (RMAT s20 ef16): 2000
    instances (the sampling instances of the paper's evaluation, Sec. VI) of
    64 distinct seeds among the vertices with an edge; depth 2, 512 picks per
    instance and layer; edge-weight bias; Philox seed 6."""
    g = rmat_csr(20, 16, 255, graph_seed)
    live = np.flatnonzero(np.diff(g.off) > 0).astype(np.uint32)
    sizes = np.full(n_inst, seeds_per_inst, dtype=np.uint64)
    idx, offs = distinct_seeds(sizes, len(live), graph_seed, stream=6)
    return SampleWorkload(g, live[idx], offs, [512, 512], "edge_weight", 6)


def workload_batched_s24(graph_seed: int = 24, n_inst: int = 4096) -> SampleWorkload:
    """RMAT s24 ef16; 4096 instances of log-uniform [64, 8192) distinct seeds;
    depth 2, fanout [25, 10]; neighbour-degree bias."""
    g = rmat_csr(24, 16, 255, graph_seed)
    sizes = loguniform_sizes(n_inst, 6.0, 7.0, graph_seed, stream=4)
    seeds, offs = distinct_seeds(sizes, g.V, graph_seed, stream=4)
    return SampleWorkload(g, seeds, offs, [25, 10], "neighbor_degree", 4)


def serving_requests(V: int, n: int, seed: int = 5):
    """The serving mix on a graph of V vertices: n requests alternating
    layered sampling and weighted walks.  Sampling: one instance of
    floor(2^(14u)) seeds (at least 1, uniform over the vertices), depth 1-3,
    fanout per layer from {5, 10, 25}, Philox seed 100 + i.  Walks:
    floor(2^(16u)) starts (at least 1, uniform), length uniform in [10, 80],
    Philox seed 200 + i.  Returns tuples ("sample", seeds, inst_offsets,
    fanout, rng_seed) and ("walk", starts, length, rng_seed)."""
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        if i % 2 == 0:
            ns = max(1, int(2 ** (14 * rng.random())))
            seeds = uniform_vertices(ns, V, 10_000 + i)
            depth = int(rng.integers(1, 4))
            fan = [int(x) for x in rng.choice([5, 10, 25], size=depth)]
            reqs.append(("sample", seeds, np.array([0, ns], dtype=np.uint64), fan, 100 + i))
        else:
            nw = max(1, int(2 ** (16 * rng.random())))
            starts = uniform_vertices(nw, V, 20_000 + i)
            reqs.append(("walk", starts, int(rng.integers(10, 81)), 200 + i))
    return reqs


def workload_serve_s26(graph_seed: int = 26) -> CSRGraph:
    """The serving graph: RMAT s26 ef16 (about 2.1 billion directed edges),
    weights uniform in [1, 255]; requests come from serving_requests."""
    return rmat_csr(26, 16, 255, graph_seed)
