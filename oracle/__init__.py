"""Oracle for C-SAW biased neighbour selection -- TEST INFRASTRUCTURE ONLY.

A ctypes wrapper over ``csaw_ref.c``, a plain single-threaded C statement of
the selection semantics (inverse transform sampling, Sec. II-B Eq. 1;
repeated and updated sampling, Sec. IV-B; EdgeBias, Eq. 3; the sampling loop
of Fig. 2(b) with Update, Eq. 4; random walk and node2vec, Sec. II-A).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library and never calls it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csaw_ref.c")
_LIB_PATH = os.path.join(_HERE, "libcsaw_ref.so")
# The mutation test points this at a deliberately broken build of csaw_ref.c.
_LIB_OVERRIDE = os.environ.get("CSAW_ORACLE_LIB")
_lib = None

NONE = 0xFFFFFFFF
FANOUT_ALL = 0xFFFFFFFF
ATTEMPT_CAP = 1024
BIAS = {"uniform": 0, "edge_weight": 1, "neighbor_degree": 2, "node2vec": 3}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (single-threaded C, -O2)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        if _LIB_OVERRIDE:
            lib = ctypes.CDLL(_LIB_OVERRIDE)
        else:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        u32, u64, i32, i64 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_int64
        lib.ref_philox4x32_10.argtypes = [P, P, P]
        lib.ref_philox4x32_10.restype = None
        lib.ref_draw.argtypes = [u64, u32, u32, u32, u32]
        lib.ref_draw.restype = u64
        lib.ref_scale.argtypes = [u64, u64]
        lib.ref_scale.restype = u64
        lib.ref_select_given_draws.argtypes = [P, u32, u32, u32, P, u32, P]
        lib.ref_select_given_draws.restype = i64
        lib.ref_select.argtypes = [P, P, P, u32, u32, u32, i32, P, u32, u64, u32, u32, u32, P]
        lib.ref_select.restype = i64
        lib.ref_walk.argtypes = [P, P, P, u32, P, P, u64, u32, i32, P, u64, P]
        lib.ref_walk.restype = i32
        lib.ref_walk_tele.argtypes = [P, P, P, u32, P, P, u64, u32, i32, P, u64, i32, u32, P]
        lib.ref_walk_tele.restype = i32
        lib.ref_sample.argtypes = [P, P, P, u32, P, P, u32, u32, P, i32, P, u64, u32,
                                   P, P, P, P]
        lib.ref_sample.restype = i32
        lib.ref_layer_sample.argtypes = [P, P, P, u32, P, P, u32, u32, P, i32, u64, u32, P, P, P, P]
        lib.ref_layer_sample.restype = i32
        lib.ref_mdrw.argtypes = [P, P, u32, P, P, u64, u32, u32, u64, P, P]
        lib.ref_mdrw.restype = i32
        lib.ref_free.argtypes = [P]
        lib.ref_free.restype = None
        lib.ref_stats.argtypes = [P, i32]
        lib.ref_stats.restype = None
        _lib = lib
    return _lib


def stats(reset: bool = False):
    """(draws consumed, picks of the selections that drew) since the last
    reset: the attempts-per-pick count of the selections run so far."""
    out = np.zeros(2, dtype=np.uint64)
    _load().ref_stats(_p(out), int(reset))
    return int(out[0]), int(out[1])


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _u32(a):
    return np.ascontiguousarray(a, dtype=np.uint32)


def philox4x32_10(ctr, key):
    lib = _load()
    c = _u32(ctr); k = _u32(key); out = np.empty(4, dtype=np.uint32)
    lib.ref_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def draw(seed: int, attempt: int, vertex: int, layer: int, instance: int) -> int:
    return int(_load().ref_draw(seed, attempt, vertex, layer, instance))


def scale(r: int, total: int) -> int:
    return int(_load().ref_scale(r, total))


def select_given_draws(b, k: int, draws, attempt_cap: int = ATTEMPT_CAP):
    """Selection on explicit biases with explicit 64-bit draws (draws[a] is
    attempt a).  Returns candidate indices in pick order, or None if the draws
    ran out before k distinct picks."""
    lib = _load()
    b = _u32(b)
    d = np.ascontiguousarray(draws, dtype=np.uint64)
    out = np.empty(max(len(b), 1), dtype=np.uint32)
    n = lib.ref_select_given_draws(_p(b), len(b), k, attempt_cap, _p(d), len(d), _p(out))
    if n == -1:
        return None
    if n < 0:
        raise MemoryError("oracle allocation failed")
    return out[:n].copy()


def _graph_args(g):
    off = np.ascontiguousarray(g.off, dtype=np.uint64)
    col = _u32(g.col)
    w = _u32(g.w) if g.w is not None else None
    return off, col, w


def select(g, v: int, k: int, bias: str, seed: int, layer: int, instance: int,
           prev: int = NONE, mult=(1, 1, 1), attempt_cap: int = ATTEMPT_CAP):
    lib = _load()
    off, col, w = _graph_args(g)
    m = _u32(mult)
    d = int(off[v + 1] - off[v])
    out = np.empty(max(d, 1), dtype=np.uint32)
    n = lib.ref_select(_p(off), _p(col), _p(w), len(off) - 1, v, k, BIAS[bias], _p(m), prev,
                       seed, layer, instance, attempt_cap, _p(out))
    if n < 0:
        raise ValueError(f"oracle select failed ({n})")
    return out[:n].copy()


TELEPORT = {None: 0, "restart": 1, "jump": 2}


def walk(g, starts, length: int, bias: str, seed: int, mult=(1, 1, 1), walker_ids=None,
         teleport=None, teleport_q32: int = 0):
    """Path matrix uint32[n][length+1]; walker_ids (uint64) gives the RNG
    instance of each row when only a subset of walkers is run.  teleport
    ("restart" or "jump") with probability teleport_q32 / 2^32 per step."""
    lib = _load()
    off, col, w = _graph_args(g)
    s = _u32(starts)
    ids = np.ascontiguousarray(walker_ids, dtype=np.uint64) if walker_ids is not None else None
    m = _u32(mult)
    path = np.empty((len(s), length + 1), dtype=np.uint32)
    if teleport is None:
        rc = lib.ref_walk(_p(off), _p(col), _p(w), len(off) - 1, _p(s), _p(ids), len(s), length,
                          BIAS[bias], _p(m), seed, _p(path))
    else:
        rc = lib.ref_walk_tele(_p(off), _p(col), _p(w), len(off) - 1, _p(s), _p(ids), len(s), length,
                               BIAS[bias], _p(m), seed, TELEPORT[teleport], teleport_q32, _p(path))
    if rc != 0:
        raise ValueError(f"oracle walk failed ({rc})")
    return path


def mdrw(g, pools, steps: int, seed: int, instance_ids=None):
    """Multi-dimensional random walk.  pools: uint32[n][pool_size] initial
    pools.  Returns (src, dst), each uint32[n][steps]; instance_ids (uint64)
    gives the RNG instance of each row when only a subset is run."""
    lib = _load()
    off, col, _ = _graph_args(g)
    pl = np.ascontiguousarray(pools, dtype=np.uint32)
    if pl.ndim != 2 or pl.shape[1] == 0:
        raise ValueError("pools must be [n][pool_size] with pool_size >= 1")
    ids = np.ascontiguousarray(instance_ids, dtype=np.uint64) if instance_ids is not None else None
    n, m = pl.shape
    src = np.empty((n, steps), dtype=np.uint32)
    dst = np.empty((n, steps), dtype=np.uint32)
    rc = lib.ref_mdrw(_p(off), _p(col), len(off) - 1, _p(pl), _p(ids), n, m, steps, seed, _p(src), _p(dst))
    if rc != 0:
        raise ValueError(f"oracle mdrw failed ({rc})")
    return src, dst


def sample(g, seeds, inst_offsets, fanout, bias: str, seed: int, attempt_cap: int = ATTEMPT_CAP,
           layer: bool = False):
    """Layered sampling (layer=True: layer sampling, fanout[l] pool entries
    per instance and layer).  Returns dict with src, dst (uint32), edge_off
    (uint64[depth*n_inst+1], grouped by layer then instance) and fsize
    (uint64[(depth+1)*n_inst], frontier size per layer and instance)."""
    lib = _load()
    off, col, w = _graph_args(g)
    s = _u32(seeds)
    io = np.ascontiguousarray(inst_offsets, dtype=np.uint64)
    fo = _u32(fanout)
    m = _u32((1, 1, 1))
    n_inst = len(io) - 1
    depth = len(fo)
    ps, pd, pe, pf = (ctypes.c_void_p() for _ in range(4))
    if layer:
        rc = lib.ref_layer_sample(_p(off), _p(col), _p(w), len(off) - 1, _p(s), _p(io), n_inst, depth,
                                  _p(fo), BIAS[bias], seed, attempt_cap,
                                  ctypes.byref(ps), ctypes.byref(pd), ctypes.byref(pe), ctypes.byref(pf))
    else:
        rc = lib.ref_sample(_p(off), _p(col), _p(w), len(off) - 1, _p(s), _p(io), n_inst, depth, _p(fo),
                            BIAS[bias], _p(m), seed, attempt_cap,
                            ctypes.byref(ps), ctypes.byref(pd), ctypes.byref(pe), ctypes.byref(pf))
    if rc != 0:
        raise ValueError(f"oracle sample failed ({rc})")
    eo = np.ctypeslib.as_array((ctypes.c_uint64 * (depth * n_inst + 1)).from_address(pe.value)).copy()
    total = int(eo[-1])
    src = np.ctypeslib.as_array((ctypes.c_uint32 * max(total, 1)).from_address(ps.value))[:total].copy()
    dst = np.ctypeslib.as_array((ctypes.c_uint32 * max(total, 1)).from_address(pd.value))[:total].copy()
    fs = np.ctypeslib.as_array((ctypes.c_uint64 * ((depth + 1) * n_inst)).from_address(pf.value)).copy()
    for p in (ps, pd, pe, pf):
        lib.ref_free(p)
    return {"src": src, "dst": dst, "edge_off": eo, "fsize": fs}
