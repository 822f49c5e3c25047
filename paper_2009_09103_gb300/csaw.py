"""Thin ctypes binding over libcsaw (include/csaw.h).

Argument marshalling only: every step of selection runs in the library's CUDA
kernels.  Device buffers are torch CUDA tensors (int32 storage holding uint32
values); host buffers are numpy arrays.  The library must have been built
(``__graft_entry__.build()`` or ``python -m paper_2009_09103_gb300.build``);
loading fails loudly otherwise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcsaw.so")
# CSAW_LIB_VARIANT=stats loads the build with the selection counters
# (csaw_selection_stats); it must be set before the first call
if os.environ.get("CSAW_LIB_VARIANT") == "stats":
    LIB_PATH = os.path.join(_PKG, "libcsaw_stats.so")
# CSAW_LIB_PATH points the binding at another build of the library
if os.environ.get("CSAW_LIB_PATH"):
    LIB_PATH = os.environ["CSAW_LIB_PATH"]

OK, ERR_INVALID, ERR_NOMEM, ERR_CUDA, ERR_OVERFLOW, ERR_TIMEOUT, ERR_ABORTED, ERR_NOT_FOUND = range(8)
MEM_HOST, MEM_DEVICE = 0, 1
NONE = 0xFFFFFFFF
FANOUT_ALL = 0xFFFFFFFF
ATTEMPT_CAP = 1024
BIAS_KINDS = {"uniform": 0, "edge_weight": 1, "neighbor_degree": 2, "node2vec": 3}

_lib = None


class CsawError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"csaw status {status}: {msg}")
        self.status = status


class Bias(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n2v_mult", ctypes.c_uint32 * 3)]


class WalkOpts(ctypes.Structure):
    _fields_ = [("teleport", ctypes.c_int32), ("teleport_q32", ctypes.c_uint32), ("build_cdf", ctypes.c_uint32),
                ("phase_ms", ctypes.POINTER(ctypes.c_float))]


TELEPORT = {None: 0, "restart": 1, "jump": 2}


class OomStats(ctypes.Structure):
    _fields_ = [("partitions", ctypes.c_uint32), ("loads", ctypes.c_uint64), ("bytes_loaded", ctypes.c_uint64),
                ("reuses", ctypes.c_uint64), ("pinned_bytes", ctypes.c_uint64), ("direct", ctypes.c_uint32)]


class OomOpts(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_uint32), ("pin_host", ctypes.c_uint32), ("direct", ctypes.c_uint32)]


class GraphInfo(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_uint32), ("n_edges", ctypes.c_uint64),
                ("max_degree", ctypes.c_uint32), ("max_weight", ctypes.c_uint32),
                ("device_bytes", ctypes.c_uint64)]


class SampleOpts(ctypes.Structure):
    _fields_ = [("attempt_cap", ctypes.c_uint32)]


class SelectTuning(ctypes.Structure):
    _fields_ = [("theta_warp", ctypes.c_uint32), ("blocks_per_sm", ctypes.c_uint32)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_uint64), ("slots", ctypes.c_uint32), ("max_batch", ctypes.c_uint32)]


class Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("bias", Bias), ("rng_seed", ctypes.c_uint64),
                ("seeds", ctypes.c_void_p), ("inst_offsets", ctypes.c_void_p),
                ("n_instances", ctypes.c_uint32), ("depth", ctypes.c_uint32), ("fanout", ctypes.c_void_p),
                ("starts", ctypes.c_void_p), ("n_walkers", ctypes.c_uint64), ("length", ctypes.c_uint32)]


class Result(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint32), ("kind", ctypes.c_int32), ("status", ctypes.c_int),
                ("depth", ctypes.c_uint32), ("n_instances", ctypes.c_uint32), ("n_edges", ctypes.c_uint64),
                ("edge_offsets", ctypes.POINTER(ctypes.c_uint64)),
                ("frontier_sizes", ctypes.POINTER(ctypes.c_uint64)),
                ("src", ctypes.POINTER(ctypes.c_uint32)), ("dst", ctypes.POINTER(ctypes.c_uint32)),
                ("n_walkers", ctypes.c_uint64), ("length", ctypes.c_uint32),
                ("path", ctypes.POINTER(ctypes.c_uint32)),
                ("device_bytes_estimate", ctypes.c_uint64),
                ("t_submit_ns", ctypes.c_int64), ("t_admit_ns", ctypes.c_int64),
                ("t_start_ns", ctypes.c_int64), ("t_finish_ns", ctypes.c_int64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("pending", ctypes.c_uint32), ("running", ctypes.c_uint32),
                ("bytes_in_use", ctypes.c_uint64), ("budget_bytes", ctypes.c_uint64)]


REQ_SAMPLE, REQ_WALK = 0, 1


class SampleView(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_uint32), ("n_instances", ctypes.c_uint32),
                ("n_edges", ctypes.c_uint64),
                ("edge_offsets", ctypes.POINTER(ctypes.c_uint64)),
                ("frontier_sizes", ctypes.POINTER(ctypes.c_uint64)),
                ("src", ctypes.POINTER(ctypes.c_void_p)), ("dst", ctypes.POINTER(ctypes.c_void_p))]


# csaw_graph_set_allocator's callbacks: alloc(bytes, stream, ctx) -> ptr,
# free(ptr, stream, ctx)
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


def lib():
    """Load libcsaw.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(LIB_PATH)
        P, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
        L.csaw_last_error.restype = ctypes.c_char_p
        L.csaw_version.restype = u32
        L.csaw_graph_create.argtypes = [P, u32, P, P, u64, i32, P, ctypes.POINTER(P)]
        L.csaw_graph_destroy.argtypes = [P]
        L.csaw_graph_get_info.argtypes = [P, ctypes.POINTER(GraphInfo)]
        L.csaw_walk.argtypes = [P, P, u64, u32, ctypes.POINTER(Bias), u64, P, i32, P]
        L.csaw_walk_ex.argtypes = [P, P, u64, u32, ctypes.POINTER(Bias), u64, P, i32, P,
                                   ctypes.POINTER(WalkOpts)]
        L.csaw_mdrw.argtypes = [P, P, u64, u32, u32, u64, P, P, i32, P]
        L.csaw_oom_plan.argtypes = [P, u32, i32, u64, P, u32, ctypes.POINTER(u32)]
        L.csaw_walk_oom.argtypes = [P, P, P, u32, u64, u64, P, u64, u32, ctypes.POINTER(Bias), u64, P,
                                    ctypes.POINTER(OomStats), P]
        L.csaw_walk_oom_ex.argtypes = [P, P, P, u32, u64, u64, P, u64, u32, ctypes.POINTER(Bias), u64, P,
                                       ctypes.POINTER(OomStats), P, ctypes.POINTER(OomOpts)]
        L.csaw_walk_oom_ex.restype = ctypes.c_int
        L.csaw_sample_oom.argtypes = [P, P, P, u32, u64, u64, P, P, u32, u32, P, ctypes.POINTER(Bias), u64,
                                      ctypes.POINTER(OomOpts), ctypes.POINTER(OomStats), P, ctypes.POINTER(P)]
        L.csaw_sample_oom.restype = ctypes.c_int
        L.csaw_graph_build_cdf.argtypes = [P, ctypes.c_int32, P]
        L.csaw_selection_stats.argtypes = [P, i32]
        L.csaw_selection_stats.restype = ctypes.c_int
        L.csaw_graph_set_allocator.argtypes = [P, ALLOC_FN, FREE_FN, P]
        L.csaw_graph_set_allocator.restype = ctypes.c_int
        L.csaw_graph_drop_cdf.argtypes = [P, ctypes.c_int32]
        if hasattr(L, "csaw_sample"):
            L.csaw_sample.argtypes = [P, P, P, u32, u32, P, ctypes.POINTER(Bias), u64, i32, P,
                                      ctypes.POINTER(P)]
            L.csaw_sample_ex.argtypes = [P, P, P, u32, u32, P, ctypes.POINTER(Bias), u64, i32, P,
                                         ctypes.POINTER(SampleOpts), ctypes.POINTER(P)]
            L.csaw_layer_sample.argtypes = [P, P, P, u32, u32, P, ctypes.POINTER(Bias), u64, i32, P,
                                            ctypes.POINTER(SampleOpts), ctypes.POINTER(P)]
            L.csaw_sample_get_view.argtypes = [P, ctypes.POINTER(SampleView)]
            L.csaw_sample_copy_edges.argtypes = [P, P, P]
            L.csaw_result_free.argtypes = [P]
            L.csaw_result_free.restype = None
        PP = ctypes.POINTER(P)
        L.csaw_sample_plan_create.argtypes = [P, u32, u64, u32, P, ctypes.POINTER(Bias), PP]
        L.csaw_sample_plan_create_ex.argtypes = [P, u32, u64, u32, P, ctypes.POINTER(Bias),
                                                 ctypes.POINTER(SampleOpts), PP]
        L.csaw_sample_plan_run.argtypes = [P, P, u64, P, u64, i32, P]
        L.csaw_sample_plan_get_view.argtypes = [P, ctypes.POINTER(SampleView)]
        L.csaw_sample_plan_copy_edges.argtypes = [P, P, P]
        L.csaw_sample_plan_get_info.argtypes = [P, ctypes.POINTER(u64), ctypes.POINTER(u32), ctypes.POINTER(u32)]
        L.csaw_sample_plan_destroy.argtypes = [P]
        L.csaw_set_select_tuning.argtypes = [P, ctypes.c_int32, ctypes.POINTER(SelectTuning)]
        L.csaw_get_select_tuning.argtypes = [P, ctypes.c_int32, ctypes.POINTER(SelectTuning)]
        L.csaw_autotune_select.argtypes = [P, P, P, u32, u32, P, ctypes.POINTER(Bias), u64, P,
                                           ctypes.POINTER(SelectTuning)]
        L.csaw_server_create.argtypes = [P, ctypes.POINTER(ServerOpts), PP]
        L.csaw_server_destroy.argtypes = [P]
        L.csaw_submit.argtypes = [P, ctypes.POINTER(Request), ctypes.POINTER(u64)]
        L.csaw_poll.argtypes = [P, u64, ctypes.c_int64, ctypes.POINTER(ctypes.POINTER(Result))]
        L.csaw_cancel.argtypes = [P, u64]
        L.csaw_server_stats.argtypes = [P, ctypes.POINTER(ServerStats)]
        for name in ("csaw_graph_create", "csaw_graph_destroy", "csaw_graph_get_info", "csaw_walk",
                     "csaw_graph_build_cdf", "csaw_graph_drop_cdf",
                     "csaw_sample", "csaw_sample_ex", "csaw_sample_get_view", "csaw_sample_copy_edges",
                     "csaw_sample_plan_create", "csaw_sample_plan_create_ex", "csaw_sample_plan_run", "csaw_sample_plan_get_view",
                     "csaw_sample_plan_copy_edges", "csaw_sample_plan_get_info", "csaw_sample_plan_destroy",
                     "csaw_set_select_tuning", "csaw_get_select_tuning", "csaw_autotune_select",
                     "csaw_server_create", "csaw_server_destroy", "csaw_submit", "csaw_poll", "csaw_cancel",
                     "csaw_server_stats"):
            if hasattr(L, name):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def selection_stats(reset: bool = False):
    """csaw_selection_stats (a library built with the counters, i.e. loaded
    with CSAW_LIB_VARIANT=stats): draws consumed, picks of the selections
    that drew, draws evaluated, updated-sampling picks, warp / CTA / hub
    items."""
    out = np.zeros(8, dtype=np.uint64)
    _check(lib().csaw_selection_stats(_ptr(out), int(reset)))
    keys = ("draws_consumed", "drawn_picks", "draws_evaluated", "updated_picks", "warp_items", "cta_items",
            "hub_items")
    return {k: int(v) for k, v in zip(keys, out)}


def _check(status: int):
    if status != OK:
        raise CsawError(status, lib().csaw_last_error().decode(errors="replace"))


def make_bias(kind: str, mult=(1, 1, 1)) -> Bias:
    b = Bias()
    b.kind = BIAS_KINDS[kind] if isinstance(kind, str) else int(kind)
    for i in range(3):
        b.n2v_mult[i] = int(mult[i])
    return b


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    if x is None:
        return None
    if _is_torch(x):
        return ctypes.c_void_p(x.data_ptr())
    return ctypes.c_void_p(x.ctypes.data)


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Graph:
    """Device-resident CSR graph (csaw_graph_create)."""

    def __init__(self, off, col, w=None, stream=None):
        L = lib()
        self._h = ctypes.c_void_p()
        if _is_torch(off):
            mem = MEM_DEVICE
            V = off.numel() - 1
            E = col.numel()
            st = _stream_handle(stream)
            keep = (off, col, w)
        else:
            mem = MEM_HOST
            off = np.ascontiguousarray(off, dtype=np.uint64)
            col = np.ascontiguousarray(col, dtype=np.uint32)
            w = None if w is None else np.ascontiguousarray(w, dtype=np.uint32)
            V, E = len(off) - 1, len(col)
            st = _stream_handle(stream) if stream is not None else None
            keep = (off, col, w)
        _check(L.csaw_graph_create(_ptr(keep[0]), V, _ptr(keep[1]), _ptr(keep[2]), E, mem, st,
                                   ctypes.byref(self._h)))

    @property
    def handle(self):
        return self._h

    def info(self) -> GraphInfo:
        gi = GraphInfo()
        _check(lib().csaw_graph_get_info(self._h, ctypes.byref(gi)))
        return gi

    def build_cdf(self, bias: str, stream=None):
        """csaw_graph_build_cdf: cache the static bias's cumulative array."""
        st = _stream_handle(stream) if stream is not None else None
        _check(lib().csaw_graph_build_cdf(self._h, BIAS_KINDS[bias], st))

    def drop_cdf(self, bias: str):
        _check(lib().csaw_graph_drop_cdf(self._h, BIAS_KINDS[bias]))

    def use_torch_allocator(self, on_alloc=None):
        """csaw_graph_set_allocator with PyTorch's caching allocator: the
        device memory of later calls on this graph is PyTorch's, and counts
        in torch.cuda.memory_allocated().  on_alloc(ptr, nbytes), if given, is
        called after each allocation."""
        import torch
        dev = torch.cuda.current_device()

        def alloc(nbytes, stream, ctx):
            try:
                st = torch.cuda.ExternalStream(stream, device=dev) if stream else None
                ptr = torch.cuda.caching_allocator_alloc(int(nbytes), device=dev, stream=st)
                if on_alloc is not None:
                    on_alloc(ptr, int(nbytes))
                return ptr
            except Exception:
                return None

        def free(ptr, stream, ctx):
            try:
                torch.cuda.caching_allocator_delete(ptr)
            except Exception:
                pass
        self._alloc_cbs = (ALLOC_FN(alloc), FREE_FN(free))   # kept alive with the graph
        _check(lib().csaw_graph_set_allocator(self._h, self._alloc_cbs[0], self._alloc_cbs[1], None))

    def use_own_allocator(self):
        """Back to the library's stream-ordered pool for later calls."""
        _check(lib().csaw_graph_set_allocator(self._h, ALLOC_FN(), FREE_FN(), None))

    def close(self):
        if self._h:
            lib().csaw_graph_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def walk(g: Graph, starts, length: int, bias="edge_weight", seed: int = 0, mult=(1, 1, 1),
         path=None, stream=None, teleport=None, teleport_q32: int = 0, build_cdf: bool = False, phase_ms=None):
    """csaw_walk (csaw_walk_ex with teleport = "restart" or "jump" and a
    per-step probability teleport_q32 / 2^32, or with build_cdf: the call
    builds the kind's cumulative array for itself and walks over it).
    Device call when `starts` is a torch CUDA tensor (returns a torch int32
    tensor [n, length+1] holding uint32 vertex ids, asynchronous on
    `stream`); host call when `starts` is a numpy array (returns numpy
    uint32)."""
    L = lib()
    b = make_bias(bias, mult) if isinstance(bias, str) else bias
    opts = None
    if teleport is not None or build_cdf or phase_ms is not None:
        # phase_ms: a list that receives [build ms, walk ms] (device time, the call waits)
        opts = WalkOpts(TELEPORT[teleport], teleport_q32, 1 if build_cdf else 0)
        if phase_ms is not None:
            ph = (ctypes.c_float * 2)()
            opts.phase_ms = ph

    def call(sp, pp, mem, st):
        if opts is None:
            return L.csaw_walk(g.handle, sp, n, length, ctypes.byref(b), seed, pp, mem, st)
        return L.csaw_walk_ex(g.handle, sp, n, length, ctypes.byref(b), seed, pp, mem, st, ctypes.byref(opts))

    def phases():
        if phase_ms is not None:
            phase_ms[:] = [float(ph[0]), float(ph[1])]

    if _is_torch(starts):
        import torch
        n = starts.numel()
        if path is None:
            path = torch.empty((n, length + 1), dtype=torch.int32, device=starts.device)
        _check(call(_ptr(starts), _ptr(path), MEM_DEVICE, _stream_handle(stream)))
        phases()
        return path
    starts = np.ascontiguousarray(starts, dtype=np.uint32)
    n = len(starts)
    if path is None:
        path = np.empty((n, length + 1), dtype=np.uint32)
    st = _stream_handle(stream) if stream is not None else None
    _check(call(_ptr(starts), _ptr(path), MEM_HOST, st))
    phases()
    return path


def oom_plan(off, budget_bytes: int, weighted: bool = True) -> np.ndarray:
    """csaw_oom_plan: the vertex ranges csaw_walk_oom would use (host only).
    Returns bounds uint32[n_partitions + 1]."""
    L = lib()
    off = np.ascontiguousarray(off, dtype=np.uint64)
    n = ctypes.c_uint32()
    _check(L.csaw_oom_plan(_ptr(off), len(off) - 1, int(weighted), budget_bytes, None, 0, ctypes.byref(n)))
    bounds = np.empty(n.value + 1, dtype=np.uint32)
    _check(L.csaw_oom_plan(_ptr(off), len(off) - 1, int(weighted), budget_bytes, _ptr(bounds), len(bounds),
                           ctypes.byref(n)))
    return bounds


def _oom_stats(st):
    return {"partitions": st.partitions, "loads": st.loads, "bytes_loaded": st.bytes_loaded, "reuses": st.reuses,
            "pinned_bytes": st.pinned_bytes, "direct": st.direct}


def walk_oom(off, col, w, starts, length: int, bias="edge_weight", seed: int = 0,
             budget_bytes: int = 1 << 30, stream=None, slots=None, pin_host: bool = False, direct: bool = False):
    """csaw_walk_oom (slots None) or csaw_walk_oom_ex: walks over a host CSR
    (numpy off uint64, col uint32, w uint32 or None) streamed through slots
    of `budget_bytes` of device memory, or (direct) read in place where the
    device reads host memory coherently.  Returns (path uint32[n, length+1],
    stats dict)."""
    L = lib()
    off = np.ascontiguousarray(off, dtype=np.uint64)
    col = np.ascontiguousarray(col, dtype=np.uint32)
    w = np.ascontiguousarray(w, dtype=np.uint32) if w is not None else None
    starts = np.ascontiguousarray(starts, dtype=np.uint32)
    b = make_bias(bias) if isinstance(bias, str) else bias
    path = np.empty((len(starts), length + 1), dtype=np.uint32)
    st = OomStats()
    sh = _stream_handle(stream) if stream is not None else None
    if slots is None and not pin_host and not direct:
        _check(L.csaw_walk_oom(_ptr(off), _ptr(col), _ptr(w), len(off) - 1, len(col), budget_bytes, _ptr(starts),
                               len(starts), length, ctypes.byref(b), seed, _ptr(path), ctypes.byref(st), sh))
    else:
        o = OomOpts(slots or 0, int(pin_host), int(direct))
        _check(L.csaw_walk_oom_ex(_ptr(off), _ptr(col), _ptr(w), len(off) - 1, len(col), budget_bytes,
                                  _ptr(starts), len(starts), length, ctypes.byref(b), seed, _ptr(path),
                                  ctypes.byref(st), sh, ctypes.byref(o)))
    return path, _oom_stats(st)


def sample_oom(off, col, w, seeds, inst_offsets, fanout, bias="edge_weight", seed: int = 0,
               budget_bytes: int = 1 << 30, slots: int = 0, pin_host: bool = False, stream=None):
    """csaw_sample_oom: layered sampling over a host CSR streamed through
    `slots` partition slots of `budget_bytes` each.  Returns (SampleResult
    with host edges, stats dict)."""
    L = lib()
    off = np.ascontiguousarray(off, dtype=np.uint64)
    col = np.ascontiguousarray(col, dtype=np.uint32)
    w = np.ascontiguousarray(w, dtype=np.uint32) if w is not None else None
    seeds = np.ascontiguousarray(seeds, dtype=np.uint32)
    io = np.ascontiguousarray(inst_offsets, dtype=np.uint64)
    fan = np.ascontiguousarray(fanout, dtype=np.uint32)
    b = make_bias(bias) if isinstance(bias, str) else bias
    o = OomOpts(slots, int(pin_host))
    st = OomStats()
    out = ctypes.c_void_p()
    _check(L.csaw_sample_oom(_ptr(off), _ptr(col), _ptr(w), len(off) - 1, len(col), budget_bytes, _ptr(seeds),
                             _ptr(io), len(io) - 1, len(fan), _ptr(fan), ctypes.byref(b), seed, ctypes.byref(o),
                             ctypes.byref(st), _stream_handle(stream) if stream is not None else None,
                             ctypes.byref(out)))
    holder = _SampleHandle(out)
    v = SampleView()
    _check(L.csaw_sample_get_view(out, ctypes.byref(v)))
    ng = v.depth * v.n_instances
    eo = np.ctypeslib.as_array(v.edge_offsets, shape=(ng + 1,)).copy()
    fs = np.ctypeslib.as_array(v.frontier_sizes, shape=(ng,)).copy() if ng else np.zeros(0, np.uint64)
    src = np.empty(v.n_edges, dtype=np.uint32)
    dst = np.empty(v.n_edges, dtype=np.uint32)
    _check(L.csaw_sample_copy_edges(out, _ptr(src), _ptr(dst)))
    del holder
    return SampleResult(v.depth, v.n_instances, v.n_edges, eo, fs, src, dst), _oom_stats(st)


def mdrw(g: Graph, pools, steps: int, seed: int = 0, src=None, dst=None, stream=None):
    """csaw_mdrw (multi-dimensional random walk).  pools is [n_instances,
    pool_size]: a torch CUDA int32 tensor (device call, asynchronous on
    `stream`, returns torch int32 tensors) or a numpy array (host call, returns
    numpy uint32).  Returns (src, dst), each [n_instances, steps]."""
    L = lib()
    if _is_torch(pools):
        import torch
        if pools.dim() != 2:
            raise ValueError("pools must be [n_instances, pool_size]")
        pools = pools.contiguous()
        n, m = pools.shape
        if src is None:
            src = torch.empty((n, steps), dtype=torch.int32, device=pools.device)
        if dst is None:
            dst = torch.empty((n, steps), dtype=torch.int32, device=pools.device)
        _check(L.csaw_mdrw(g.handle, _ptr(pools), n, m, steps, seed, _ptr(src), _ptr(dst),
                           MEM_DEVICE, _stream_handle(stream)))
        return src, dst
    pools = np.ascontiguousarray(pools, dtype=np.uint32)
    if pools.ndim != 2:
        raise ValueError("pools must be [n_instances, pool_size]")
    n, m = pools.shape
    if src is None:
        src = np.empty((n, steps), dtype=np.uint32)
    if dst is None:
        dst = np.empty((n, steps), dtype=np.uint32)
    st = _stream_handle(stream) if stream is not None else None
    _check(L.csaw_mdrw(g.handle, _ptr(pools), n, m, steps, seed, _ptr(src), _ptr(dst), MEM_HOST, st))
    return src, dst


@dataclass
class SampleResult:
    depth: int
    n_instances: int
    n_edges: int
    edge_offsets: np.ndarray      # uint64[depth*n_instances+1]
    frontier_sizes: np.ndarray    # uint64[depth*n_instances]
    src: object                   # host array (all layers), or list of per-layer device tensors
    dst: object


class _SampleHandle:
    def __init__(self, h):
        self.h = h

    def __del__(self):
        try:
            if self.h:
                lib().csaw_result_free(self.h)
        except Exception:
            pass


def layer_sample(g: Graph, seeds, inst_offsets, layer_sizes, bias="edge_weight", seed: int = 0,
                 stream=None, to_host: bool = True, attempt_cap=None) -> SampleResult:
    """csaw_layer_sample (layer sampling: layer_sizes[l] picks per instance
    from the pool of all its frontier's edges).  Same arguments and result
    as sample()."""
    return sample(g, seeds, inst_offsets, layer_sizes, bias, seed, stream, to_host, attempt_cap, _layer=True)


def sample(g: Graph, seeds, inst_offsets, fanout, bias="edge_weight", seed: int = 0,
           stream=None, to_host: bool = True, attempt_cap=None, _layer: bool = False) -> SampleResult:
    """csaw_sample.  seeds/inst_offsets: numpy (host call) or torch CUDA
    tensors (device call).  Returns edges copied to host when to_host, else
    torch tensors that alias a library-owned result kept alive by the returned
    object."""
    L = lib()
    b = make_bias(bias) if isinstance(bias, str) else bias
    fan = np.ascontiguousarray(fanout, dtype=np.uint32)
    out = ctypes.c_void_p()
    if _is_torch(seeds):
        mem = MEM_DEVICE
        n_inst = inst_offsets.numel() - 1
        st = _stream_handle(stream)
    else:
        mem = MEM_HOST
        seeds = np.ascontiguousarray(seeds, dtype=np.uint32)
        inst_offsets = np.ascontiguousarray(inst_offsets, dtype=np.uint64)
        n_inst = len(inst_offsets) - 1
        st = _stream_handle(stream) if stream is not None else None
    opts = SampleOpts(ATTEMPT_CAP if attempt_cap is None else attempt_cap)
    fn = L.csaw_layer_sample if _layer else L.csaw_sample_ex
    _check(fn(g.handle, _ptr(seeds), _ptr(inst_offsets), n_inst, len(fan), _ptr(fan),
              ctypes.byref(b), seed, mem, st, ctypes.byref(opts), ctypes.byref(out)))
    holder = _SampleHandle(out)
    v = SampleView()
    _check(L.csaw_sample_get_view(out, ctypes.byref(v)))
    ng = v.depth * v.n_instances
    eo = np.ctypeslib.as_array(v.edge_offsets, shape=(ng + 1,)).copy()
    fs = np.ctypeslib.as_array(v.frontier_sizes, shape=(ng,)).copy() if ng else np.zeros(0, np.uint64)
    if to_host:
        src = np.empty(v.n_edges, dtype=np.uint32)
        dst = np.empty(v.n_edges, dtype=np.uint32)
        _check(L.csaw_sample_copy_edges(out, _ptr(src), _ptr(dst)))
        return SampleResult(v.depth, v.n_instances, v.n_edges, eo, fs, src, dst)
    # per-layer device arrays (torch int32 views of library-owned memory)
    srcs, dsts = [], []
    for l in range(v.depth):
        n_l = int(eo[(l + 1) * v.n_instances] - eo[l * v.n_instances])
        srcs.append(_wrap_device(v.src[l], n_l, holder))
        dsts.append(_wrap_device(v.dst[l], n_l, holder))
    res = SampleResult(v.depth, v.n_instances, v.n_edges, eo, fs, srcs, dsts)
    res._holder = holder
    return res


def _wrap_device(ptr, n, holder):
    """A torch int32 view of library-owned device memory (kept alive by holder)."""
    import torch

    class _Arr:
        def __init__(self):
            self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<i4",
                                             "data": (int(ptr or 0), False), "version": 2}
    t = torch.as_tensor(_Arr(), device="cuda") if n else torch.empty(0, dtype=torch.int32, device="cuda")
    t._csaw_holder = holder
    return t


# --------------------------------------------------------------------------
# Batched plans (csaw_sample_plan_*)

class SamplePlan:
    """The multi-instance sampling pipeline captured in a CUDA graph."""

    def __init__(self, g: Graph, n_instances: int, max_seeds: int, fanout, bias="edge_weight",
                 attempt_cap=None):
        L = lib()
        self._g = g
        self._fan = np.ascontiguousarray(fanout, dtype=np.uint32)
        b = make_bias(bias) if isinstance(bias, str) else bias
        self._h = ctypes.c_void_p()
        self.n_instances = n_instances
        opts = SampleOpts(ATTEMPT_CAP if attempt_cap is None else attempt_cap)
        _check(L.csaw_sample_plan_create_ex(g.handle, n_instances, max_seeds, len(self._fan), _ptr(self._fan),
                                            ctypes.byref(b), ctypes.byref(opts), ctypes.byref(self._h)))

    def run(self, seeds, inst_offsets, seed: int = 0, stream=None):
        L = lib()
        if _is_torch(seeds):
            n = seeds.numel()
            _check(L.csaw_sample_plan_run(self._h, _ptr(seeds), n, _ptr(inst_offsets), seed, MEM_DEVICE,
                                          _stream_handle(stream)))
        else:
            self._keep = (np.ascontiguousarray(seeds, dtype=np.uint32),
                          np.ascontiguousarray(inst_offsets, dtype=np.uint64))
            st = _stream_handle(stream) if stream is not None else None
            _check(L.csaw_sample_plan_run(self._h, _ptr(self._keep[0]), len(self._keep[0]), _ptr(self._keep[1]),
                                          seed, MEM_HOST, st))

    def result(self) -> SampleResult:
        """Waits for the last run; edges copied to host."""
        L = lib()
        v = SampleView()
        _check(L.csaw_sample_plan_get_view(self._h, ctypes.byref(v)))
        ng = v.depth * v.n_instances
        eo = np.ctypeslib.as_array(v.edge_offsets, shape=(ng + 1,)).copy()
        fs = np.ctypeslib.as_array(v.frontier_sizes, shape=(ng,)).copy() if ng else np.zeros(0, np.uint64)
        src = np.empty(v.n_edges, dtype=np.uint32)
        dst = np.empty(v.n_edges, dtype=np.uint32)
        _check(L.csaw_sample_plan_copy_edges(self._h, _ptr(src), _ptr(dst)))
        return SampleResult(v.depth, v.n_instances, v.n_edges, eo, fs, src, dst)

    def n_edges(self) -> int:
        v = SampleView()
        _check(lib().csaw_sample_plan_get_view(self._h, ctypes.byref(v)))
        return int(v.n_edges)

    def info(self):
        b, t, k = ctypes.c_uint64(), ctypes.c_uint32(), ctypes.c_uint32()
        _check(lib().csaw_sample_plan_get_info(self._h, ctypes.byref(b), ctypes.byref(t), ctypes.byref(k)))
        return {"device_bytes": b.value, "theta_warp": t.value, "select_blocks": k.value}

    def close(self):
        if self._h:
            lib().csaw_sample_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def set_select_tuning(g: Graph, bias: str, theta_warp: int, blocks_per_sm: int = 0):
    t = SelectTuning(theta_warp, blocks_per_sm)
    _check(lib().csaw_set_select_tuning(g.handle, BIAS_KINDS[bias], ctypes.byref(t)))


def get_select_tuning(g: Graph, bias: str):
    t = SelectTuning()
    _check(lib().csaw_get_select_tuning(g.handle, BIAS_KINDS[bias], ctypes.byref(t)))
    return {"theta_warp": t.theta_warp, "blocks_per_sm": t.blocks_per_sm}


def autotune_select(g: Graph, seeds, inst_offsets, fanout, bias="edge_weight", seed: int = 0):
    """csaw_autotune_select on a host workload; returns the chosen tuning."""
    s = np.ascontiguousarray(seeds, dtype=np.uint32)
    io = np.ascontiguousarray(inst_offsets, dtype=np.uint64)
    f = np.ascontiguousarray(fanout, dtype=np.uint32)
    b = make_bias(bias)
    t = SelectTuning()
    _check(lib().csaw_autotune_select(g.handle, _ptr(s), _ptr(io), len(io) - 1, len(f), _ptr(f), ctypes.byref(b),
                                      seed, _stream_handle(None), ctypes.byref(t)))
    return {"theta_warp": t.theta_warp, "blocks_per_sm": t.blocks_per_sm}


# --------------------------------------------------------------------------
# Serving (csaw_server_*, csaw_submit, csaw_poll)

@dataclass
class ServedResult:
    status: int
    kind: int
    sample: object          # SampleResult or None
    path: object            # numpy [n, L+1] or None
    estimate: int
    t_submit_ns: int
    t_admit_ns: int
    t_start_ns: int
    t_finish_ns: int


class Server:
    def __init__(self, g: Graph, budget_bytes: int, slots: int = 4, max_batch: int = 0):
        """max_batch: requests a slot runs together (0 = the library's
        default, 1 = one request per launch)."""
        self._g = g
        o = ServerOpts(budget_bytes, slots, max_batch)
        self._h = ctypes.c_void_p()
        _check(lib().csaw_server_create(g.handle, ctypes.byref(o), ctypes.byref(self._h)))

    def submit_walk(self, starts, length: int, bias="edge_weight", seed: int = 0, mult=(1, 1, 1)) -> int:
        st = np.ascontiguousarray(starts, dtype=np.uint32)
        r = Request()
        r.kind = REQ_WALK
        r.bias = make_bias(bias, mult)
        r.rng_seed = seed
        r.starts = st.ctypes.data
        r.n_walkers = len(st)
        r.length = length
        t = ctypes.c_uint64()
        _check(lib().csaw_submit(self._h, ctypes.byref(r), ctypes.byref(t)))
        return t.value

    def submit_sample(self, seeds, inst_offsets, fanout, bias="edge_weight", seed: int = 0) -> int:
        s = np.ascontiguousarray(seeds, dtype=np.uint32)
        io = np.ascontiguousarray(inst_offsets, dtype=np.uint64)
        f = np.ascontiguousarray(fanout, dtype=np.uint32)
        r = Request()
        r.kind = REQ_SAMPLE
        r.bias = make_bias(bias)
        r.rng_seed = seed
        r.seeds = s.ctypes.data if len(s) else None
        r.inst_offsets = io.ctypes.data
        r.n_instances = len(io) - 1
        r.depth = len(f)
        r.fanout = f.ctypes.data
        t = ctypes.c_uint64()
        _check(lib().csaw_submit(self._h, ctypes.byref(r), ctypes.byref(t)))
        return t.value

    def poll(self, ticket: int, timeout_us: int = -1, copy: bool = True):
        """Returns a ServedResult (raises CsawError on timeout, unknown ticket,
        or a failed request)."""
        L = lib()
        out = ctypes.POINTER(Result)()
        st = L.csaw_poll(self._h, ticket, timeout_us, ctypes.byref(out))
        if not out:
            _check(st)
        r = out.contents
        sample = path = None
        if st == OK and copy:
            if r.kind == REQ_SAMPLE:
                ng = r.depth * r.n_instances
                eo = np.ctypeslib.as_array(r.edge_offsets, shape=(ng + 1,)).copy()
                fs = np.ctypeslib.as_array(r.frontier_sizes, shape=(max(ng, 1),))[:ng].copy()
                n = int(r.n_edges)
                src = np.ctypeslib.as_array(r.src, shape=(max(n, 1),))[:n].copy()
                dst = np.ctypeslib.as_array(r.dst, shape=(max(n, 1),))[:n].copy()
                sample = SampleResult(r.depth, r.n_instances, n, eo, fs, src, dst)
            else:
                n, ln = int(r.n_walkers), int(r.length)
                path = np.ctypeslib.as_array(r.path, shape=(max(n, 1) * (ln + 1),))[: n * (ln + 1)].reshape(n, ln + 1).copy()
        res = ServedResult(st, r.kind, sample, path, r.device_bytes_estimate, r.t_submit_ns, r.t_admit_ns,
                           r.t_start_ns, r.t_finish_ns)
        L.csaw_result_free(ctypes.cast(out, ctypes.c_void_p))
        if st != OK:
            raise CsawError(st, L.csaw_last_error().decode(errors="replace"))
        return res

    def cancel(self, ticket: int):
        _check(lib().csaw_cancel(self._h, ticket))

    def stats(self):
        s = ServerStats()
        _check(lib().csaw_server_stats(self._h, ctypes.byref(s)))
        return {"pending": s.pending, "running": s.running, "bytes_in_use": s.bytes_in_use,
                "budget_bytes": s.budget_bytes}

    def close(self):
        if self._h:
            lib().csaw_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
