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


class GraphInfo(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_uint32), ("n_edges", ctypes.c_uint64),
                ("max_degree", ctypes.c_uint32), ("max_weight", ctypes.c_uint32),
                ("device_bytes", ctypes.c_uint64)]


class SampleView(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_uint32), ("n_instances", ctypes.c_uint32),
                ("n_edges", ctypes.c_uint64),
                ("edge_offsets", ctypes.POINTER(ctypes.c_uint64)),
                ("frontier_sizes", ctypes.POINTER(ctypes.c_uint64)),
                ("src", ctypes.POINTER(ctypes.c_void_p)), ("dst", ctypes.POINTER(ctypes.c_void_p))]


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
        if hasattr(L, "csaw_sample"):
            L.csaw_sample.argtypes = [P, P, P, u32, u32, P, ctypes.POINTER(Bias), u64, i32, P,
                                      ctypes.POINTER(P)]
            L.csaw_sample_get_view.argtypes = [P, ctypes.POINTER(SampleView)]
            L.csaw_sample_copy_edges.argtypes = [P, P, P]
            L.csaw_result_free.argtypes = [P]
            L.csaw_result_free.restype = None
        for name in ("csaw_graph_create", "csaw_graph_destroy", "csaw_graph_get_info", "csaw_walk",
                     "csaw_sample", "csaw_sample_get_view", "csaw_sample_copy_edges"):
            if hasattr(L, name):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


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
         path=None, stream=None):
    """csaw_walk.  Device call when `starts` is a torch CUDA tensor (returns a
    torch int32 tensor [n, length+1] holding uint32 vertex ids, asynchronous on
    `stream`); host call when `starts` is a numpy array (returns numpy uint32)."""
    L = lib()
    b = make_bias(bias, mult) if isinstance(bias, str) else bias
    if _is_torch(starts):
        import torch
        n = starts.numel()
        if path is None:
            path = torch.empty((n, length + 1), dtype=torch.int32, device=starts.device)
        _check(L.csaw_walk(g.handle, _ptr(starts), n, length, ctypes.byref(b), seed, _ptr(path),
                           MEM_DEVICE, _stream_handle(stream)))
        return path
    starts = np.ascontiguousarray(starts, dtype=np.uint32)
    n = len(starts)
    if path is None:
        path = np.empty((n, length + 1), dtype=np.uint32)
    st = _stream_handle(stream) if stream is not None else None
    _check(L.csaw_walk(g.handle, _ptr(starts), n, length, ctypes.byref(b), seed, _ptr(path),
                       MEM_HOST, st))
    return path


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


def sample(g: Graph, seeds, inst_offsets, fanout, bias="edge_weight", seed: int = 0,
           stream=None, to_host: bool = True) -> SampleResult:
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
    _check(L.csaw_sample(g.handle, _ptr(seeds), _ptr(inst_offsets), n_inst, len(fan), _ptr(fan),
                         ctypes.byref(b), seed, mem, st, ctypes.byref(out)))
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
