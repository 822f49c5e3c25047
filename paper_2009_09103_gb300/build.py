"""Build libcsaw.so in-tree for sm_103a with nvcc.

One object per translation unit, compiled in parallel, linked into a shared
library with the CUDA runtime linked statically.  Cross-compiles without a GPU.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJ_DIR = os.path.join(PKG, "_objs")
LIB_PATH = os.path.join(PKG, "libcsaw.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-I", INCLUDE, "-I", CSRC]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers_mtime():
    hs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return max((os.path.getmtime(h) for h in hs), default=0.0)


def _compile(src, extra, verbose):
    obj = os.path.join(OBJ_DIR, os.path.basename(src)[:-3] + ".o")
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), _headers_mtime()) and not extra:
        return obj
    cmd = [_nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stderr}")
    if verbose and r.stderr.strip():
        print(r.stderr)
    os.replace(obj + ".tmp", obj)
    return obj


STATS_LIB_PATH = os.path.join(PKG, "libcsaw_stats.so")
STATS_SOURCES = ("csaw_sample.cu",)   # the translation units that keep selection counters


def _compile_to(src, flags, obj, verbose):
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), _headers_mtime()):
        return obj
    cmd = [_nvcc(), *ARCH, *NVCC_FLAGS, *flags, "-c", src, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)} {' '.join(flags)}:\n{r.stderr}")
    if verbose and r.stderr.strip():
        print(r.stderr)
    os.replace(obj + ".tmp", obj)
    return obj


def _link(objs, path, force):
    newest = max(os.path.getmtime(o) for o in objs)
    if force or not os.path.exists(path) or os.path.getmtime(path) < newest:
        tmp = path + f".tmp{os.getpid()}"
        r = subprocess.run([_nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs],
                           capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc link failed:\n{r.stderr}")
        os.replace(tmp, path)


def build(force: bool = False, verbose: bool = False, extra_flags=(), stats: bool = True) -> str:
    """libcsaw.so, and libcsaw_stats.so (the same library with the selection
    counters of the attempts-per-pick measurement compiled in, -DCSAW_STATS),
    all translation units compiled in parallel."""
    os.makedirs(OBJ_DIR, exist_ok=True)
    srcs = sources()
    if force:
        for o in glob.glob(os.path.join(OBJ_DIR, "*.o")):
            os.remove(o)
    extra = list(extra_flags)
    stem = lambda src: os.path.join(OBJ_DIR, os.path.basename(src)[:-3])
    jobs = [(src, extra, stem(src) + ".o") for src in srcs]
    if extra:   # a one-off variant: always rebuilt
        for _, _, obj in jobs:
            if os.path.exists(obj):
                os.remove(obj)
    stats = stats and not extra
    if stats:
        jobs += [(src, ["-DCSAW_STATS"], stem(src) + "_stats.o") for src in srcs
                 if os.path.basename(src) in STATS_SOURCES]
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        list(ex.map(lambda j: _compile_to(j[0], j[1], j[2], verbose), jobs))
    objs = [stem(src) + ".o" for src in srcs]
    _link(objs, LIB_PATH, force or bool(extra))
    if stats:
        sobjs = [stem(src) + ("_stats.o" if os.path.basename(src) in STATS_SOURCES else ".o") for src in srcs]
        _link(sobjs, STATS_LIB_PATH, force)
    return LIB_PATH


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
