"""The C-ABI library builds, loads, and exports every entry point that
include/*.h declares (no GPU needed: nothing here calls into the device)."""
import ctypes
import glob
import os
import re

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def libcsaw():
    from paper_2009_09103_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(csaw_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("csaw_graph_create", "csaw_graph_destroy", "csaw_walk", "csaw_sample",
                     "csaw_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(libcsaw):
    missing = [n for n in declared_functions() if not hasattr(libcsaw, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_no_oracle_or_fallback_in_product_path():
    # The product library and its binding never reach the oracle or a CPU path.
    pkg = os.path.join(ROOT, "paper_2009_09103_gb300")
    for f in glob.glob(os.path.join(pkg, "*.py")) + glob.glob(os.path.join(pkg, "csrc", "*")):
        text = open(f).read()
        assert "import oracle" not in text and "from oracle" not in text, f
        assert "csaw_ref" not in text, f


def test_version_and_error_string_without_gpu(libcsaw):
    libcsaw.csaw_version.restype = ctypes.c_uint32
    assert libcsaw.csaw_version() >= 10000
    libcsaw.csaw_last_error.restype = ctypes.c_char_p
    assert isinstance(libcsaw.csaw_last_error(), bytes)
