"""Partition planning of out-of-memory walks (host only, no GPU)."""
import ctypes

import numpy as np
import pytest

from paper_2009_09103_gb300 import inputs


@pytest.fixture(scope="module")
def csaw():
    from paper_2009_09103_gb300 import build
    build.build()
    from paper_2009_09103_gb300 import csaw as c
    return c


def need(off, a, b, weighted):
    """Device bytes of partition [a, b): offsets of its rows, then per edge."""
    return 8 * (b - a + 1) + (16 if weighted else 4) * int(off[b] - off[a])


@pytest.mark.parametrize("weighted", [True, False])
def test_plan_ranges_fit_and_are_greedy(csaw, weighted):
    g = inputs.rmat_csr(11, 8, 40, 3)
    off = g.off
    maxrow = int(np.diff(off).max())
    for budget in (need(off, 0, 1, weighted) + (16 if weighted else 4) * maxrow + 64, 50_000, 10**6, 10**12):
        b = csaw.oom_plan(off, budget, weighted)
        assert b[0] == 0 and b[-1] == g.V and (np.diff(b.astype(np.int64)) > 0).all()
        for q in range(len(b) - 1):
            assert need(off, int(b[q]), int(b[q + 1]), weighted) <= budget
            if q + 1 < len(b) - 1:   # greedy: the next row would not fit
                assert need(off, int(b[q]), int(b[q + 1]) + 1, weighted) > budget
        if budget == 10**12:
            assert len(b) == 2


def test_plan_errors(csaw):
    off = np.array([0, 3, 100, 104], dtype=np.uint64)
    with pytest.raises(csaw.CsawError):   # vertex 1's row of 97 edges does not fit
        csaw.oom_plan(off, 16 * 97, True)
    b = csaw.oom_plan(off, 16 * 97 + 16, True)
    assert list(b) == [0, 1, 2, 3]
    L = csaw.lib()
    n = ctypes.c_uint32()
    short = np.empty(2, dtype=np.uint32)
    assert L.csaw_oom_plan(csaw._ptr(off), 3, 1, 16 * 97 + 16, csaw._ptr(short), 2, ctypes.byref(n)) != 0
    bad = np.array([0, 5, 2], dtype=np.uint64)
    with pytest.raises(csaw.CsawError):   # decreasing offsets
        csaw.oom_plan(bad, 10**6, True)
