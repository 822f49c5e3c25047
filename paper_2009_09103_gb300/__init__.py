"""C-SAW biased neighbour selection on GB300.

The compute path is the C-ABI library ``libcsaw.so`` (hand-written CUDA for
sm_103a, declared in ``include/csaw.h``); ``paper_2009_09103_gb300.csaw`` is a
thin ctypes binding over it.  Importing this package loads nothing; the binding
loads the library on first use and raises if it is missing.
"""
