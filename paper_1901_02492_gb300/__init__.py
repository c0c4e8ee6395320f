"""GB300-native shift-and-stack likelihood search (Whidden et al., arXiv:1901.02492).

The compute path is the C-ABI library libkb.so (include/kb.h) with hand-written
sm_103a kernels; ``binding`` is its thin ctypes binding and ``build`` compiles
it in-tree.  Import ``paper_1901_02492_gb300.binding`` to use the library: the
import fails when libkb.so has not been built (there is no fallback).
"""
__all__ = ["binding", "build"]
