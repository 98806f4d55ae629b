"""GB300-native tree-level QCD matrix elements (arXiv:0909.5257 hot path).

The compute path lives in the CUDA library built from ``csrc/`` and is reached
through the C ABI declared in ``include/mea.h``; ``paper_0909_5257_gb300.mea``
is the thin ctypes binding.  Importing this package loads nothing.
"""
