"""GB300-native geometric multigrid for the nodal ghost finite element method.

The compute path lives in ``csrc/`` (CUDA for sm_103a behind a C ABI declared
in ``include/ghostmg.h``); ``ghostmg`` is the thin ctypes binding.
"""
