"""GB300-native (sm_103a) implementation of the Acc-FEM contact hot path (arXiv 2503.06922).

The compute path is the C-ABI library ``libaccfem.so`` (``include/accfem.h``); ``accfem`` is its
thin ctypes binding.  Build the library with ``paper_2503_06922_gb300.build.build()``.
"""
