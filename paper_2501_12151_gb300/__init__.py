"""GB300-native tensor-network FEM solver for linear elasticity (QTT + AMEn).

The compute path lives in the CUDA/C++ library ``libtnfem.so`` built from ``csrc/``; the
Python module ``paper_2501_12151_gb300.tnfem`` is a thin ctypes binding over its C ABI
(``include/tnfem.h``).  Importing this package does not load the library; importing
``paper_2501_12151_gb300.tnfem`` does, and raises if it has not been built.
"""
