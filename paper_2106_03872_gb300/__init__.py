"""GB300-native Kohn-Sham hot path (plane-wave DFT/TDDFT, arXiv 2106.03872).

Submodules: ``ks`` (ctypes binding of include/ks.h, loads the CUDA library), ``build``
(in-tree nvcc build), ``inputs`` (seeded synthetic workloads).  Importing the package
itself loads nothing.
"""
