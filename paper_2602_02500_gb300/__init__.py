"""GB300 (sm_103a) implementation of IFNSO, Iteration-Free Newton-Schulz
Orthogonalization (arXiv 2602.02500), behind the C ABI of include/ifnso.h.

* ``paper_2602_02500_gb300._build``  builds libifnso.so in-tree with nvcc.
* ``paper_2602_02500_gb300.ifnso``   the ctypes binding (loads the library;
  raises ImportError if it is missing: there is no non-CUDA fallback).
"""
