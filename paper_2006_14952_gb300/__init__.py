"""GB300-native Gaussian-truncated short-range FMM (Wang, "A Hybrid Fast
Multipole Method for Cosmological N-body Simulations", Secs. 2.1-2.3).

``hfmm``       - ctypes binding of the C-ABI library ``libhfmm.so`` (argument
                 marshalling only; every step runs in the CUDA kernels).
``workloads``  - seeded synthetic particle sets (no method arithmetic).
``build``      - compiles the CUDA library for sm_103a.
"""
__all__ = ["hfmm", "workloads", "build"]
