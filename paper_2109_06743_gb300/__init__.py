"""GB300-native hot path of the moment-fitting PFC Vlasov solver of
Allmann-Rahn, Lautenbach and Grauer (arXiv:2109.06743).

* ``paper_2109_06743_gb300.abi``       -- ctypes binding of the C-ABI library
  ``libvlasov.so`` (hand-written sm_103a CUDA kernels behind ``include/vlasov.h``).
* ``paper_2109_06743_gb300.driver``    -- Algorithm 1 time loop over the C-ABI.
* ``paper_2109_06743_gb300.workloads`` -- seeded synthetic inputs.
* ``paper_2109_06743_gb300.build``     -- nvcc build of the library.

Importing the package does not load the CUDA library; ``abi.lib()`` does, and
raises if it is missing (there is no CPU fallback).
"""
__all__ = ["abi", "driver", "workloads", "build"]
