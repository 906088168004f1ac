"""GB300-native interior-penalty DG solver for alpha u - eps Lap u + b.grad u = f
(Uzunca & Karasozen, arXiv:1502.02941).

The compute path lives in the CUDA library ``libdg.so`` (``csrc/``) behind the
C ABI declared in ``include/dg.h``; ``dg`` is its ctypes binding.  Importing
this package does not load the library; ``dg.load()`` does, and fails loudly
when it has not been built.
"""
__all__ = ["dg", "workloads", "build"]
