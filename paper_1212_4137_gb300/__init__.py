"""GB300-native alternating-maximization (AM) sparse PCA (Richtarik et al., arXiv 1212.4137).

The package holds:
  * ``csrc/``   -- the CUDA kernels and the C-ABI library ``libspca.so`` (sm_103a);
  * ``spca``    -- a thin ctypes binding with the same names as ``include/spca.h``;
  * ``inputs``  -- seeded synthetic inputs shared by tests and the benchmark
                   (no arithmetic of the method lives there);
  * ``build``   -- the nvcc build step.

Importing the package loads nothing; ``spca.load()`` loads the compiled library and
raises if it is missing.  There is no CPU fallback.
"""

__all__ = ["inputs", "spca", "build"]
