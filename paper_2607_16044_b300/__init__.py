"""B300-native explicit DG right-hand side for compressible flow.

The compute path is the CUDA library ``libdgx.so`` (built by
``__graft_entry__.build()``) behind the C ABI declared in ``include/dgx.h``;
``paper_2607_16044_b300.dgx`` is its Python binding.  ``inputs`` holds the
seeded mesh / state generators.  Nothing here falls back to the CPU: the
binding raises if the library or a CUDA device is missing.
"""
__all__ = ["inputs", "dgx"]
