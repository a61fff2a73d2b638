"""GB300-native point-cloud tomography (arXiv 2403.07631): tomogram
construction, scene evaluation and slice simplification as hand-written
sm_103a CUDA kernels behind the C ABI of include/tct.h.

``tct`` is the ctypes binding (same names as the C entry points), ``scenes``
the seeded synthetic point-cloud generators, ``build`` the in-tree nvcc build
of libtct.so.  Importing the package does not load the library; the first
call into ``tct`` does, and raises if it has not been built.
"""
__all__ = ["tct", "scenes", "build"]
