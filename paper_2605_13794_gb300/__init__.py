"""gsblitz: GB300-native (sm_103a) CUDA hot path of BlitzGS 3DGS training.

The compute lives in libgsblitz.so (C ABI in include/gsblitz.h); ``binding``
marshals torch CUDA tensors into it.  ``synth`` draws seeded synthetic inputs.
Importing the package does not load the CUDA library; the first call does,
and fails loudly if it has not been built (``build.build()``).
"""
__all__ = ["binding", "synth", "build"]
