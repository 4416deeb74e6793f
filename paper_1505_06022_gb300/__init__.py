"""GB300-native stackless-BVH ray casting and stochastic progressive photon mapping.

The compute path is the CUDA library ``_build/libgsp.so`` (C ABI in include/gsp.h); ``gsp``
is its Python binding and ``inputs`` builds seeded synthetic scenes and rays.
"""
__all__ = ["gsp", "inputs", "build"]
