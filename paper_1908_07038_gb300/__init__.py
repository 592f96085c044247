"""GB300 (sm_103a) median-dual finite-volume nabla operators on the
octahedral reduced Gaussian grid: gradient, divergence, Laplacian and the
adjoints of gradient and divergence on field[node][level].

``capi`` is the ctypes binding of the C ABI (include/atlas_gb.h) under the
same names; ``atlas`` wraps the handles and takes torch CUDA tensors;
``batch`` holds the persistent batched launch and its autotuner.  Importing
``capi`` (or anything that uses it) needs the built libatlasgb.so.
"""
__all__ = ["capi", "atlas", "batch", "build"]
