"""GB300-native grayscale lambda-thinning (sm_103a CUDA kernels behind a C-ABI).

``thin`` is the ctypes binding of libthin.so, ``synth`` the seeded image
generator, ``build`` the in-tree nvcc build.
"""
__all__ = ["thin", "synth", "build"]
