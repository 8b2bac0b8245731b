"""GB300-native radar scan simulator (RadaRays method, arXiv 2310.03505).

``rr``      ctypes binding of the C ABI (include/rr.h) -- the product path.
``scenes``  seeded synthetic scenes, sensor settings and poses (inputs only).
``build``   nvcc build of the CUDA library librr.so for sm_103a.
"""
