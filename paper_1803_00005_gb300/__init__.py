"""GB300-native HGF multi-label aggregation + WTA (arXiv 1803.00005).

Submodules:
  hgf   - ctypes binding of the C ABI in include/hgf.h (libhgf.so, built by .build)
  build - nvcc build of libhgf.so for sm_103a
  synth - seeded synthetic stereo / cost-volume inputs
The binding is imported lazily so that the generator can be used without the library.
"""
