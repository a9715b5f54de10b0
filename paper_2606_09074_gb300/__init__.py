"""GB300 (sm_103a) implementation of REFINE's rendering-free primitive
importance, ratio pruning and compaction (arXiv 2606.09074, Sec. 3.2-3.3).

Submodules:
  binding  ctypes binding of the C ABI in include/refine.h (librefine.so)
  build    nvcc build of librefine.so
  synth    seeded synthetic scenes and camera rigs (inputs only)
"""
