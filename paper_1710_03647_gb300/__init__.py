"""GB300 solver for the initial credit problem of energy games (arXiv 1710.03647).

Submodules:
  gen    seeded synthetic arenas (inputs only)
  eg     ctypes binding of libeg.so, the CUDA solver behind include/eg.h
  build  nvcc build of libeg.so for sm_103a
"""
