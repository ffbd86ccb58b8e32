"""GB300-native Walk-on-Interfaces estimator (sm_103a CUDA behind a C ABI).

Submodules:
  woi        ctypes binding of libwoi.so (the C ABI in include/woi.h)
  build      compiles libwoi.so for sm_103a
  workloads  seeded synthetic inputs
  parallel   walk-range sharding and moment merging across ranks
"""
