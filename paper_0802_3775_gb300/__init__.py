"""GB300-native Maxwell-Bloch FDTD (Conti & Fratalocchi, arXiv 0802.3775).

Modules
  fdtd    -- ctypes binding of libfdtd.so (the C ABI in include/fdtd.h)
  batch   -- batched persistent stepping of many grids, autotuner
  serve   -- continuous-batching request server
  inputs  -- seeded synthetic inputs (opal sphere lists, probes, workloads)
  build   -- in-tree nvcc build of libfdtd.so (sm_103a)

Importing the package loads nothing; the CUDA library is loaded on first use
of the binding and a missing library raises instead of falling back.
"""
