"""GB300-native piston-gap library: the GMAF hot path (arXiv 2511.06824).

`gmaf` is the ctypes binding of the C ABI (include/gmaf.h) implemented by
libgmaf.so; `build` compiles that library for sm_103a; `inputs` generates the
seeded synthetic workloads.  Importing the package loads nothing: the CUDA
library is loaded on first use of the binding and raises if it is missing.
"""
