"""GB300-native algebraic hybridization and static condensation for H(div) (arXiv:1801.08914).

Submodules: `hyb` (ctypes binding of libhyb.so; importing it needs torch and the built
library), `inputs` (seeded synthetic workloads), `build` (nvcc build of libhyb.so).
This package file imports nothing so that `inputs` can be used without CUDA.
"""
