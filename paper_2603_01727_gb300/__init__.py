"""GB300 (sm_103a) implementation of one time step of the low-Mach flame-sheet
solver of arXiv 2603.01727 (Severino et al.): C ABI in include/lowmach.h, CUDA
kernels in csrc/, ctypes binding in lowmach.py, in-tree build in build.py."""
