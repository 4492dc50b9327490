"""GB300 (sm_103a) implementation of blocked randomized QB (randQB_b) from
Martinsson & Voronin, arXiv:1503.07157.

The computation lives in librqb.so (C ABI declared in include/rqb.h, CUDA
kernels under csrc/); the submodule `rqb` is its Python binding and `build`
compiles it.
"""
