"""Seeded synthetic inputs shared by the CUDA-library tests, the oracle tests
and the benchmark.  Holds no integral arithmetic: only random geometries,
exponents, contraction coefficients (with a conventional normalisation
factor folded in), shell-pair and quartet lists, and weight tensors."""
from .workloads import *  # noqa: F401,F403
