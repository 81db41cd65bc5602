"""GB300 (sm_103a) implementation of the stochastic-collocation lattice
Boltzmann hot path of arXiv:2508.18202: CUDA kernels behind the C ABI of
include/sclbm.h, with a thin ctypes binding (sclbm.py)."""
