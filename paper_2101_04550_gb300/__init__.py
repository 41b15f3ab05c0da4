"""GB300-native extended lattice Boltzmann step (arXiv 2101.04550).

The compute path is the C-ABI library ``_build/libelbm.so`` (hand-written CUDA
for sm_103a); :mod:`paper_2101_04550_gb300.elbm` is its ctypes binding.  The
library is loaded on first use and its absence is an error: there is no CPU
fallback.
"""
