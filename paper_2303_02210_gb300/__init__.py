"""GB300-native hot path of the growing-tissue lattice Boltzmann method
(Killeen, Partridge, Bertrand & Lee, arXiv 2303.02210).

The compute lives in hand-written CUDA kernels behind a C ABI
(``include/lbm.h``); ``paper_2303_02210_gb300.lbm`` is the thin ctypes binding.
Importing the package loads nothing; the CUDA library is loaded on first use
and its absence is an error, never a fallback.
"""
