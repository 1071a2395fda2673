"""GB300-native lattice information-theoretic clustering (Bauckhage & Kersting, arXiv:1310.7114).

The compute path is the CUDA library ``libitc.so`` (``csrc/``); :mod:`.itc` is its ctypes binding.
Importing this package loads nothing; the library is loaded on first use and its absence is an
error, never a fallback.
"""
