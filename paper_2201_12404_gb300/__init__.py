"""GB300-native entropic multi-relaxation-time two-phase lattice Boltzmann
(Hosseini, Dorschner & Karlin, arXiv:2201.12404).

The compute path is the CUDA library ``liblbm.so`` (C ABI declared in
``include/lbm.h``); ``paper_2201_12404_gb300.lbm`` is its ctypes binding.
Importing this package loads nothing; the binding loads the library on first
use and raises if it has not been built.
"""
