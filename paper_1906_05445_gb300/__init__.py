"""GB300-native lattice Boltzmann library for curved no-slip walls:
interpolated bounce-back and direct-forcing immersed boundary
(Peng, Ayala & Wang, arXiv 1906.05445).

Importing the package loads nothing; ``paper_1906_05445_gb300.lbm`` binds the
CUDA library (``liblbm.so``) and raises if it has not been built.
"""
__all__ = ["lbm", "workloads"]
