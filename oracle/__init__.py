"""Plain FP64 CPU oracle of the lattice Boltzmann no-slip path of
Peng, Ayala & Wang (arXiv 1906.05445).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU-baseline
leg of the benchmark may import this package; the library under
``paper_1906_05445_gb300`` never does.  It shares no code with the CUDA path.
"""
from .oracle import (  # noqa: F401
    BB, BGK, BOUZIDI_LIN, BOUZIDI_QUAD, CYLINDER_Z, D2Q9, D3Q19, IBM, MRT, NONE,
    SPHERE, YU_LIN, YU_QUAD, OracleSim, build, collide, equilibrium,
    ibb_coeffs, ibm_interp, ibm_spread, lattice, lib, mrt_default_rates,
    mrt_matrix, phi,
)
