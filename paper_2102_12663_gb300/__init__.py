"""GB300-native coupled lattice Boltzmann solver for aqueous-humor flow
(arXiv 2102.12663): D2Q9 incompressible flow with Boussinesq buoyancy, D2Q4
heat transport and Darcy drag in the trabecular meshwork, behind the C-ABI
library declared in include/lbm.h.

The CUDA library is loaded lazily by ``paper_2102_12663_gb300.lbm``; importing
the package alone loads nothing.
"""
