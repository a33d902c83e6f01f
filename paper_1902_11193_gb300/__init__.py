"""GB300-native D3Q19-MRT lattice Boltzmann permeability solver.

Rao & Schaefer, "Lattice Boltzmann Models for Micro-tomographic Pore-spaces"
(arXiv:1902.11193): Stokes flow through a segmented voxel image with halfway
bounceback, a body force and periodic boundaries, relaxation rates from the
paper's Sets A-E, permeability from the converged mean velocity.

The compute path is the C-ABI library ``liblbm_gb300.so`` (hand-written CUDA
for sm_103a, declared in ``include/lbm.h``); ``lbm`` is its ctypes binding and
``geometry`` the seeded voxel-image generators.  Submodules load lazily, so
importing the package needs no GPU.
"""
__all__ = ["lbm", "geometry"]
