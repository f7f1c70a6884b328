"""Seeded synthetic tight-binding inputs for the mArnoldi solver.

This package builds atomic structures (jittered diamond, random-packed amorphous
carbon) and turns them into the sparse LCAO pair (H, S) in block-sparse-row
(BSR) form with 4x4 orbital blocks.  It holds no arithmetic of the mArnoldi
method itself: both the CPU oracle and the CUDA path take its output as input.

The paper (Hoshi, Yamazaki, Akiyama, arXiv:1307.3218) computes on LCAO matrices
H and S that are sparse, real-symmetric and M x M with S positive definite
(Section 2, the text around Eq. 1).  The paper's own structures (the 10^8-atom
sp2-sp3 carbon of Fig. 1(a), the poly-fluorene of Fig. 1(b)) are not available,
so these generators stand in for them with the same shapes: 4 orbitals per
carbon atom, neighbour blocks from atom pairs inside a cutoff.
"""

from .structures import Structure, diamond, amorphous_carbon, spatial_sort
from .polymer import polyfluorene
from .tbmodel import (TBSystem, amorphous_system, build_tb, build_tb_derivatives, carbon_params,
                      config_c1, config_c2, polymer_system, tiny_hydrocarbon, tiny_system)

__all__ = [
    "Structure", "diamond", "amorphous_carbon", "spatial_sort",
    "TBSystem", "build_tb", "build_tb_derivatives", "carbon_params", "config_c1", "config_c2", "tiny_system",
    "amorphous_system", "tiny_hydrocarbon", "polyfluorene", "polymer_system",
]
