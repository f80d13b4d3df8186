"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This package holds no arithmetic of the lattice Boltzmann method itself: only
permeability fields, body-force fields, leaf lists and the unit conversions of
the paper's experiments. Both the oracle tests and the CUDA tests draw their
inputs from here, so the two implementations always see identical inputs.
"""

from .fields import (  # noqa: F401
    gaussian_random_field,
    lognormal_kappa,
    lognormal_kappa3d,
    quadtree_leaves,
    uniform_leaves,
    stratified_tiles,
    channel_kappa,
    block_kappa_eq22,
    layered_kappa,
    checkerboard_kappa,
    fiveblock_kappa_eq23,
    fiveblock_coarse_kappa_eq24,
    sinusoidal_g_field,
    crop_periodic,
)
from .units import LatticeUnits, paper_experiment  # noqa: F401
