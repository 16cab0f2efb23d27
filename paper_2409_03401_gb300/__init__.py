"""GB300-native (sm_103a) fused lattice Boltzmann step of the grand-potential
phase-field model for two-phase ternary fluids with flow.

The compute path is the CUDA library liblbm_gb300.so behind the C-ABI of
include/lbm.h; ``Simulation`` binds it to torch-owned device memory.
"""
from .lattice import Simulation, droplet_stats
from ._lib import LBMError

__all__ = ["Simulation", "LBMError", "droplet_stats", "build"]


def build(force=False):
    from .build import build as _build
    return _build(force=force)
