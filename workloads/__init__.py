"""Seeded synthetic inputs shared by the FP64 oracle tests and the CUDA path.

Holds the parameter container, the SplitMix64 stream, droplet placement and
the initial-field recipes. None of the lattice Boltzmann arithmetic lives here.
"""
from .params import LBMParams
from .rng import SplitMix64
from . import droplets, configs

__all__ = ["LBMParams", "SplitMix64", "droplets", "configs"]
