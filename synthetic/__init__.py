"""Seeded synthetic inputs for the time-stepped Poisson workloads.

This package only produces inputs (right-hand sides, coefficient fields, grid
sides).  It holds none of the solver's or the network's arithmetic, so both the
FP64 oracle and the CUDA path can draw their inputs from it.

The paper's benchmark moves localized sources ("charged particles") around the
square [-1,1]^2 with zero-Dirichlet walls (Sec. 3, benchmark description;
Fig. "poisson").  Its exact source sequences are not published, so these
generators stand in for them with the same structure: a few signed Gaussian
bumps whose centres and amplitudes change from step to step.
"""

from .rng import SplitMix64, splitmix64_stream, uniform_stream, normal_stream
from .sources import (
    grid_coords,
    MovingGaussians2D,
    RandomWalkSources2D,
    Dipoles2D,
    MovingGaussians3D,
    batched_instances,
    batched_sides,
    lognormal_kappa,
    mode_rhs_2d,
)

__all__ = [
    "SplitMix64", "splitmix64_stream", "uniform_stream", "normal_stream",
    "grid_coords", "MovingGaussians2D", "RandomWalkSources2D", "Dipoles2D", "MovingGaussians3D",
    "batched_instances", "batched_sides", "lognormal_kappa", "mode_rhs_2d",
]
