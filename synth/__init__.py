"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module only draws numbers and lays out phase maps; it contains none of
the solver's arithmetic (no gradient symbol, projection, constitutive law or
solver step).  Every generator is deterministic given its seed.

Array conventions: a grid is given as ``dims = (Nx, Ny)`` (2D) or
``(Nx, Ny, Nz)`` (3D); arrays are C-ordered with x fastest, i.e. numpy shape
``(Ny, Nx)`` or ``(Nz, Ny, Nx)``.  Phase maps are ``uint8``.
"""
from .micro import (
    grid_shape,
    circular_inclusion,
    random_spheres,
    random_circles,
    laminate,
    gel_sites,
    damage_snapshot,
    random_field,
    five_smooth_sizes,
)

__all__ = [
    "grid_shape",
    "circular_inclusion",
    "random_spheres",
    "random_circles",
    "laminate",
    "gel_sites",
    "damage_snapshot",
    "random_field",
    "five_smooth_sizes",
]
