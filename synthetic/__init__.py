"""Seeded synthetic inputs for the block tridiagonal solver.

This package only *builds* linear systems (the 2D PDE discretisations of
Section 3 and Section 4 of the paper, see ``pde.py``) and right-hand sides.  It
contains none of the solver's arithmetic, so both the CPU oracle and the CUDA
path can consume its outputs without sharing any code with one another.
"""

from .pde import (  # noqa: F401
    BlockTridiag,
    gaussian_random_field,
    poisson,
    variable_diffusion,
    convection_diffusion,
    helmholtz,
    random_blocks,
    strip_kernel_blocks,
    make_config,
    rhs_uniform,
    CONFIGS,
)
