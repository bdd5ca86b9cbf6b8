"""Seeded synthetic inputs for the short-range force path.

This package is shared by the CUDA path's tests and benchmark and by the CPU
oracle's tests.  It holds only input generation: particle sets with the
shapes, sizes and clustering of the paper's workloads, and the default
coefficients of the grid-force polynomial (an input of the force law, Eq. 7
of the paper: the paper fits the filtered grid force but does not print the
fit).  None of the force, binning or list arithmetic lives here.
"""

from .workloads import (  # noqa: F401
    Workload,
    uniform_box,
    lattice_zeldovich,
    clustered_box,
    batched_volumes,
    make_config,
    CONFIG_NAMES,
)
from .gridfit import default_coeffs, fit_coeffs, gaussian_grid_force  # noqa: F401
