"""Seeded synthetic inputs shared by the oracle tests and the GPU path.

This package draws random numbers and lays out basis sets, coordinates and
densities.  It holds none of the integral arithmetic: no normalisation, no
Gaussian products, no Boys function, no screening.  Both the CPU oracle and
the CUDA library consume the plain arrays it returns.
"""

from .molecules import (  # noqa: F401
    ANGSTROM_TO_BOHR,
    Molecule,
    config_tiny,
    config_medium,
    config_high_l,
    config_scf,
    config_served_requests,
    custom_molecule,
    random_psd_density,
    ncart,
)
