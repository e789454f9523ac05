"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package holds no arithmetic of the integral-equation method: it only
produces material maps (relative permittivity real part and conductivity per
voxel, and a relative permeability for the magnetic tests), source positions/moments and random coefficient vectors, all from
seeded NumPy PCG64 generators.  The complex permittivity, the susceptibility,
the Green tensors and everything else the method computes are derived
independently by each side from these raw inputs.
"""

from .phantoms import (  # noqa: F401
    Grid,
    sphere_phantom,
    head_phantom,
    body_phantom,
    inclusion_phantom,
    random_tissue,
    random_permeability,
    ring_dipoles,
    body_dipoles,
    inclusion_dipoles,
    random_coefficients,
    workload,
    WORKLOADS,
    serving_stream,
)
