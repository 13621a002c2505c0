"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds input generators only: mesh coordinates and cells,
per-cell conductivity tensors, stimulus masks and seeded random numbers.
It holds none of the time-stepping or discretisation arithmetic of the
method (no assembly, no ionic model, no Runge-Kutta-Chebyshev recurrence).
Both the CPU oracle and the CUDA path receive exactly the arrays built here.
"""

from .meshes import (  # noqa: F401
    line_mesh,
    square_tri_mesh,
    slab_tet_mesh,
    shell_tet_mesh,
)
from .fields import (  # noqa: F401
    isotropic_D,
    axis_D,
    fibre_D,
    harmonic_sigma,
    corner_mask,
    radius_mask,
    splitmix64,
    u01,
)
from .configs import Workload, make_workload, WORKLOADS  # noqa: F401
