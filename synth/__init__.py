"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This package holds no arithmetic of the implicit filter: it only builds meshes
(vertex coordinates, triangle tables, land masks) and random fields.  Both the
CUDA library and the CPU oracle receive the same arrays from here, so any
disagreement between them is a disagreement in the filter itself.

The shapes follow the workloads of the paper (Sect. 3 and 5): split-square
regular triangulations (the paper's Fig. 2 construction), quasi-uniform
unstructured triangulations of the sphere at ~10^4..10^7 vertices with a land
mask, and random fields whose energy spectrum falls as k^-3.
"""

from .meshes import (  # noqa: F401
    periodic_split_square,
    periodic_equilateral,
    icosphere,
    land_mask,
    triangle_centroids,
)
from .fields import (  # noqa: F401
    grf_periodic,
    grf_sphere,
    log_wavenumbers,
)
from .configs import workload, sphere_mesh  # noqa: F401
