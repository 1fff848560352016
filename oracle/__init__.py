"""Oracle: a plain, slow, FP64 CPU restatement of the implicit filter.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or runs
this package; only the tests, the smoke check and the bench's CPU-baseline leg
do.  It shares no code, table or constant with the CUDA library.

What it computes (Nowak, Danilov, Mueller, Liu, "Implementation of implicit
filter for spatial spectra extraction"):
  * Eq. 1-2: the filtered field solves (1 + gamma (-l^2 Lap)^n) phi_l = phi, gamma = 1/2,
    k = 1/l (Sect. 2.1 and Sect. 6).
  * Sect. 2.1.1: P1 finite elements on median-dual control volumes,
    S = M^L + (1/2) D~ for n = 1 and S = M^L + (1/2) D~ (M^L)^-1 D~ for n = 2,
    with D~_vv' = l^2 int grad N_v . grad N_v'  and  M^L = diag(A_v).
  * Sect. 2.1.2: the vector Laplacian at vertices with the metric operator T
    and the cell-to-vertex projection R, and the simplified cell Laplacian of
    Eq. 6.
  * Sect. 2.2.2: the system is solved in residual form (initial guess phi) by
    conjugate gradients.
  * Coarse-grained spectra: differences of filtered energies over k (Sect. 4
    and 5 use them; the paper prints no formula, see `spectrum`).

Parity status of each function is stated in its module docstring; the pins
that check the oracle against closed forms live in tests/.
"""

from .mesh import ocean_subset, cell_subset, edge_vectors  # noqa: F401
from .operators import (  # noqa: F401
    scalar_vertex_operators, vector_vertex_operators, cell_operators, order_operator,
    voronoi_vertex_operators, circumcenter_cell_operators,
)
from .reorder import rcm_order, check_rcm_order, hilbert_index, curve_keys, curve_order  # noqa: F401
from .solve import (  # noqa: F401
    cg, filter_field, filter_dense, residual_certificate, refined_certificate, relative_residual, Problem,
    lambda_max_minv_k,
    build_problem,
    shifted_factors, filter_shifted,
)
from .spectrum import filtered_energy, spectrum  # noqa: F401
