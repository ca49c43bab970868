"""FP64 CPU oracle for the quasi-implicit ADS wildfire time step.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference that
the CUDA path is checked against.  Only the test suite, the smoke check of
the build entry point and the CPU-baseline leg of the benchmark may import
or run it; the product path never does.

It shares no code with the CUDA path.  It is written from the paper:

* the energy-balance model and its parameters (Sec. 2, Eq. energy, Table
  "Model parameters") and the normalised operator form (start of Sec. 3);
* the 1-D mass, stiffness and advection matrices (Sec. 3.1 "Matrix
  formulation");
* the Peaceman-Rachford scheme (Sec. 3.1, Eq. PR and its variational and
  Kronecker forms) and the Strang / Crank-Nicolson scheme (Sec. 3.2);
* the right-hand-side integration with fuel depletion (Sec. 7, listing
  "compute_rhs").

Every system is solved as its plain definition: the 2-D operator is
assembled by 2-D Gauss quadrature over the elements (not as a Kronecker
product) and solved by a sparse LU with partial pivoting ("direct" mode).
For grids too large for that, "ads" mode solves the same system by
independent 1-D banded solves with partial pivoting (Sec. 4); the tests pin
"ads" to "direct" on small grids.

Parity status of each function is stated in its module header.
"""
from .physics import Params, derived_constants, source_terms  # noqa: F401
from .bspline import knots, gauss01, eval_local, element_tables  # noqa: F401
from .matrices import matrices_1d, assemble_2d  # noqa: F401
from .rhs import load_vectors  # noqa: F401
from .step import Problem  # noqa: F401
