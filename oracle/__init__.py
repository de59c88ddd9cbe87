"""Plain FP64 CPU oracle for the O(a)-improved Wilson-Dirac operator of
openQ*D (Sec. 2.3, eqs. dirac, wilson-dirac, frw-covder, bkw-covder, sw-term),
its even-odd preconditioned form (Sec. 2.3, definition of D-hat), the C*
orbifold geometry (Sec. 2.1) and the solvers (Sec. 4.4; App. A).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
baseline leg of the benchmark import this package.  It shares no code with the
CUDA library and never imports it.  Everything here is written for readability
(explicit 4x4 gamma matrices, explicit 3x3 products, no fusion), vectorised
over lattice sites with NumPy.
"""
from .lattice import Geometry  # noqa: F401
from .dirac import Flavour, GaugeField, DiracOperator  # noqa: F401
