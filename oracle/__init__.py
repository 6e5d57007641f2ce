"""Plain FP64 CPU oracle for one time step of Papanastasiou-regularised
Herschel-Bulkley incompressible flow (Sverdrup, Nikiforakis & Almgren,
arXiv:1803.00417, Sec. III).

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously-correct
restatement of the method that the CUDA library is checked against.  Only the
test-suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` leg of
``bench.py`` (plus its ``--impl reference`` arm) may import it.  It shares no
code with the CUDA path and imports nothing from the product package.

Layout: a d-dimensional array is indexed ``a[i, j(, k)]`` with numpy axis ``a``
equal to spatial direction ``a`` (x, y, z).  Velocities are lists of ``d``
cell-centred arrays, pressure is a nodal array with ``N_a + 1`` points per axis.

Every routine is pinned by a ``-m "not gpu"`` test against something other than
itself (closed forms, dense solves, exact polynomial reproduction, symmetry),
except where its header says "parity unpinned".
"""

from .grid import Grid  # noqa: F401
from .rheology import strain_rate_norm, viscosity  # noqa: F401
from .step import StepResult, step, SolverParams, Rheology  # noqa: F401
