"""Plain FP64 CPU oracle for MRCM-OS-preconditioned flexible GMRES.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or execute this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py`` use it.  It shares no code with the CUDA path (``paper_2606_08883_gb300``) and imports
nothing from it; inputs reach it as plain numpy arrays.

Every function follows the paper step by step, in numpy/scipy with float64 throughout:

* ``grid``       -- fine operator A and right-hand side b (Sec. 3, Eq. 1a-1d, two-point-flux reading).
* ``partition``  -- subdomains, oversampled regions, Robin sides, coarse numbering (Sec. 2.1, Fig. 1).
* ``local``      -- Robin / Dirichlet local operators on boxes (Eq. 5-6, Eq. 11, Eq. 15).
* ``mrcm``       -- informed multiplier spaces (Eq. 15), multiscale basis functions, the coupling
                    system (Eq. 13-14), the preconditioner T (modified MRCM-O, Sec. 3) and the
                    overlapping-Schwarz smoothing sweeps (Sec. 2.1, step 4 of MRCM-OS).
* ``gmres``      -- restarted right-preconditioned GMRES storing Z (Algorithm 1).

Parity status per function is listed in each module header; every function here is pinned by a
``-m "not gpu"`` test in ``tests/test_oracle_*.py`` except the paper's table iteration counts, which
depend on readings the paper leaves open (parity unpinned, reported side by side only).
"""

from .grid import (DIRICHLET, NEUMANN, SIDES, face_area, half_transmissibility,  # noqa: F401
                   transmissibilities, rhs, matvec, fluxes)
from .partition import Partition  # noqa: F401
from .mrcm import MRCMOS  # noqa: F401
from .gmres import fgmres  # noqa: F401
from .solve import solve, apply_precond  # noqa: F401
