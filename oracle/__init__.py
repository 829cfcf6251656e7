"""Plain FP64 CPU oracle for the batched implicit-Euler / Parareal / MLMC path.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test-suite, the smoke check
of ``__graft_entry__`` and the CPU-baseline / reference arm of ``bench.py``
may import or run anything in this package.  The CUDA path never calls it and
shares no code with it: it has its own assembly, its own direct solver and
its own time loop, written step by step from the paper:

* ``fem``      -- Galerkin matrices M, K and load vectors r of Eq. 3-5 on P1
                  triangles, homogeneous Dirichlet rows/columns eliminated.
* ``stepper``  -- implicit Euler, Eq. 6-7, with a banded Cholesky factor of
                  M/dt + K (reverse Cuthill-McKee ordering) reused each step;
                  the quantities of interest of Eq. 26 and the time-averaged
                  magnetic energy.
* ``parareal`` -- the Parareal update of Eq. 12, serial.
* ``mlmc``     -- the Monte Carlo and telescoping MLMC estimators, Eq. 8-9.
* ``planner``  -- the paper's time/effort model, Eq. 13-25.

Every function is FP64.  Library primitives used as single steps: scipy's
reverse Cuthill-McKee ordering, LAPACK banded Cholesky (``cholesky_banded`` /
``cho_solve_banded``), sparse matrix-vector products and ``math.fsum``.
"""
from . import fem, stepper, parareal, mlmc, planner  # noqa: F401
