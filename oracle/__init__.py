"""Plain FP64 CPU oracle of the IBM time step (test infrastructure only).

This package is test infrastructure.  Only `tests/`, `__graft_entry__.smoke()`
and the CPU-baseline leg of `bench.py` may import it.  It shares no code with
the CUDA library and never imports the product package; the only thing both
sides consume is the plain data made by `inputs/`.

It follows the paper (Luchini et al., "A simple and efficient second-order
immersed-boundary method for the incompressible Navier-Stokes equations"):
  * staggered grid and 3-point central differences           Sec. 2.1
  * staircase classification and internal-pressure rule       Sec. 3.3
  * IBM centre-weight correction lambda                       Sec. 2.2, Eq. (disclapl-extr), (lambda)
  * implicit exponential-fitted update A w^{n+1} - B w^n = C F Sec. 2.4, Eq. (generic), (Bexpr), (expint)
  * Rai-Moin RK3 combined with the implicit IBM               Eq. (rk3-rai)
  * incremental pressure-correction projection                Sec. 2.1, Sec. 3.3
Every floating-point computation is FP64 numpy, in the order the formulas are
written, with no blocking or fusion.  Where the paper is silent the reading
taken is stated next to the code and listed in the design notes.

A stretched wall-normal grid (face heights given) is supported by the grid, the operators,
the projection, the weights and the steady solver (readings in the design notes, pins in
tests/test_oracle_stretched.py); the force accounting stays uniform-grid only.  A translating
cylinder or sphere (reading in solver.py, pins in tests/test_oracle_moving_body.py) is
reclassified at every step.

Parity status: every function here is pinned by a `-m "not gpu"` test against
a closed form, a value printed in the paper, an invariant or a brute-force
solve (tests/test_oracle_*.py).  No function is "parity unpinned".
"""
from .grid import Grid
from .geometry import LevelSet
from .classify import Classification, classify
from .weights import Weights, build_weights, B_of_x, RK3_A, RK3_B, RK3_C, RK3_T
from .momentum import rhs, stage_update
from .poisson import divergence, gradient, solve_spectral, solve_direct
from .solver import OracleSolver
from . import steady

__all__ = ["Grid", "LevelSet", "Classification", "classify", "Weights", "build_weights",
           "B_of_x", "RK3_A", "RK3_B", "RK3_C", "rhs", "stage_update",
           "divergence", "gradient", "solve_spectral", "solve_direct", "OracleSolver", "steady"]
