"""CPU FP64 oracle for the octree multigrid-preconditioned CG solve.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, links or executes
anything under oracle/; only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline leg use it.  It shares no code with the CUDA library: the octree is built
from per-depth sorted key sets (the library uses dense flag grids), the operator is
an explicit scipy CSR matrix (the library is matrix-free), the coarse operators come
from the paper's Alg. 3 written per coarse cell and are checked against explicit
R A P triple products, and the cycle and Krylov loop are the paper's Alg. 4 and
Alg. 1 written over those matrices.

Modules:
  octree  - refinement, face 2:1 balance, canonical leaf / face / level tables (Sec. 3)
  operator - leaf coefficients (Sec. 2.1, Eq. projection-poisson-system; Sec. 3.1
             T-junction ghosts), Alg. 3 coarsening, level matrices, composite A
  mg      - FAS-style mu-cycle (Alg. 4) and the plain mu-cycle (Alg. 2)
  pcg     - preconditioned CG (Alg. 1); preconditioned BiCGStab for the adjoint system
  adjoint - gradients of a loss through the solve: transpose solve and per-face dL/dbeta

Every function is pinned by tests in tests/test_oracle_*.py against closed forms,
worked values printed in the paper, invariants, brute force and dense solves.
"""
