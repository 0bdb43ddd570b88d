"""FP64 CPU oracle for Welsch-norm MM non-rigid registration with Anderson
acceleration (Yao, Deng, Xu, Zhang, "Fast and Robust Non-Rigid Registration
Using Accelerated Majorization-Minimization").

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, obviously correct
restatement of the paper in float64 numpy/scipy. It exists to check the CUDA
library. Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import it; the library never calls it and there is no
CPU fallback anywhere in the product path.

It shares no code with the CUDA library. Its only shared dependency is the
seeded input generator ``synth`` (which contains none of the method's
arithmetic).

Modules:
  graph      Sec. 3.1 and Algorithm 1 (Euclidean reading), the edge-length
             normalisation r_ij of Sec. 3.2, mean spacing l-bar.
  geodesic   exact geodesic distances on triangle meshes and Algorithm 1 for
             a mesh source (geodesic D, ball by breadth-first search,
             sub-mesh per node), l-bar as the mean mesh edge length.
  model      Eq. (deformed_position), closest points, Welsch function,
             regularisation residual D_ij, rotation projection, energy Eq. (2).
  surrogate  Sec. 3.3.2 matrix form (W_a, F, Q, W_r, H, Y, J, Z) and the
             normal equations K X = B.
  anderson   Sec. 3.3.4 Anderson acceleration least squares and mix.
  solver     Algorithm 2 (stage loop, MM + AA passes, safeguard).
  unrolled   K plain MM steps at fixed nu and their reverse-mode derivative
             w.r.t. the initial transforms and the source positions.
  lbfgs      the preliminary version's solver (fixed closest points + inner
             L-BFGS with a backtracking line search), a comparison solver.

Parity pins: every function is pinned by the tests in tests/test_oracle_*.py
against closed forms, invariants, brute force and library routines.
"""
from . import graph, geodesic, model, surrogate, anderson, solver, unrolled, lbfgs  # noqa: F401
