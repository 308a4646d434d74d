"""FP64 CPU oracle for BundleFusion's global pose alignment (Dai et al. 2017, Sec. 4.3-4.4).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of what the GPU library computes, used to check it.  Only the test
suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import
it; the library never calls it and shares no code with it.

Layout (each function cites the passage of the paper it restates):
  lie.py          rigid-motion helpers: exponential map, pose composition (Sec. 4.3)
  frames.py       per-frame preprocessing: validity, normals, intensity gradient (Sec. 4.1.1, 4.3)
  association.py  dense projective association, decided in FP32 (Sec. 4.3, dense matching)
  residuals.py    sparse / geometric / photometric residuals and Jacobians (Sec. 4.3)
  system.py       explicit normal equations J^T J dX = -J^T F (Sec. 4.4)
  solver.py       PCG with (block-)Jacobi preconditioner, Gauss-Newton, residual max (Sec. 4.4, 4.4.1)
  hierarchy.py    chunk / keyframe pose composition (Sec. 4.2)

Parity pins (tests/test_oracle_*.py) tie it to the mathematics: zero residual at
ground truth, finite-difference Jacobians, gauge invariance, the Kabsch closed form,
brute-force least squares on tiny problems, PCG against a direct solve, and the
residual count identity R = 3 N_corr + |E| (|I| + |D|) of Sec. 4.4.
"""
from . import lie, frames, association, residuals, system, solver, hierarchy  # noqa: F401
from .system import SolveParams  # noqa: F401
