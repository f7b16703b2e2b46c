"""FP64 CPU oracle for the GMRES + C-AMG solve phase of arXiv:2112.14681.

TEST INFRASTRUCTURE ONLY. Nothing on the product path imports this package: only the tests,
the smoke check and the CPU-baseline leg of the benchmark call it. It shares no code with the
CUDA path; both sides receive the same inputs from the `workloads` generators.

Contents (each function cites the passage it restates):
  kernels  -- SpMV, splitting A = L + D + U, smoother sweeps (polynomial Gauss-Seidel, ILU(0)
              with Neumann-series triangular solves, ILUT with Jacobi iterations and Ruiz
              scaling (Algorithm 2), l1-Jacobi) in a "definition" mode
              (explicit truncated power sums) and a "direct" mode (forward/backward
              substitution), restriction, prolongation, coarse solve, Gram reduction and
              basis update of the one-reduce Arnoldi step.
  vcycle   -- one Ruge-Stuben V-cycle with zero initial guess.
  setup    -- the Ruge-Stuben setup of Sec. 5.1 (strength, PMIS with SplitMix64 weights,
              BAMG-direct interpolation, Galerkin product, coarse inverse, fixed-point ILU(0)
              factors) that the GPU setup computes.
  gmres    -- classical right-preconditioned MGS-GMRES(m) (Saad-Schultz) and a plain
              restatement of the one-reduce truncated-Neumann MGS-GMRES (Algorithm 1) with
              T = I - L or T = (I + L)^-1.

All arithmetic is float64 (numpy / scipy.sparse library primitives for products).
"""
from . import kernels, vcycle, gmres, setup  # noqa: F401
from .kernels import SmootherParams  # noqa: F401
