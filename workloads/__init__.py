"""Seeded synthetic inputs shared by the CUDA solve path and the CPU oracle.

This package holds matrix and right-hand-side generators and the host-side Ruge-Stuben
setup (strength, PMIS, BAMG-direct interpolation, Galerkin product, ILU(0) factors, coarse
inverse). None of the solve-phase arithmetic (GMRES, V-cycle, smoothers) lives here.
"""
from .matrices import poisson2d_5pt, pressure3d_7pt, q1_27pt_graded, rhs_uniform, edge_sizes  # noqa: F401
from .hierarchy import Hierarchy, Level, build_hierarchy  # noqa: F401
