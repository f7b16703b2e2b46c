"""One Ruge-Stuben V-cycle used as the GMRES preconditioner (Sec. 5; Sec. 1: one V-cycle of
C-AMG preconditions the Krylov method).

z = vcycle(H, r): level l, starting from x = 0 --
  pre-smooth (forward sweeps), residual, restrict, recurse, prolongate and correct,
  post-smooth (backward sweeps). The coarsest level is solved directly (dense LU) when the
  hierarchy provides a dense inverse, otherwise by `coarse_sweeps` smoother sweeps.
"""
from __future__ import annotations

import numpy as np

from . import kernels as K


def level_smoother(H, l: int, p: K.SmootherParams) -> str:
    """Which smoother runs on level l: 'ilu', 'poly' or 'jacobi' (hybrid = ILU on the finest
    level only, Sec. 6.2)."""
    lev = H.levels[l]
    if p.smoother == K.JACOBI_L1:
        return "jacobi"
    kind = "ilut" if getattr(lev, "ilu_form", 0) == 1 else "ilu"
    if p.smoother == K.ILU0 and lev.ilu_L is not None:
        return kind
    if p.smoother == K.HYBRID_ILU0 and l == 0 and lev.ilu_L is not None:
        return kind
    return "poly"


def smooth(H, l: int, b, x, p: K.SmootherParams, backward: bool):
    lev = H.levels[l]
    kind = level_smoother(H, l, p)
    if kind == "ilu":
        return K.ilu0_sweep(lev.ilu_L, lev.ilu_U, lev.ilu_dinv, lev.A, b, x, p.ilu_terms_L, p.ilu_terms_U, p.mode)
    if kind == "ilut":
        return K.ilut_sweep(lev.ilu_L, lev.ilu_U, lev.ilu_dr, lev.ilu_dc, lev.A, b, x, p.ilu_terms_L, p.ilu_terms_U,
                            p.mode)
    if kind == "jacobi":
        return K.l1_jacobi_sweep(lev.A, b, x)
    return K.poly_gs_sweep(lev.A, b, x, p.neumann_terms, backward=backward, mode=p.mode, ranks=p.ranks)


def vcycle(H, b: np.ndarray, p: K.SmootherParams, l: int = 0) -> np.ndarray:
    lev = H.levels[l]
    if l == H.nlevels - 1:
        if H.coarse_inv is not None:
            return K.coarse_direct(lev.A, b)
        x = np.zeros_like(b)
        for _ in range(p.coarse_sweeps):
            x = smooth(H, l, b, x, p, backward=False)
        return x
    x = np.zeros_like(b)
    for _ in range(p.pre_sweeps):
        x = smooth(H, l, b, x, p, backward=False)
    r = K.residual(lev.A, b, x)
    e = vcycle(H, K.restrict(lev.R, r), p, l + 1)
    x = K.prolong(lev.P, x, e)
    for _ in range(p.post_sweeps):
        x = smooth(H, l, b, x, p, backward=True)
    return x
