"""Synthetic pressure-Poisson matrices shaped like the paper's workloads.

The paper's own matrices (Nalu-Wind McAlister wing, N = 3.1M/3.2M; PeleLM nodal projection,
N = 1.4M/11M; Sec. 6) are not available; these seeded stand-ins have the same structure:
symmetric positive definite M-matrices from cell-centred finite volumes (PeleLM-like variable
density) and nodal finite elements on stretched meshes (Nalu-Wind-like high aspect ratio).

Every generator returns a scipy.sparse.csr_matrix with float64 values, int32 indices, sorted
column indices and an explicit diagonal.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

# Independent streams per purpose so the density field and the right-hand side never share draws.
_TAG_DENSITY = 1
_TAG_RHS = 2
_TAG_SIZES = 3
_TAG_PERM = 4


def _rng(seed: int, tag: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(tag)])


def _finish(A: sp.spmatrix) -> sp.csr_matrix:
    A = sp.csr_matrix(A)
    A.sum_duplicates()
    A.sort_indices()
    A.indices = A.indices.astype(np.int32, copy=False)
    A.indptr = A.indptr.astype(np.int32, copy=False)
    return A


def poisson2d_5pt(nx: int, ny: int | None = None) -> sp.csr_matrix:
    """2D 5-point -Laplace on nx*ny interior nodes, Dirichlet boundary eliminated.

    Stencil [-1, -1, 4, -1, -1]; natural (x fastest) ordering; n = nx*ny,
    nnz = 5n - 2nx - 2ny.
    """
    ny = nx if ny is None else ny
    n = nx * ny
    idx = np.arange(n).reshape(ny, nx)
    rows = [idx.ravel()]
    cols = [idx.ravel()]
    vals = [np.full(n, 4.0)]
    for a, b in ((idx[:, :-1], idx[:, 1:]), (idx[:-1, :], idx[1:, :])):
        a = a.ravel()
        b = b.ravel()
        rows += [a, b]
        cols += [b, a]
        vals += [np.full(a.size, -1.0), np.full(a.size, -1.0)]
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return _finish(A)


def pressure3d_7pt(e: int, sigma: float = 1.0, seed: int = 0, ey: int | None = None, ez: int | None = None) -> sp.csr_matrix:
    """Cell-centred FV discretisation of -div(rho^-1 grad p) on an e*ey*ez box (h = 1).

    rho = exp(xi), xi ~ N(0, sigma^2) i.i.d. per cell. Interior face coefficient is the harmonic
    mean of rho^-1 on its two cells, 2 / (rho_L + rho_R). Dirichlet p = 0 on the x- and y-faces
    and on z = 0 (ghost cell: 2 * rho_c^-1 added to the diagonal); homogeneous Neumann on
    z = max. The matrix is an SPD M-matrix with n = e*ey*ez rows; for a cube of edge e,
    nnz = n + 6 e^2 (e - 1).
    """
    ey = e if ey is None else ey
    ez = e if ez is None else ez
    n = e * ey * ez
    rho = np.exp(sigma * _rng(seed, _TAG_DENSITY).standard_normal(n)).reshape(ez, ey, e)
    inv = 1.0 / rho
    idx = np.arange(n).reshape(ez, ey, e)
    diag = np.zeros((ez, ey, e))
    rows, cols, vals = [], [], []
    for axis in (2, 1, 0):  # x, y, z neighbours
        sl_a = [slice(None)] * 3
        sl_b = [slice(None)] * 3
        sl_a[axis] = slice(0, -1)
        sl_b[axis] = slice(1, None)
        ra, rb = rho[tuple(sl_a)], rho[tuple(sl_b)]
        coef = 2.0 / (ra + rb)
        diag[tuple(sl_a)] += coef
        diag[tuple(sl_b)] += coef
        a = idx[tuple(sl_a)].ravel()
        b = idx[tuple(sl_b)].ravel()
        c = coef.ravel()
        rows += [a, b]
        cols += [b, a]
        vals += [-c, -c]
    # Dirichlet ghost contributions: x = 0, x = max, y = 0, y = max, z = 0.
    diag[:, :, 0] += 2.0 * inv[:, :, 0]
    diag[:, :, -1] += 2.0 * inv[:, :, -1]
    diag[:, 0, :] += 2.0 * inv[:, 0, :]
    diag[:, -1, :] += 2.0 * inv[:, -1, :]
    diag[0, :, :] += 2.0 * inv[0, :, :]
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return _finish(A)


def _graded_coords(e: int, aspect: float) -> np.ndarray:
    """Node coordinates of e interior nodes on [0, 1] (plus two boundary nodes), with the
    spacing growing geometrically from the z = 0 wall until it reaches the uniform spacing.
    Returns the e + 2 node positions including both boundary nodes."""
    h = 1.0 / (e + 1)
    hmin = h / aspect
    # Find growth ratio q so that spacings hmin*q^k capped at h fill [0, 1] with e+1 cells.
    def total(q):
        s = hmin * q ** np.arange(e + 1)
        return np.minimum(s, h).sum()
    lo, hi = 1.0, 4.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if total(mid) < 1.0:
            lo = mid
        else:
            hi = mid
    s = np.minimum(hmin * hi ** np.arange(e + 1), h)
    s *= 1.0 / s.sum()
    return np.concatenate([[0.0], np.cumsum(s)])


def q1_27pt_graded(e: int, aspect: float = 100.0, seed: int = 0, permute: bool = True) -> sp.csr_matrix:
    """Trilinear (Q1) finite-element Laplacian on e^3 interior nodes of the unit cube.

    Uniform spacing in x and y; in z the spacing is graded geometrically from the z = 0 wall
    with h_x / h_z,min = aspect. Dirichlet on all faces (boundary nodes eliminated). Each row has
    up to 27 entries. With permute=True a seeded symmetric random permutation is applied and
    then reverse Cuthill-McKee, so the stored ordering is an RCM ordering of a scrambled mesh.
    """
    from scipy.sparse.csgraph import reverse_cuthill_mckee

    hx = 1.0 / (e + 1)
    zc = _graded_coords(e, aspect)
    hz = np.diff(zc)  # e + 1 cell heights
    # 1D element matrices (linear elements): stiffness K = [1 -1; -1 1]/h, mass M = h/6 [2 1; 1 2]
    Kx = np.array([[1.0, -1.0], [-1.0, 1.0]]) / hx
    Mx = np.array([[2.0, 1.0], [1.0, 2.0]]) * hx / 6.0
    n1 = e + 2  # nodes per direction incl. boundary
    nint = e
    # Assemble element by element in vectorised form over all (e+1)^3 cells.
    ce = e + 1
    cx, cy, cz = np.meshgrid(np.arange(ce), np.arange(ce), np.arange(ce), indexing="ij")
    cx, cy, cz = cx.ravel(), cy.ravel(), cz.ravel()
    hzc = hz[cz]
    rows, cols, vals = [], [], []
    interior = lambda ix, iy, iz: (ix >= 1) & (ix <= nint) & (iy >= 1) & (iy <= nint) & (iz >= 1) & (iz <= nint)
    lid = lambda ix, iy, iz: (ix - 1) + nint * ((iy - 1) + nint * (iz - 1))
    for a in range(8):
        ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
        for b in range(8):
            bx, by, bz = b & 1, (b >> 1) & 1, (b >> 2) & 1
            Kz = np.where(az == bz, 1.0, -1.0) / hzc
            Mz = np.where(az == bz, 2.0, 1.0) * hzc / 6.0
            v = (Kx[ax, bx] * Mx[ay, by] * Mz + Mx[ax, bx] * Kx[ay, by] * Mz + Mx[ax, bx] * Mx[ay, by] * Kz)
            ix_a, iy_a, iz_a = cx + ax, cy + ay, cz + az
            ix_b, iy_b, iz_b = cx + bx, cy + by, cz + bz
            m = interior(ix_a, iy_a, iz_a) & interior(ix_b, iy_b, iz_b)
            rows.append(lid(ix_a[m], iy_a[m], iz_a[m]))
            cols.append(lid(ix_b[m], iy_b[m], iz_b[m]))
            vals.append(v[m])
    n = nint ** 3
    A = _finish(sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n)))
    if permute:
        perm = _rng(seed, _TAG_PERM).permutation(n)
        A = _finish(A[perm][:, perm])
        rcm = reverse_cuthill_mckee(A, symmetric_mode=True)
        A = _finish(A[rcm][:, rcm])
    return A


def rhs_uniform(n: int, seed: int = 0) -> np.ndarray:
    """Right-hand side b ~ U[-1, 1]^n (float64)."""
    return _rng(seed, _TAG_RHS).uniform(-1.0, 1.0, n)


def edge_sizes(count: int, lo: int, hi: int, seed: int = 0) -> np.ndarray:
    """Cube edges e_s ~ U{lo..hi} (inclusive) for batched / served systems."""
    return _rng(seed, _TAG_SIZES).integers(lo, hi + 1, size=count)
