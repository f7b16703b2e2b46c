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


def _graded_coords(e: int, aspect: float, growth: float = 1.1) -> np.ndarray:
    """Node coordinates (e interior + 2 boundary nodes) on [0, 1] in the wall-normal direction:
    the first cell is h_u / aspect, each next cell is `growth` times the previous one until it
    reaches the uniform size h_u of the remaining cells; h_u is chosen so the cells fill [0, 1]."""
    ncell = e + 1
    k = np.arange(ncell)
    rel = np.minimum(growth ** k / aspect, 1.0)  # cell sizes in units of h_u
    hu = 1.0 / rel.sum()
    return np.concatenate([[0.0], np.cumsum(rel * hu)])


def _fe1d(h: np.ndarray):
    """Assembled 1D linear-element stiffness K and mass M on the interior nodes, for element
    lengths h[0..e] (e interior nodes, Dirichlet ends eliminated)."""
    e = h.size - 1
    Kd = 1.0 / h[:-1] + 1.0 / h[1:]
    Ko = -1.0 / h[1:-1]
    Md = (h[:-1] + h[1:]) / 3.0
    Mo = h[1:-1] / 6.0
    K = sp.diags([Ko, Kd, Ko], [-1, 0, 1], shape=(e, e), format="csr")
    M = sp.diags([Mo, Md, Mo], [-1, 0, 1], shape=(e, e), format="csr")
    return K, M


def _sym_permute(A: sp.csr_matrix, perm: np.ndarray) -> sp.csr_matrix:
    """P A P^T for the ordering `perm` (new row k is old row perm[k]): the host setup library's
    parallel form of scipy's A[perm, :][:, perm] with sorted columns (bitwise the same)."""
    from .hierarchy import _load
    n = A.shape[0]
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    rp = np.ascontiguousarray(A.indptr, dtype=np.int32)
    ci = np.ascontiguousarray(A.indices, dtype=np.int32)
    v = np.ascontiguousarray(A.data, dtype=np.float64)
    brp = np.empty(n + 1, np.int32)
    bci = np.empty(A.nnz, np.int32)
    bv = np.empty(A.nnz, np.float64)
    _load().nsw_sym_permute(n, rp, ci, v, perm, brp, bci, bv)
    B = sp.csr_matrix((bv, bci, brp), shape=A.shape)
    B.has_sorted_indices = True
    return B


def _q1_assemble(Kx, Mx, Kz, Mz) -> sp.csr_matrix:
    """Mz(x)My(x)Kx + Mz(x)Ky(x)Mx + Kz(x)My(x)Mx by the host setup library (the products and
    sums of scipy's kron / + in the same order, so bitwise the same matrix)."""
    from .hierarchy import _load
    e = Kx.shape[0]
    d = lambda M: np.ascontiguousarray(M.diagonal(), dtype=np.float64)
    o = lambda M: np.ascontiguousarray(M.diagonal(1) if e > 1 else np.zeros(1), dtype=np.float64)
    n = e ** 3
    nnz = (3 * e - 2) ** 3
    rp = np.empty(n + 1, np.int64)
    ci = np.empty(nnz, np.int32)
    v = np.empty(nnz, np.float64)
    got = _load().nsw_q1_assemble(e, d(Kx), o(Kx), d(Mx), o(Mx), d(Kz), o(Kz), d(Mz), o(Mz), rp, ci, v)
    A = sp.csr_matrix((v[:got], ci[:got], rp.astype(np.int32)), shape=(n, n))
    A.has_sorted_indices = True
    return A


def q1_27pt_graded(e: int, aspect: float = 100.0, seed: int = 0, permute: bool = True,
                   growth: float = 1.1) -> sp.csr_matrix:
    """Trilinear (Q1) finite-element Laplacian on e^3 interior nodes of the unit cube.

    Uniform spacing in x and y; in z the element heights grow geometrically (ratio `growth` per
    cell) from the z = 0 wall, starting at h_u / aspect, until they reach the uniform spacing h_u. Dirichlet on all faces
    (boundary nodes eliminated). The Q1 stiffness matrix of a tensor-product mesh is the sum of
    Kronecker products of assembled 1D matrices: A = Mz(x)My(x)Kx + Mz(x)Ky(x)Mx + Kz(x)My(x)Mx
    (x fastest), up to 27 entries per row, nnz = (3e - 2)^3. With permute=True a seeded symmetric
    random permutation is applied and then reverse Cuthill-McKee.
    """
    from scipy.sparse.csgraph import reverse_cuthill_mckee

    hx = np.full(e + 1, 1.0 / (e + 1))
    hz = np.diff(_graded_coords(e, aspect, growth))
    Kx, Mx = _fe1d(hx)
    Kz, Mz = _fe1d(hz)
    A = _q1_assemble(Kx, Mx, Kz, Mz)
    if permute:
        A = _sym_permute(A, _rng(seed, _TAG_PERM).permutation(A.shape[0]))
        rcm = reverse_cuthill_mckee(A, symmetric_mode=True)
        A = _sym_permute(A, np.asarray(rcm))
    return A


def rhs_uniform(n: int, seed: int = 0) -> np.ndarray:
    """Right-hand side b ~ U[-1, 1]^n (float64)."""
    return _rng(seed, _TAG_RHS).uniform(-1.0, 1.0, n)


def edge_sizes(count: int, lo: int, hi: int, seed: int = 0) -> np.ndarray:
    """Cube edges e_s ~ U{lo..hi} (inclusive) for batched / served systems."""
    return _rng(seed, _TAG_SIZES).integers(lo, hi + 1, size=count)
