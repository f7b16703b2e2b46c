"""Per-kernel FP64 references (plain loops / library primitives, no blocking or fusion).

Splitting convention (Sec. 5.2): A = L + D + U with L strictly lower, D diagonal and U strictly
upper. ILU convention (Sec. 5.3.2): A ~ (I + L_s) D_U (I + U_s).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

POLY_GS = 0
JACOBI_L1 = 1
ILU0 = 2
HYBRID_ILU0 = 3


@dataclass
class SmootherParams:
    """Solve-phase parameters shared by the oracle V-cycle (mirrors the library's parameters).

    smoother: POLY_GS, JACOBI_L1, ILU0 (ILU on every level that has factors) or HYBRID_ILU0
    (ILU on the finest level only, polynomial Gauss-Seidel below; Sec. 6.2).
    neumann_terms: k terms of the truncated series for (D+L)^-1 (k = 1 is Jacobi).
    ilu_terms_L / ilu_terms_U: terms of the series for (I+L_s)^-1 and (I+U_s)^-1.
    ranks: the rows of every level are dealt to this many contiguous blocks (MPI ranks in the
    paper's runs); the polynomial Gauss-Seidel triangular parts keep only the couplings inside a
    block (hybrid block-Jacobi: Gauss-Seidel within a rank, Jacobi across ranks), while every
    residual uses the whole level operator. ILU factors come with the hierarchy (those of the
    block diagonal when it was built for ranks > 1).
    pre_sweeps / post_sweeps: sweeps per level (forward before, backward after the coarse
    correction for polynomial Gauss-Seidel).
    coarse_sweeps: sweeps on the coarsest level when it has no dense direct solve.
    mode: "definition" (truncated power sums) or "direct" (substitution, the limit of the series).
    """
    smoother: int = POLY_GS
    neumann_terms: int = 2
    ilu_terms_L: int = 3
    ilu_terms_U: int = 3
    pre_sweeps: int = 1
    post_sweeps: int = 1
    coarse_sweeps: int = 4
    mode: str = "definition"
    ranks: int = 1  # hybrid block-Jacobi across this many row blocks per level (Sec. 5.2, Sec. 6)


# ---------------------------------------------------------------------------------------------
# Basic products
# ---------------------------------------------------------------------------------------------

def spmv(A: sp.csr_matrix, x: np.ndarray) -> np.ndarray:
    """y = A x (the matrix-vector product every smoother here is built from, Sec. 1)."""
    return A @ x


def residual(A, b, x):
    """r = b - A x (eq. relres numerator)."""
    return b - A @ x


def split_ldu(A: sp.csr_matrix):
    """A = L + D + U: strictly lower, diagonal (as a vector), strictly upper (Sec. 5.2).
    The split of a given matrix object is computed once and remembered on that object."""
    cached = getattr(A, "_oracle_ldu", None)
    if cached is None:
        A2 = sp.csr_matrix(A)
        cached = (sp.tril(A2, k=-1, format="csr"), A2.diagonal().copy(), sp.triu(A2, k=1, format="csr"))
        try:
            A._oracle_ldu = cached
        except AttributeError:
            pass
    return cached


def row_blocks(n: int, ranks: int) -> np.ndarray:
    """Offsets of `ranks` contiguous row blocks of ceil(n / ranks) rows (the last may be short or
    empty): block q holds rows off[q] .. off[q+1]-1."""
    if ranks < 1:
        raise ValueError("ranks must be >= 1")
    size = -(-n // ranks)
    return np.minimum(np.arange(ranks + 1, dtype=np.int64) * size, n)


def local_block(A: sp.csr_matrix, ranks: int) -> sp.csr_matrix:
    """The block-diagonal part of A over the row blocks of row_blocks(n, ranks) (the same split of
    the columns): a_ij kept when rows i and j lie in the same block, the local matrix each rank
    relaxes with in a hybrid smoother (Sec. 5.2). ranks = 1 returns A itself."""
    if ranks == 1:
        return A
    cache = getattr(A, "_oracle_blocks", None)
    if cache is None:
        cache = {}
        try:
            A._oracle_blocks = cache
        except AttributeError:
            pass
    if ranks not in cache:
        C = sp.coo_matrix(A)
        off = row_blocks(A.shape[0], ranks)
        bi = np.searchsorted(off, C.row, side="right")
        bj = np.searchsorted(off, C.col, side="right")
        keep = bi == bj
        cache[ranks] = sp.csr_matrix((C.data[keep], (C.row[keep], C.col[keep])), shape=A.shape)
    return cache[ranks]


def l1_diagonal(A: sp.csr_matrix) -> np.ndarray:
    """d_ii = sum_j |a_ij|, the pointwise l1-Jacobi diagonal (Sec. 6.1 comparison smoother)."""
    cached = getattr(A, "_oracle_l1", None)
    if cached is None:
        cached = np.asarray(abs(sp.csr_matrix(A)).sum(axis=1)).ravel()
        try:
            A._oracle_l1 = cached
        except AttributeError:
            pass
    return cached


# ---------------------------------------------------------------------------------------------
# Smoother sweeps. Each returns the updated x; b and x are not modified.
# ---------------------------------------------------------------------------------------------

def poly_gs_sweep(A, b, x, terms: int, backward: bool = False, mode: str = "definition", ranks: int = 1):
    """One polynomial Gauss-Seidel sweep (Sec. 5.2, eqs. polynomial / jr-initial-guess / jr).

    x <- x + M^-1 r with r = b - A x and M = D + L (forward) or D + U (backward).
    definition: M^-1 is replaced by the truncated Neumann series
        sum_{j=0}^{terms-1} (-D^-1 T)^j D^-1,  T = L (forward) or U (backward),
    evaluated as explicit terms t_0 = D^-1 r, t_{j+1} = -D^-1 (T t_j), g = sum_j t_j.
    direct: g = M^-1 r by forward (or backward) substitution, the classical GS sweep (eq. one-stage).
    ranks > 1 (hybrid block-Jacobi, Sec. 5.2): L and U are those of local_block(A, ranks), the
    couplings inside each rank's block; r still uses the whole A.
    """
    L, d, U = split_ldu(local_block(A, ranks))
    T = U if backward else L
    r = residual(A, b, x)
    if mode == "direct":
        M = sp.csr_matrix(T + sp.diags(d))
        g = spla.spsolve_triangular(M, r, lower=not backward)
    else:
        t = r / d
        g = t.copy()
        for _ in range(terms - 1):
            t = -(T @ t) / d
            g = g + t
    return x + g


def ilu0_sweep(Ls, Us, dinv, A, b, x, terms_L: int, terms_U: int, mode: str = "definition"):
    """One ILU(0) smoother sweep with Neumann-series triangular solves (Sec. 5.3.2, eq. Neumann;
    Algorithm 2 with row scaling in place of Ruiz scaling, as its footnote allows).

    x <- x + (I + U_s)^-1 D_U^-1 (I + L_s)^-1 r, r = b - A x.
    definition: (I + L_s)^-1 ~ sum_{j<terms_L} (-L_s)^j and (I + U_s)^-1 ~ sum_{j<terms_U} (-U_s)^j,
    evaluated term by term. direct: both triangular systems by substitution.
    """
    r = residual(A, b, x)
    n = r.size
    if mode == "direct":
        I = sp.identity(n, format="csr")
        y = spla.spsolve_triangular(sp.csr_matrix(I + Ls), r, lower=True, unit_diagonal=True)
        f = dinv * y
        v = spla.spsolve_triangular(sp.csr_matrix(I + Us), f, lower=False, unit_diagonal=True)
    else:
        t = r.copy()
        y = t.copy()
        for _ in range(terms_L - 1):
            t = -(Ls @ t)
            y = y + t
        f = dinv * y
        t = f.copy()
        v = t.copy()
        for _ in range(terms_U - 1):
            t = -(Us @ t)
            v = v + t
    return x + v


def ilut_sweep(Ls, U, dr, dc, A, b, x, terms_L: int, terms_U: int, mode: str = "definition"):
    """One ILUT smoother sweep with Jacobi triangular iterations and Ruiz scaling (Algorithm 2),
    applied to the residual equation: x <- x + v with r = b - A x and
      y^(k) = y^(k-1) + (r - L y^(k-1)),  L = I + L_s, y^(0) = 0, k = 1..terms_L;
      U~ = D_r U D_c, y~ = D_r y, D = diag(U~)^-1;
      v^(k) = v^(k-1) + D (y~ - U~ v^(k-1)), v^(0) = 0, k = 1..terms_U;  v = D_c v.
    (U v = y is equivalent to U~ (D_c^-1 v) = D_r y, which fixes where D_r and D_c act.)
    direct: y = L^-1 r and v = U^-1 y by substitution (the limit of both iterations)."""
    r = residual(A, b, x)
    n = r.size
    I = sp.identity(n, format="csr")
    Lfull = sp.csr_matrix(I + Ls)
    if mode == "direct":
        y = spla.spsolve_triangular(Lfull, r, lower=True, unit_diagonal=True)
        v = spla.spsolve_triangular(sp.csr_matrix(U), y, lower=False)
        return x + v
    y = np.zeros(n)
    for _ in range(terms_L):
        y = y + (r - Lfull @ y)
    Ut = sp.csr_matrix(sp.diags(dr) @ U @ sp.diags(dc))
    yt = dr * y
    Dinv = 1.0 / Ut.diagonal()
    v = np.zeros(n)
    for _ in range(terms_U):
        v = v + Dinv * (yt - Ut @ v)
    return x + dc * v


def l1_jacobi_sweep(A, b, x):
    """x <- x + D_l1^-1 (b - A x) (Sec. 5.3.1, Jacobi in non-compact form, with l1 diagonal)."""
    return x + residual(A, b, x) / l1_diagonal(A)


def restrict(R, r):
    """b_{l+1} = R_l r_l with R = P^T (Sec. 5, Galerkin formulation)."""
    return R @ r


def prolong(P, x, e):
    """x_l <- x_l + P_l e_{l+1} (Sec. 5)."""
    return x + P @ e


def coarse_direct(Ac, b):
    """Direct coarse solve on the coarsest level (Sec. 5: 'often a direct solver'):
    dense LU with partial pivoting (LAPACK gesv via numpy)."""
    return np.linalg.solve(Ac.toarray() if sp.issparse(Ac) else Ac, b)


# ---------------------------------------------------------------------------------------------
# One-reduce Arnoldi step pieces (Algorithm 1, steps 6-12)
# ---------------------------------------------------------------------------------------------

def gram(V: np.ndarray, vt: np.ndarray, w: np.ndarray):
    """The single global reduction of step i (Algorithm 1 step 6, eq. matvec):
    a = [V_i, vt]^T vt and s = [V_i, vt]^T w, where V_i holds the i normalised columns
    (shape n x i) and vt is the not-yet-normalised newest vector. Plain dot products."""
    cols = [V[:, j] for j in range(V.shape[1])] + [vt]
    a = np.array([float(np.dot(c, vt)) for c in cols])
    s = np.array([float(np.dot(c, w)) for c in cols])
    return a, s


def update(V: np.ndarray, vt: np.ndarray, w: np.ndarray, beta: float, h: np.ndarray):
    """Lagged normalisation and projection (Algorithm 1 steps 8 and 12):
    v_i = vt / beta and the next unnormalised vector w / beta - [V_i, v_i] h."""
    v = vt / beta
    nxt = w / beta
    for j in range(V.shape[1]):
        nxt = nxt - h[j] * V[:, j]
    nxt = nxt - h[V.shape[1]] * v
    return v, nxt


def project(Lrows: np.ndarray, r: np.ndarray, T_mode: str = "trunc") -> np.ndarray:
    """Projection coefficients h = T r of Algorithm 1 step 11, with L the strictly lower
    triangular (i+1) x (i+1) matrix of basis inner products (eq. GS, eq. matvec):
      trunc: T = I - L, the truncated Neumann series (Sec. 3 corollary);
      exact: T = (I + L)^-1 by forward substitution (the ICWY MGS correction, Sec. 2)."""
    k = r.size
    if T_mode == "trunc":
        return r - Lrows[:k, :k] @ r
    if T_mode == "exact":
        h = np.zeros(k)
        for q in range(k):
            h[q] = r[q] - np.dot(Lrows[q, :q], h[:q])
        return h
    raise ValueError("T_mode must be 'trunc' or 'exact'")


def ilu0_fixed_point_sweep(A: sp.csr_matrix, Ls: sp.csr_matrix, U: sp.csr_matrix):
    """One Jacobi-style fixed-point sweep for the ILU(0) factors on pattern(A) (the fixed-point
    ILU the paper's conclusions propose for the setup), written with the sparse product
    M = L_s U restricted to the pattern:
      i > j:  l_ij = (a_ij - (M_ij - l_ij u_jj)) / u_jj      (sum over k < j only)
      i <= j: u_ij = a_ij - M_ij                               (sum over k < i)
    Returns the new (L_s, U) on the pattern of A."""
    A = sp.csr_matrix(A)
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    cols = A.indices
    M = sp.csr_matrix(Ls @ U)
    m = np.asarray(M[rows, cols]).ravel()
    l = np.asarray(Ls[rows, cols]).ravel()
    u = np.asarray(U[rows, cols]).ravel()
    ud = U.diagonal()
    lower = rows > cols
    new = np.where(lower, (A.data - (m - l * ud[cols])) / ud[cols], A.data - m)
    shape = A.shape
    Ln = sp.csr_matrix((np.where(lower, new, 0.0), (rows, cols)), shape=shape)
    Un = sp.csr_matrix((np.where(lower, 0.0, new), (rows, cols)), shape=shape)
    Ln.eliminate_zeros()
    Un.eliminate_zeros()
    return Ln, Un


def ilu0_fixed_point(A: sp.csr_matrix, sweeps: int):
    """`sweeps` fixed-point sweeps from l_ij = a_ij / a_jj (i > j), u_ij = a_ij (i <= j)."""
    A = sp.csr_matrix(A)
    d = A.diagonal()
    Ls = sp.csr_matrix(sp.tril(A, -1) @ sp.diags(1.0 / d))
    U = sp.csr_matrix(sp.triu(A, 0))
    for _ in range(sweeps):
        Ls, U = ilu0_fixed_point_sweep(A, Ls, U)
    return Ls, U
