"""Ruge-Stuben hierarchy built on the host, fed identically to the CUDA path and the oracle.

Per level l: A_l (CSR), P_l (prolongation from level l+1 to l), R_l = P_l^T, and on requested
levels the ILU(0) factors A_l ~ (I + L_s) D_U (I + U_s). The coarsest level carries its dense
inverse when it has at most `coarse_max` rows. Coarse operators are the Galerkin products
A_{l+1} = R_l A_l P_l (Sec. 5, eq. A_k).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libnsw_setup.so")
_SRC = os.path.join(_HERE, "csrc", "amg_setup.cpp")
_lib = None


def build_setup_library(force: bool = False) -> str:
    """Compile the host setup library (g++, OpenMP) next to this file."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O3", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_setup_library())
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        lib.nsw_amg_coarsen.argtypes = [ctypes.c_int, i32p, i32p, f64p, ctypes.c_double, ctypes.c_uint64, i32p]
        lib.nsw_amg_coarsen.restype = ctypes.c_int
        lib.nsw_amg_interp.argtypes = [ctypes.c_int, i32p, i32p, f64p, ctypes.c_double, i32p, i32p, i32p, f64p]
        lib.nsw_amg_interp.restype = ctypes.c_int64
        lib.nsw_ilu0.argtypes = [ctypes.c_int, i32p, i32p, f64p, i32p, i32p, f64p, i32p, i32p, f64p, f64p]
        lib.nsw_ilu0.restype = ctypes.c_int
        i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
        lib.nsw_spgemm_count.argtypes = [ctypes.c_int, ctypes.c_int, i32p, i32p, i32p, i32p, i64p]
        lib.nsw_spgemm_count.restype = ctypes.c_int64
        lib.nsw_spgemm_fill.argtypes = [ctypes.c_int, ctypes.c_int, i32p, i32p, f64p, i32p, i32p, f64p, i64p, i32p, f64p]
        lib.nsw_spgemm_fill.restype = None
        lib.nsw_set_strength_mode.argtypes = [ctypes.c_int]
        lib.nsw_set_strength_mode.restype = None
        lib.nsw_ilut.argtypes = [ctypes.c_int, i32p, i32p, f64p, ctypes.c_double, ctypes.c_int, i32p, i32p, f64p, i32p,
                                 i32p, f64p, i64p]
        lib.nsw_ilut.restype = ctypes.c_int
        lib.nsw_ruiz.argtypes = [ctypes.c_int, i32p, i32p, f64p, ctypes.c_double, ctypes.c_int, f64p, f64p]
        lib.nsw_ruiz.restype = ctypes.c_int
        lib.nsw_ruiz_dep.argtypes = [ctypes.c_int, i32p, i32p, f64p, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                     f64p, f64p, f64p]
        lib.nsw_ruiz_dep.restype = ctypes.c_int
        lib.nsw_q1_assemble.argtypes = [ctypes.c_int] + [f64p] * 8 + [i64p, i32p, f64p]
        lib.nsw_q1_assemble.restype = ctypes.c_int64
        lib.nsw_sym_permute.argtypes = [ctypes.c_int, i32p, i32p, f64p, i32p, i32p, i32p, f64p]
        lib.nsw_sym_permute.restype = None
        _lib = lib
    return _lib


def _csr(A) -> sp.csr_matrix:
    A = sp.csr_matrix(A)
    A.sum_duplicates()
    A.sort_indices()
    A.indices = A.indices.astype(np.int32, copy=False)
    A.indptr = A.indptr.astype(np.int32, copy=False)
    return A


@dataclass
class Level:
    A: sp.csr_matrix
    P: sp.csr_matrix | None = None  # n_l x n_{l+1}
    R: sp.csr_matrix | None = None  # n_{l+1} x n_l
    ilu_L: sp.csr_matrix | None = None  # strictly lower L_s
    ilu_U: sp.csr_matrix | None = None  # ILU(0): strictly upper U_s (rows scaled by 1/u_ii); ILUT: U with diagonal
    ilu_dinv: np.ndarray | None = None  # ILU(0): 1/u_ii
    ilu_form: int = 0  # 0: ILU(0) in row-scaled LDU form; 1: ILUT with Ruiz scalings ilu_dr, ilu_dc
    ilu_dr: np.ndarray | None = None
    ilu_dc: np.ndarray | None = None

    @property
    def n(self) -> int:
        return self.A.shape[0]


@dataclass
class Hierarchy:
    levels: list[Level]
    coarse_inv: np.ndarray | None = None  # dense inverse of the coarsest A, row-major
    theta: float = 0.25
    seed: int = 0
    info: dict = field(default_factory=dict)

    @property
    def nlevels(self) -> int:
        return len(self.levels)

    def operator_complexity(self) -> float:
        return sum(l.A.nnz for l in self.levels) / self.levels[0].A.nnz


def spgemm(A: sp.csr_matrix, B: sp.csr_matrix) -> sp.csr_matrix:
    """C = A B with the OpenMP setup library (rows sorted; result independent of thread count)."""
    lib = _load()
    A, B = _csr(A), _csr(B)
    m, k = A.shape
    if B.shape[0] != k:
        raise ValueError("shape mismatch")
    n = B.shape[1]
    crp = np.empty(m + 1, np.int64)
    nnz = lib.nsw_spgemm_count(m, n, A.indptr, A.indices, B.indptr, B.indices, crp)
    if nnz >= 2 ** 31:
        raise ValueError("product too large for int32 indices")
    cci = np.empty(max(nnz, 1), np.int32)
    cv = np.empty(max(nnz, 1), np.float64)
    lib.nsw_spgemm_fill(m, n, A.indptr, A.indices, A.data, B.indptr, B.indices, B.data, crp, cci, cv)
    C = sp.csr_matrix((cv[:nnz], cci[:nnz], crp.astype(np.int32)), shape=(m, n))
    C.has_sorted_indices = True
    return C


def coarsen(A: sp.csr_matrix, theta: float, seed: int) -> tuple[np.ndarray, int]:
    lib = _load()
    n = A.shape[0]
    cf = np.empty(n, np.int32)
    nc = lib.nsw_amg_coarsen(n, A.indptr, A.indices, A.data, theta, seed & 0xFFFFFFFFFFFFFFFF, cf)
    if nc < 0:
        raise ValueError("coarsening failed")
    return cf, nc


def interpolation(A: sp.csr_matrix, theta: float, cf: np.ndarray, nc: int) -> sp.csr_matrix:
    lib = _load()
    n = A.shape[0]
    prp = np.empty(n + 1, np.int32)
    pci = np.empty(A.nnz + n, np.int32)
    pv = np.empty(A.nnz + n, np.float64)
    nnz = lib.nsw_amg_interp(n, A.indptr, A.indices, A.data, theta, cf, prp, pci, pv)
    if nnz < 0:
        raise ValueError("interpolation failed: an F-row without strong C-neighbours or zero denominator")
    return sp.csr_matrix((pv[:nnz].copy(), pci[:nnz].copy(), prp), shape=(n, nc))


def ilu0(A: sp.csr_matrix):
    """ILU(0) on pattern(A): returns (L_s, U_s, dU_inv) with A ~ (I + L_s) diag(1/dU_inv) (I + U_s)."""
    lib = _load()
    n = A.shape[0]
    rows = np.repeat(np.arange(n), np.diff(A.indptr))
    nl = int(np.count_nonzero(A.indices < rows))
    nu = int(np.count_nonzero(A.indices > rows))
    lrp, lci, lv = np.empty(n + 1, np.int32), np.empty(max(nl, 1), np.int32), np.empty(max(nl, 1), np.float64)
    urp, uci, uv = np.empty(n + 1, np.int32), np.empty(max(nu, 1), np.int32), np.empty(max(nu, 1), np.float64)
    dinv = np.empty(n, np.float64)
    rc = lib.nsw_ilu0(n, A.indptr, A.indices, A.data, lrp, lci, lv, urp, uci, uv, dinv)
    if rc != 0:
        raise ValueError(f"ILU(0) zero pivot in row {-rc - 1}")
    L = sp.csr_matrix((lv[:nl], lci[:nl], lrp), shape=(n, n))
    U = sp.csr_matrix((uv[:nu], uci[:nu], urp), shape=(n, n))
    return _csr(L), _csr(U), dinv


def dep_bound(n: int, nu: float) -> float:
    """The bound of the paper's theorem on a scaled upper triangular U = I + U_s (eq. depU):
    dep(U) <= sqrt((2 sqrt(n) + nu) nu), nu = ||U_s||_F."""
    return float(np.sqrt((2.0 * np.sqrt(n) + nu) * nu))


def ruiz_dep(U: sp.csr_matrix, tol: float = 1e-3, maxit: int = 50, dep_factor: float = 1.0):
    """Ruiz scaling of the upper triangular U with the dep(U)-based early termination (Sec. 5.3):
    stop when Henrici's dep of the scaled factor is below dep_factor times the eq. depU bound,
    when it stops decreasing (keeping the previous scaling), or as plain Ruiz. Returns
    (dr, dc, info) with info = dict(dep, nu, bound, dep_unscaled, reason, sweeps)."""
    U = _csr(U)
    n = U.shape[0]
    dr, dc, info = np.ones(n), np.ones(n), np.zeros(7)
    _load().nsw_ruiz_dep(n, U.indptr, U.indices, U.data, float(tol), int(maxit), float(dep_factor), dr, dc, info)
    reasons = {0: "tol", 1: "dep_below_bound", 2: "dep_increased", 3: "maxit"}
    return dr, dc, {"dep": info[0], "nu": info[1], "bound": info[2], "dep_unscaled": info[3],
                    "reason": reasons[int(info[4])], "sweeps": int(info[5])}


def ilut(A: sp.csr_matrix, droptol: float = 1e-2, lfil: int = 5, ruiz: bool = True, ruiz_tol: float = 1e-3,
         ruiz_maxit: int = 50, ruiz_stop: str = "tol", dep_factor: float = 1.0):
    """ILUT(droptol, lfil) factors A ~ (I + L_s) U and Ruiz scalings D_r, D_c of U
    (Algorithm 2). Returns (L_s, U with diagonal, dr, dc); dr = dc = 1 without Ruiz.
    ruiz_stop="tol" runs Ruiz until the row/column maxima are within ruiz_tol of one;
    ruiz_stop="dep" adds the dep(U)-based early termination (ruiz_dep)."""
    lib = _load()
    A = _csr(A)
    n = A.shape[0]
    lrp, urp = np.empty(n + 1, np.int32), np.empty(n + 1, np.int32)
    lci, lv = np.empty(max(n * lfil, 1), np.int32), np.empty(max(n * lfil, 1), np.float64)
    uci, uv = np.empty(n * (lfil + 1), np.int32), np.empty(n * (lfil + 1), np.float64)
    counts = np.zeros(2, np.int64)
    rc = lib.nsw_ilut(n, A.indptr, A.indices, A.data, float(droptol), int(lfil), lrp, lci, lv, urp, uci, uv, counts)
    if rc != 0:
        raise ValueError(f"ILUT zero pivot in row {-rc - 1}")
    nl, nu = int(counts[0]), int(counts[1])
    L = _csr(sp.csr_matrix((lv[:nl].copy(), lci[:nl].copy(), lrp), shape=(n, n)))
    U = _csr(sp.csr_matrix((uv[:nu].copy(), uci[:nu].copy(), urp), shape=(n, n)))
    dr, dc = np.ones(n), np.ones(n)
    if ruiz and ruiz_stop == "dep":
        dr, dc, _ = ruiz_dep(U, ruiz_tol, ruiz_maxit, dep_factor)
    elif ruiz:
        lib.nsw_ruiz(n, U.indptr, U.indices, U.data, float(ruiz_tol), int(ruiz_maxit), dr, dc)
    return L, U, dr, dc


def block_diagonal(A: sp.csr_matrix, ranks: int) -> sp.csr_matrix:
    """A with every coupling between different row blocks dropped; the blocks are `ranks`
    contiguous ranges of ceil(n / ranks) rows (columns split the same way): the local matrices
    of `ranks` MPI ranks that each own one range."""
    A = _csr(A)
    if ranks <= 1:
        return A
    n = A.shape[0]
    size = -(-n // ranks)
    rows = np.repeat(np.arange(n), np.diff(A.indptr))
    keep = (rows // size) == (A.indices // size)
    B = sp.csr_matrix((A.data[keep], A.indices[keep], np.concatenate([[0], np.cumsum(
        np.bincount(rows[keep], minlength=n))])), shape=A.shape)
    return _csr(B)


def build_hierarchy(A, theta: float = 0.25, max_levels: int = 25, coarse_max: int = 512, seed: int = 0,
                    ilu_levels=(0,), min_coarse: int = 1, direct_max: int = 512, strength: str = "abs",
                    ilu: str = "ilu0", droptol: float = 1e-2, lfil: int = 5, ruiz_stop: str = "tol",
                    ranks: int = 1) -> Hierarchy:
    """Build the Ruge-Stuben hierarchy of A (strength theta, PMIS, BAMG-direct, Galerkin RAP).

    Coarsening stops when a level has at most `coarse_max` rows, when `max_levels` levels exist,
    or when a coarsening step keeps more than 90% of the points. ILU(0) factors are attached to
    the levels listed in `ilu_levels` (None for every non-coarsest level); ilu="ilut" attaches
    ILUT(droptol, lfil) factors with Ruiz scalings of U instead (Algorithm 2; ruiz_stop="dep" for the
    dep(U)-based early termination of Sec. 5.3). The coarsest level
    gets a dense inverse when it has at most `direct_max` rows. ranks > 1: the ILU factors are
    those of the block diagonal over `ranks` contiguous row blocks (block_diagonal), as each rank
    of a hybrid smoother factors its local matrix (Sec. 5.2); the operators stay whole.
    strength="abs" compares |a_ij|
    (Sec. 5.1 as printed); strength="neg" compares -a_ij (classical Ruge-Stuben, for matrices
    with positive off-diagonal entries such as Q1 stiffness on high-aspect elements).
    """
    A = _csr(A)
    _load().nsw_set_strength_mode(1 if strength == "neg" else 0)
    levels = [Level(A=A)]
    while len(levels) < max_levels and levels[-1].n > coarse_max:
        Al = levels[-1].A
        cf, nc = coarsen(Al, theta, seed + 7919 * len(levels))
        if nc < min_coarse or nc >= 0.9 * Al.shape[0] or nc == 0:
            break
        P = _csr(interpolation(Al, theta, cf, nc))
        R = _csr(P.T)
        Ac = _csr(spgemm(R, spgemm(Al, P)))
        levels[-1].P, levels[-1].R = P, R
        levels.append(Level(A=Ac))
    want = range(len(levels) - 1) if ilu_levels is None else ilu_levels
    for l in want:
        if 0 <= l < len(levels) - 1:
            Al = block_diagonal(levels[l].A, ranks)
            if ilu == "ilut":
                lev = levels[l]
                lev.ilu_L, lev.ilu_U, lev.ilu_dr, lev.ilu_dc = ilut(Al, droptol, lfil, ruiz_stop=ruiz_stop)
                lev.ilu_form = 1
            else:
                levels[l].ilu_L, levels[l].ilu_U, levels[l].ilu_dinv = ilu0(Al)
    H = Hierarchy(levels=levels, theta=theta, seed=seed)
    if levels[-1].n <= direct_max:
        H.coarse_inv = np.ascontiguousarray(np.linalg.inv(levels[-1].A.toarray()))
    H.info = {"n": [l.n for l in levels], "nnz": [int(l.A.nnz) for l in levels],
              "operator_complexity": H.operator_complexity()}
    return H
