"""FP64 restatement of the Ruge-Stuben setup (Sec. 5.1) that the GPU setup computes.

TEST INFRASTRUCTURE ONLY (see the package header): nothing on the product path imports it.

  strength        S_i = { j != i : |a_ij| >= theta max_{k != i} |a_ik| }  (Sec. 5.1; "neg" mode
                  compares -a_ij, the classical sign-aware form)
  pmis_uniforms   the PMIS random numbers: one SplitMix64 step (Steele, Lea & Flood, OOPSLA 2014;
                  Vigna's public-domain reference) per point, from the state seed ^ (C * (i + 1))
  pmis            PMIS coarsening (Sec. 5.1; De Sterck, Yang & Heys 2006): weights
                  lambda_i = |S^T_i| + u_i, rounds of local maxima over S_i u S^T_i among the
                  undecided points, undecided points that strongly depend on a new C-point
                  become F; then F-points left without a strong C-neighbour are promoted to C in
                  index order (a reading: the paper does not say what happens to them)
  bamg_direct     BAMG-direct interpolation with f = 1, closed form of eq. (bamgdir):
                  w_ij = -(a_ij + beta_i / n_{C_i^s}) / (a_ii + sum_{k weak} a_ik),
                  beta_i = sum of the strong F-neighbour couplings
  mm_ext          MM-ext interpolation W = -[(D_FF + D_gamma)^-1 (A^s_FF + D_beta)] [D_beta^-1 A^s_FC]
  galerkin        R = P^T, A_c = R (A P)  (Sec. 5, eq. A_k)
  coarse_inverse  dense inverse of the coarsest operator
  ilu0_factors    ILU(0) by fixed-point sweeps (kernels.ilu0_fixed_point) in the row-scaled LDU
                  form the solve phase consumes: A ~ (I + L_s) diag(1/dinv) (I + U_s)
  setup           the level loop: coarsen while n > coarse_max, stop when a step keeps more than
                  90% of the points; level l is coarsened with seed + 7919 (l + 1)

Integer decisions (strength flags, PMIS states) are taken in float64 like the library does.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .kernels import ilu0_fixed_point

MASK64 = (1 << 64) - 1
SPLITMIX_GAMMA = 0x9E3779B97F4A7C15
PMIS_STREAM = 0xA24BAED4963EE407


def splitmix64_next(state: int) -> tuple[int, int]:
    """One step of SplitMix64: advance the state by the golden gamma and mix it.
    Returns (new_state, output)."""
    state = (state + SPLITMIX_GAMMA) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return state, z ^ (z >> 31)


def pmis_uniforms(seed: int, n: int) -> np.ndarray:
    """u_i in [0, 1): the top 53 bits of one SplitMix64 output from state seed ^ (C (i + 1))."""
    u = np.empty(n)
    for i in range(n):
        _, out = splitmix64_next((seed ^ ((PMIS_STREAM * (i + 1)) & MASK64)) & MASK64)
        u[i] = (out >> 11) * 2.0 ** -53
    return u


def _rows(A: sp.csr_matrix) -> np.ndarray:
    return np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))


def strength(A: sp.csr_matrix, theta: float, mode: str = "abs") -> np.ndarray:
    """Strong-connection flag for every stored entry of A (CSR order). An off-diagonal entry is
    strong when its measure (|a_ij|, or -a_ij in "neg" mode) is nonzero and at least theta times
    the row's largest off-diagonal measure; rows whose largest measure is <= 0 have none."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    s = np.zeros(A.nnz, dtype=bool)
    for i in range(n):
        lo, hi = A.indptr[i], A.indptr[i + 1]
        cols, vals = A.indices[lo:hi], A.data[lo:hi]
        off = cols != i
        meas = np.abs(vals) if mode == "abs" else -vals
        if not off.any():
            continue
        mx = float(np.max(meas[off]))
        if mx <= 0.0:
            continue
        thr = theta * mx
        s[lo:hi] = off & (vals != 0.0) & (meas >= thr)
    return s


def strength_matrix(A: sp.csr_matrix, s: np.ndarray) -> sp.csr_matrix:
    """S as a 0/1 CSR matrix: S[i, j] = 1 when j is in S_i (i strongly depends on j)."""
    A = sp.csr_matrix(A)
    S = sp.csr_matrix((s.astype(np.float64), A.indices.copy(), A.indptr.copy()), shape=A.shape)
    S.eliminate_zeros()
    return S


def pmis(A: sp.csr_matrix, s: np.ndarray, seed: int, promote: bool = True):
    """PMIS C/F splitting. Returns (cf, nc): cf[i] = coarse index of a C-point, -1 for F."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    S = strength_matrix(A, s)
    ST = sp.csr_matrix(S.T)
    infl = np.diff(ST.indptr)  # |S^T_i|: how many points strongly depend on i
    lam = infl + pmis_uniforms(seed, n)
    # "j beats i" when (lambda_j, j) > (lambda_i, i) lexicographically
    order = np.lexsort((np.arange(n), lam))
    rank = np.empty(n, dtype=np.int64)
    rank[order] = np.arange(n)
    UNDEC, C, F = 0, 1, 2
    st = np.zeros(n, dtype=np.int8)
    st[infl == 0] = F  # influences no point: never an interpolation point
    nbr = sp.csr_matrix(((S + ST) > 0).astype(np.int8))
    for _ in range(10 * n + 10):
        und = st == UNDEC
        if not und.any():
            break
        new_c = np.zeros(n, dtype=bool)
        for i in np.flatnonzero(und):
            js = nbr.indices[nbr.indptr[i]:nbr.indptr[i + 1]]
            js = js[(js != i) & (st[js] == UNDEC)]
            new_c[i] = not np.any(rank[js] > rank[i])
        st[new_c] = C
        for i in np.flatnonzero(st == UNDEC):
            js = S.indices[S.indptr[i]:S.indptr[i + 1]]
            if np.any(new_c[js]):
                st[i] = F
    if promote:
        for i in range(n):
            if st[i] == F:
                js = S.indices[S.indptr[i]:S.indptr[i + 1]]
                if not np.any(st[js] == C):
                    st[i] = C
    cf = np.full(n, -1, dtype=np.int64)
    cpts = np.flatnonzero(st == C)
    cf[cpts] = np.arange(cpts.size)
    return cf, int(cpts.size)


def bamg_direct(A: sp.csr_matrix, s: np.ndarray, cf: np.ndarray, nc: int) -> sp.csr_matrix:
    """Prolongation P (n x nc): unit rows at C-points; at an F-point i the closed-form BAMG-direct
    weights over its strong C-neighbours C_i^s, with weak couplings lumped into the diagonal and
    the strong F-couplings beta_i spread evenly over C_i^s."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    rows, cols, vals = [], [], []
    for i in range(n):
        if cf[i] >= 0:
            rows.append(i), cols.append(cf[i]), vals.append(1.0)
            continue
        lo, hi = A.indptr[i], A.indptr[i + 1]
        aii = weak = beta = 0.0
        strong_c = []
        for p in range(lo, hi):
            j, a = A.indices[p], A.data[p]
            if j == i:
                aii += a
            elif not s[p]:
                weak += a
            elif cf[j] >= 0:
                strong_c.append(p)
            else:
                beta += a
        den = aii + weak
        if den == 0.0 or not strong_c:
            raise ValueError(f"interpolation undefined in row {i}")
        for p in strong_c:
            rows.append(i), cols.append(cf[A.indices[p]]), vals.append(-(A.data[p] + beta / len(strong_c)) / den)
    P = sp.csr_matrix((vals, (rows, cols)), shape=(n, nc))
    P.sort_indices()
    return P


def mm_ext(A: sp.csr_matrix, s: np.ndarray, cf: np.ndarray, nc: int) -> sp.csr_matrix:
    """MM-ext interpolation (Sec. 5.1): with A = D + A^s + A^w split by the strength flags and the
    F/C blocks of the splitting,
        W = -[(D_FF + D_gamma)^-1 (A^s_FF + D_beta)] [D_beta^-1 A^s_FC],
        D_beta = diag(A^s_FC 1_C),  D_gamma = diag(A^w_FF 1_F + A^w_FC 1_C),
    and P = [W; I] in the original ordering. An F-point with beta = 0 (no strong C-neighbour)
    contributes no distance-two path (its row of D_beta^-1 A^s_FC is taken as zero)."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    rows = _rows(A)
    cols = A.indices
    off = rows != cols
    strong = s.astype(bool) & off
    weak = off & ~strong
    Fp = np.flatnonzero(cf < 0)
    fidx = np.full(n, -1)
    fidx[Fp] = np.arange(Fp.size)
    As = sp.csr_matrix((np.where(strong, A.data, 0.0), cols.copy(), A.indptr.copy()), shape=A.shape)
    Aw = sp.csr_matrix((np.where(weak, A.data, 0.0), cols.copy(), A.indptr.copy()), shape=A.shape)
    Cmask = cf >= 0
    As_FF = As[Fp][:, Fp]
    As_FC = As[Fp][:, np.flatnonzero(Cmask)]
    Aw_F = Aw[Fp]
    d_FF = A.diagonal()[Fp]
    beta = np.asarray(As_FC.sum(axis=1)).ravel()
    gamma = np.asarray(Aw_F.sum(axis=1)).ravel()  # A^w_FF 1_F + A^w_FC 1_C
    inv_beta = np.where(beta != 0.0, 1.0 / np.where(beta != 0.0, beta, 1.0), 0.0)
    M1 = sp.diags(1.0 / (d_FF + gamma)) @ (As_FF + sp.diags(beta))
    M2 = sp.diags(inv_beta) @ As_FC
    W = -sp.csr_matrix(M1 @ M2)
    W.sum_duplicates()
    P = sp.lil_matrix((n, nc))
    Wc = W.tocoo()
    P[Fp[Wc.row], Wc.col] = Wc.data
    P[np.flatnonzero(Cmask), cf[Cmask]] = 1.0
    P = sp.csr_matrix(P)
    P.sort_indices()
    return P


def galerkin(A: sp.csr_matrix, P: sp.csr_matrix):
    """R = P^T and the Galerkin coarse operator A_c = R (A P)."""
    R = sp.csr_matrix(P.T)
    R.sort_indices()
    Ac = sp.csr_matrix(R @ sp.csr_matrix(A @ P))
    Ac.sort_indices()
    return R, Ac


def coarse_inverse(A: sp.csr_matrix) -> np.ndarray:
    return np.linalg.inv(A.toarray())


def ilu0_factors(A: sp.csr_matrix, sweeps: int):
    """(L_s, U_s, dinv) with A ~ (I + L_s) diag(1/dinv) (I + U_s), from `sweeps` fixed-point
    sweeps: U_s = diag(U)^-1 (U - diag(U)), dinv = 1 / diag(U)."""
    Ls, U = ilu0_fixed_point(A, sweeps)
    d = U.diagonal()
    Us = sp.csr_matrix(sp.diags(1.0 / d) @ sp.triu(U, 1))
    Us.sort_indices()
    Ls = sp.csr_matrix(Ls)
    Ls.sort_indices()
    return Ls, Us, 1.0 / d


def setup(A: sp.csr_matrix, theta: float = 0.25, strength_mode: str = "abs", max_levels: int = 25,
          coarse_max: int = 512, direct_max: int = 512, seed: int = 0, ilu_levels=(0,), ilu_sweeps: int = 3,
          interp: str = "bamg"):
    """The whole hierarchy: a list of per-level dicts (A, s, cf, P, R, and ILU factors on the
    requested non-coarsest levels) and the dense coarse inverse (None above direct_max)."""
    levels = [{"A": sp.csr_matrix(A)}]
    while len(levels) < max_levels and levels[-1]["A"].shape[0] > coarse_max:
        lev = levels[-1]
        Al = lev["A"]
        s = strength(Al, theta, strength_mode)
        cf, nc = pmis(Al, s, seed + 7919 * len(levels))
        if nc == 0 or nc >= 0.9 * Al.shape[0]:
            break
        P = bamg_direct(Al, s, cf, nc) if interp == "bamg" else mm_ext(Al, s, cf, nc)
        R, Ac = galerkin(Al, P)
        lev.update(s=s, cf=cf, P=P, R=R)
        levels.append({"A": Ac})
    for l in ilu_levels:
        if 0 <= l < len(levels) - 1:
            levels[l]["ilu"] = ilu0_factors(levels[l]["A"], ilu_sweeps)
    Ac = levels[-1]["A"]
    cinv = coarse_inverse(Ac) if Ac.shape[0] <= direct_max else None
    return levels, cinv
