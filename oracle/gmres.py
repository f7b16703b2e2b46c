"""GMRES references.

gmres_mgs       -- classical right-preconditioned MGS-GMRES(m) of Saad and Schultz (Sec. 1;
                   Sec. 4 cites it as the algorithm whose convergence the truncated variant
                   reproduces), flexible form (Z stored), Givens rotations, restarts from the
                   true residual.
gmres_onereduce -- a plain restatement of Algorithm 1 (one-reduce MGS-GMRES with lagged
                   normalisation) with right preconditioning and T = I - L ("trunc") or
                   T = (I + L)^-1 ("exact", forward substitution). Used to check the corollary of
                   Sec. 3 that the truncation leaves convergence unchanged.

Both stop when the implicit residual |g_{k+1}| <= rtol * ||b|| (eq. relres), then confirm with
the true residual b - A x and restart if it is not yet below the tolerance. The iteration count
is the total number of Arnoldi columns used over all cycles.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import kernels as K


@dataclass
class GmresResult:
    x: np.ndarray
    iters: int
    restarts: int
    converged: bool
    relres_true: float
    relres_implicit: float
    history: list = field(default_factory=list)  # implicit relative residual per column
    V: np.ndarray | None = None  # basis of the last cycle (n x (k+1)), for diagnostics
    Z: np.ndarray | None = None  # preconditioned directions of the last cycle (n x k)
    H: np.ndarray | None = None  # Hessenberg of the last cycle ((k+1) x k)
    L: np.ndarray | None = None  # one-reduce only: accumulated strictly lower L of the last cycle


def _givens(a: float, b: float):
    """Rotation (c, s) with [c s; -s c] [a; b] = [rho; 0]."""
    if b == 0.0:
        return 1.0, 0.0
    rho = np.hypot(a, b)
    return a / rho, b / rho


class _Givens:
    """Incremental QR of the Hessenberg matrix by Givens rotations; g holds the rotated rhs."""

    def __init__(self, m: int, beta0: float):
        self.c = np.zeros(m)
        self.s = np.zeros(m)
        self.R = np.zeros((m + 1, m))
        self.g = np.zeros(m + 1)
        self.g[0] = beta0

    def add_column(self, j: int, h: np.ndarray):
        """h has j+2 entries: column j of H including the subdiagonal h[j+1]."""
        h = h.copy()
        for k in range(j):
            t = self.c[k] * h[k] + self.s[k] * h[k + 1]
            h[k + 1] = -self.s[k] * h[k] + self.c[k] * h[k + 1]
            h[k] = t
        c, s = _givens(h[j], h[j + 1])
        self.c[j], self.s[j] = c, s
        h[j] = c * h[j] + s * h[j + 1]
        h[j + 1] = 0.0
        self.R[: j + 1, j] = h[: j + 1]
        self.g[j + 1] = -s * self.g[j]
        self.g[j] = c * self.g[j]
        return abs(self.g[j + 1])

    def solve(self, k: int) -> np.ndarray:
        """Back substitution R[:k,:k] y = g[:k] (the least-squares minimiser, Algorithm 1 end)."""
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (self.g[i] - np.dot(self.R[i, i + 1:k], y[i + 1:k])) / self.R[i, i]
        return y


def gmres_mgs(A, b, M=None, x0=None, m: int = 30, rtol: float = 1e-8, maxit: int = 1000) -> GmresResult:
    """Classical flexible MGS-GMRES(m), right preconditioned: A M^-1 u = b, x = M^-1 u."""
    M = M or (lambda v: v.copy())
    n = b.size
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return GmresResult(np.zeros(n), 0, 0, True, 0.0, 0.0)
    iters, restarts, hist = 0, -1, []
    relres_imp = np.inf
    V = Z = Hm = None
    while True:
        r = b - A @ x
        beta = float(np.linalg.norm(r))
        relres = beta / bnorm
        if relres <= rtol or iters >= maxit:
            return GmresResult(x, iters, max(restarts, 0), relres <= rtol, relres, min(relres_imp, relres), hist, V, Z, Hm)
        restarts += 1
        V = np.zeros((n, m + 1))
        Z = np.zeros((n, m))
        Hm = np.zeros((m + 1, m))
        V[:, 0] = r / beta
        G = _Givens(m, beta)
        k = 0
        for j in range(m):
            Z[:, j] = M(V[:, j])
            w = A @ Z[:, j]
            for i in range(j + 1):  # modified Gram-Schmidt: one dot and one axpy per column
                Hm[i, j] = float(np.dot(V[:, i], w))
                w = w - Hm[i, j] * V[:, i]
            Hm[j + 1, j] = float(np.linalg.norm(w))
            res = G.add_column(j, Hm[: j + 2, j])
            iters += 1
            k = j + 1
            relres_imp = res / bnorm
            hist.append(relres_imp)
            if Hm[j + 1, j] != 0.0:
                V[:, j + 1] = w / Hm[j + 1, j]
            if Hm[j + 1, j] == 0.0 or res <= rtol * bnorm or iters >= maxit:
                break
        y = G.solve(k)
        x = x + Z[:, :k] @ y
        V, Z, Hm = V[:, : k + 1], Z[:, :k], Hm[: k + 1, :k]


def inf_norm(A) -> float:
    """||A||_inf: the largest row sum of |a_ij|."""
    if sp.issparse(A):
        return float(abs(sp.csr_matrix(A)).sum(axis=1).max())
    return float(np.abs(np.asarray(A)).sum(axis=1).max())


def gmres_onereduce(A, b, M=None, x0=None, m: int = 30, rtol: float = 1e-8, maxit: int = 1000,
                    T_mode: str = "trunc", stop: str = "relres") -> GmresResult:
    """Algorithm 1 restated with right preconditioning (z = M^-1 vt) and the scalings the
    printed algorithm leaves implicit:

      step i (0-based): vt is the newest unnormalised vector, V the i normalised ones.
        z = M^-1 vt, w = A z                                       (step 5)
        a = [V, vt]^T vt, s = [V, vt]^T w                          (step 6, one reduction)
        beta = sqrt(a_i)                                           (step 7)
        v_i = vt / beta, z <- z / beta, w <- w / beta              (step 8, lagged normalisation)
        r_j = s_j / beta (j < i), r_i = s_i / beta^2               (step 9)
        L[i, :i] = a_{:i} / beta                                   (step 10, new row of L)
        h = T r with T = I - L (trunc) or (I + L)^-1 (exact)       (step 11)
        vt <- w - [V, v_i] h;  H[:i+1, i] = h                      (step 12)
        beta also closes column i-1: H[i, i-1] = beta, then Givens  (steps 13-14)
    After the last step the subdiagonal of the final column is ||vt||.
    Steps 6, 8/12 and 11 are the per-kernel references kernels.gram, kernels.update and
    kernels.project, so the Arnoldi-relation, orthogonality and L = tril(V^T V) checks of this
    solver also check those three functions.
    stop = "relres": ||b - A x|| / ||b|| <= rtol (eq. relres). stop = "nrbe": the norm-wise
    relative backward error beta(x) = ||b - A x|| / (||b|| + ||A||_inf ||x||) <= rtol (Sec. 3);
    inside a cycle the implicit residual is tested against rtol (||b|| + ||A||_inf ||x_0||) with
    x_0 the cycle's start, and the true residual at the cycle's end decides with beta(x).
    """
    if T_mode not in ("trunc", "exact"):
        raise ValueError("T_mode must be 'trunc' or 'exact'")
    if stop not in ("relres", "nrbe"):
        raise ValueError("stop must be 'relres' or 'nrbe'")
    anorm = inf_norm(A) if stop == "nrbe" else 0.0
    M = M or (lambda v: v.copy())
    n = b.size
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return GmresResult(np.zeros(n), 0, 0, True, 0.0, 0.0)
    iters, restarts, hist = 0, -1, []
    relres_imp = np.inf
    Vout = Zout = Hout = Lout = None
    while True:
        vt = b - A @ x
        rnorm = float(np.linalg.norm(vt))
        relres = rnorm / bnorm
        den = bnorm + anorm * float(np.linalg.norm(x))  # the cycle's tolerance scale (= ||b|| for relres)
        crit = rnorm / den
        if crit <= rtol or iters >= maxit:
            return GmresResult(x, iters, max(restarts, 0), crit <= rtol, relres, min(relres_imp, relres), hist,
                               Vout, Zout, Hout, Lout)
        restarts += 1
        V = np.zeros((n, m + 1))
        Z = np.zeros((n, m))
        Hm = np.zeros((m + 1, m))
        Lm = np.zeros((m + 1, m + 1))
        G = None
        k = 0
        done = False
        for i in range(m + 1):
            if i < m and iters + i < maxit:
                z = M(vt)
                w = A @ z
                a, s = K.gram(V[:, :i], vt, w)
                beta = float(np.sqrt(a[i]))
            else:  # no further column: only the lagged norm of the last vector is needed
                beta = float(np.linalg.norm(vt))
                z = w = None
            if i == 0:
                G = _Givens(m, beta)
            else:
                Hm[i, i - 1] = beta
                res = G.add_column(i - 1, Hm[: i + 1, i - 1])
                k = i
                relres_imp = res / bnorm
                hist.append(relres_imp)
                if beta == 0.0 or res <= rtol * den or iters + i >= maxit:
                    done = True
            if done or z is None:
                break
            if beta == 0.0:  # exact breakdown at the start: b - A x = 0 handled above
                break
            Z[:, i] = z / beta
            r = np.concatenate([s[:i] / beta, [s[i] / beta ** 2]])
            Lm[i, :i] = a[:i] / beta
            h = K.project(Lm, r, T_mode)
            Hm[: i + 1, i] = h
            V[:, i], vt = K.update(V[:, :i], vt, w, beta, h)
        iters += k
        if k == 0:
            return GmresResult(x, iters, restarts, False, relres, relres_imp, hist)
        y = G.solve(k)
        x = x + Z[:, :k] @ y
        if Hm[k, k - 1] != 0.0:
            V[:, k] = vt / Hm[k, k - 1]
        Vout, Zout, Hout = V[:, : k + 1].copy(), Z[:, :k].copy(), Hm[: k + 1, :k].copy()
        Lout = Lm[:k, :k].copy()

def sk_norm(L: np.ndarray) -> float:
    """||S_k||_2 with S_k = (I + U_k)^-1 U_k and U_k = L^T, the strictly upper part of V_k^T V_k
    (Sec. 3, after Paige, Rozloznik and Strakos): 0 for an orthonormal basis, 1 exactly when the
    columns of V_k are linearly dependent."""
    L = np.tril(np.asarray(L, dtype=np.float64), -1)
    k = L.shape[0]
    if k == 0:
        return 0.0
    U = L.T
    S = np.linalg.solve(np.eye(k) + U, U)
    return float(np.linalg.norm(S, 2))
