"""Row-sharded one-reduce GMRES with the hybrid block-Jacobi V-cycle over torch.distributed.

Test infrastructure (like the rest of this package): the data distribution and exchange pattern
of the paper's multi-rank runs, restated for CPU ranks with the gloo backend.

* Every level's rows are dealt to the ranks in contiguous blocks (kernels.row_blocks); rank q
  holds its rows of A_l, P_l, R_l and of every vector.
* A product with a distributed vector gathers the whole vector first (all_gather). The paper's
  ranks exchange only the halo entries their rows touch (Sec. 2, the matvec of eq. matvec); the
  gathered vector gives the same numbers.
* Smoothers are hybrid (Sec. 5.2): the residual uses the rank's rows of the whole operator after
  the gather, the Gauss-Seidel / ILU triangular parts only the couplings inside the rank's block,
  so a smoother's Neumann terms need no communication.
* Each Arnoldi step of Algorithm 1 needs ONE global reduction: the 2(i+1) inner products of
  step 6 (eq. matvec) are summed over the ranks by a single all_reduce. The Givens rotations,
  the triangular solve and the projection coefficients are replicated on every rank. A cycle
  adds the reductions of its true residual norm.

gmres_onereduce_sharded follows oracle.gmres.gmres_onereduce step for step (stop = "relres",
T = I - L or (I + L)^-1), so with one rank it gives the same result, and with P ranks it matches
gmres_onereduce with the P-block hybrid V-cycle up to the order of the cross-rank sums.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import torch
import torch.distributed as dist

from . import kernels as K
from .gmres import GmresResult, _Givens
from .vcycle import level_smoother


class Comm:
    """The collectives of one rank, with counters (all_reduce calls by purpose, all_gathers)."""

    def __init__(self):
        self.rank = dist.get_rank()
        self.size = dist.get_world_size()
        self.allreduce = {}
        self.allgather = 0

    def sum(self, v: np.ndarray, purpose: str) -> np.ndarray:
        t = torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).clone()
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        self.allreduce[purpose] = self.allreduce.get(purpose, 0) + 1
        return t.numpy()

    def gather(self, local: np.ndarray, off: np.ndarray) -> np.ndarray:
        """The whole vector from every rank's block (blocks of row_blocks sizes)."""
        width = int(np.max(np.diff(off))) if off.size > 1 else 0
        buf = torch.zeros(max(width, 1), dtype=torch.float64)
        buf[: local.size] = torch.from_numpy(local)
        parts = [torch.zeros_like(buf) for _ in range(self.size)]
        dist.all_gather(parts, buf)
        self.allgather += 1
        return np.concatenate([parts[q][: off[q + 1] - off[q]].numpy() for q in range(self.size)])


@dataclass
class _Level:
    n: int
    off: np.ndarray          # row blocks of this level
    A: sp.csr_matrix         # the rank's rows of A (all columns)
    Lb: sp.csr_matrix        # strictly lower part of the rank's diagonal block
    Ub: sp.csr_matrix        # strictly upper part of the rank's diagonal block
    d: np.ndarray            # the rank's diagonal entries
    l1: np.ndarray           # the rank's l1 row sums (whole rows)
    R: sp.csr_matrix | None  # the rank's rows of R (rows of the next level's block)
    P: sp.csr_matrix | None  # the rank's rows of P
    iL: sp.csr_matrix | None  # ILU factors restricted to the rank's block
    iU: sp.csr_matrix | None
    idinv: np.ndarray | None
    Afull: sp.csr_matrix     # whole operator (coarsest level: its dense solve on every rank)


class ShardedHierarchy:
    """The rank's share of a hierarchy (whole-matrix inputs, as every rank reads them)."""

    def __init__(self, H, comm: Comm, p: K.SmootherParams):
        self.comm, self.p, self.H = comm, p, H
        q = comm.rank
        P = comm.size
        self.levels = []
        for l, lev in enumerate(H.levels):
            n = lev.A.shape[0]
            off = K.row_blocks(n, P)
            r0, r1 = int(off[q]), int(off[q + 1])
            A = sp.csr_matrix(lev.A)
            Ab = sp.csr_matrix(A[r0:r1, r0:r1])
            nxt = None
            if l + 1 < len(H.levels):
                nc = H.levels[l + 1].A.shape[0]
                nxt = K.row_blocks(nc, P)
            ilu = getattr(lev, "ilu_L", None) is not None and getattr(lev, "ilu_form", 0) == 0
            self.levels.append(_Level(
                n=n, off=off, A=sp.csr_matrix(A[r0:r1]), Lb=sp.tril(Ab, k=-1, format="csr"),
                Ub=sp.triu(Ab, k=1, format="csr"), d=A.diagonal()[r0:r1].copy(),
                l1=K.l1_diagonal(A)[r0:r1].copy(),
                R=sp.csr_matrix(lev.R[int(nxt[q]):int(nxt[q + 1])]) if nxt is not None else None,
                P=sp.csr_matrix(lev.P[r0:r1]) if nxt is not None else None,
                iL=sp.csr_matrix(sp.csr_matrix(lev.ilu_L)[r0:r1, r0:r1]) if ilu else None,
                iU=sp.csr_matrix(sp.csr_matrix(lev.ilu_U)[r0:r1, r0:r1]) if ilu else None,
                idinv=np.asarray(lev.ilu_dinv)[r0:r1].copy() if ilu else None, Afull=A))

    # ---- one level's pieces (local vectors are the rank's rows) ----
    def residual(self, l, b, x):
        L = self.levels[l]
        return b - L.A @ self.comm.gather(x, L.off)

    def smooth(self, l, b, x, backward):
        p, L = self.p, self.levels[l]
        kind = level_smoother(self.H, l, p)
        r = self.residual(l, b, x)
        if kind == "jacobi":
            return x + r / L.l1
        if kind == "ilu":
            t = r.copy()
            y = t.copy()
            for _ in range(p.ilu_terms_L - 1):
                t = -(L.iL @ t)
                y = y + t
            f = L.idinv * y
            t = f.copy()
            v = t.copy()
            for _ in range(p.ilu_terms_U - 1):
                t = -(L.iU @ t)
                v = v + t
            return x + v
        if kind != "poly":
            raise NotImplementedError(f"sharded smoother '{kind}'")
        T = L.Ub if backward else L.Lb
        t = r / L.d
        g = t.copy()
        for _ in range(p.neumann_terms - 1):
            t = -(T @ t) / L.d
            g = g + t
        return x + g

    def vcycle(self, b, l=0):
        """z = M^-1 b, the hybrid V-cycle of oracle.vcycle.vcycle on the rank's rows."""
        p, L, H = self.p, self.levels[l], self.H
        if l == len(self.levels) - 1:
            if H.coarse_inv is not None:
                bf = self.comm.gather(b, L.off)
                z = K.coarse_direct(L.Afull, bf)
                return z[int(L.off[self.comm.rank]):int(L.off[self.comm.rank + 1])]
            x = np.zeros_like(b)
            for _ in range(p.coarse_sweeps):
                x = self.smooth(l, b, x, backward=False)
            return x
        x = np.zeros_like(b)
        for _ in range(p.pre_sweeps):
            x = self.smooth(l, b, x, backward=False)
        r = self.residual(l, b, x)
        bc = L.R @ self.comm.gather(r, L.off)
        e = self.vcycle(bc, l + 1)
        x = x + L.P @ self.comm.gather(e, self.levels[l + 1].off)
        for _ in range(p.post_sweeps):
            x = self.smooth(l, b, x, backward=True)
        return x


def gmres_onereduce_sharded(SH: ShardedHierarchy, b_loc: np.ndarray, m: int = 30, rtol: float = 1e-8,
                            maxit: int = 1000, T_mode: str = "trunc") -> GmresResult:
    """Algorithm 1 on the rank's rows (see oracle.gmres.gmres_onereduce for the step list); every
    inner product is a rank-local partial sum followed by a sum over the ranks, the 2(i+1)
    products of a step in one all_reduce. Returns the rank's rows of x."""
    comm = SH.comm
    L0 = SH.levels[0]
    dot = lambda u, v, purpose: float(comm.sum(np.array([np.dot(u, v)]), purpose)[0])
    n = b_loc.size
    x = np.zeros(n)
    bnorm = np.sqrt(dot(b_loc, b_loc, "norm_b"))
    if bnorm == 0.0:
        return GmresResult(x, 0, 0, True, 0.0, 0.0)
    iters, restarts, hist = 0, -1, []
    relres_imp = np.inf
    while True:
        vt = b_loc - L0.A @ comm.gather(x, L0.off)
        rnorm = np.sqrt(dot(vt, vt, "true_residual"))
        relres = rnorm / bnorm
        if relres <= rtol or iters >= maxit:
            return GmresResult(x, iters, max(restarts, 0), relres <= rtol, relres, min(relres_imp, relres), hist)
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
                z = SH.vcycle(vt)
                w = L0.A @ comm.gather(z, L0.off)
                cols = [V[:, j] for j in range(i)] + [vt]
                part = np.array([np.dot(c, vt) for c in cols] + [np.dot(c, w) for c in cols])
                red = comm.sum(part, "gram")  # the one reduction of step i (Algorithm 1 step 6)
                a, s = red[: i + 1], red[i + 1:]
                beta = float(np.sqrt(a[i]))
            else:
                beta = np.sqrt(dot(vt, vt, "last_norm"))
                z = w = None
            if i == 0:
                G = _Givens(m, beta)
            else:
                Hm[i, i - 1] = beta
                res = G.add_column(i - 1, Hm[: i + 1, i - 1])
                k = i
                relres_imp = res / bnorm
                hist.append(relres_imp)
                if beta == 0.0 or res <= rtol * bnorm or iters + i >= maxit:
                    done = True
            if done or z is None:
                break
            if beta == 0.0:
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
