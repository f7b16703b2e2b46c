"""Batched solves (block-diagonal batching, lock-step GMRES with per-system state) against the
FP64 oracle run on every system separately."""
import numpy as np
import pytest

import oracle.kernels as K
from oracle.gmres import gmres_onereduce
from oracle.vcycle import vcycle as ovcycle
from workloads import build_hierarchy, pressure3d_7pt, rhs_uniform

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2112_14681_b300 import nsamg  # noqa: E402

EDGES = [6, 9, 7, 12, 8, 10]
_sys = None


def systems():
    global _sys
    if _sys is None:
        out = []
        for k, e in enumerate(EDGES):
            A = pressure3d_7pt(e, seed=100 + k)
            H = build_hierarchy(A, max_levels=3, coarse_max=8, direct_max=10_000, ilu_levels=None, seed=k)
            assert H.nlevels == 3 and H.coarse_inv is not None
            out.append((A, H, rhs_uniform(A.shape[0], 200 + k)))
        _sys = out
    return _sys


def oparams(p):
    return K.SmootherParams(smoother=p.smoother, neumann_terms=p.neumann_terms, ilu_terms_L=p.ilu_terms_L,
                            ilu_terms_U=p.ilu_terms_U, pre_sweeps=p.pre_sweeps, post_sweeps=p.post_sweeps)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("fp32", [0, 1])
@pytest.mark.parametrize("smoother", [K.POLY_GS, K.HYBRID_ILU0])
def test_batch_vcycle_is_per_system_vcycle(fp32, smoother):
    S = systems()
    p = nsamg.default_params(smoother=smoother, vcycle_fp32=fp32)
    with nsamg.batch_setup([H for _, H, _ in S], p) as h:
        off = h.offsets
        r = np.concatenate([b for _, _, b in S])
        z = torch.empty(h.n, dtype=torch.float64, device="cuda")
        nsamg.apply_vcycle(h, dev(r), z)
        torch.cuda.synchronize()
        zg = z.cpu().numpy()
    tol = 1e-4 if fp32 else 1e-11
    for k, (A, H, b) in enumerate(S):
        want = ovcycle(H, b, oparams(p))
        got = zg[off[k]:off[k + 1]]
        assert np.linalg.norm(got - want) <= tol * np.linalg.norm(want), k


@pytest.mark.parametrize("fp32", [0, 1])
@pytest.mark.parametrize("smoother", [K.POLY_GS, K.HYBRID_ILU0])
@pytest.mark.parametrize("graph,krylov_fp64", [(1, 0), (0, 0), (1, 1)])
def test_batch_solve_matches_oracle_per_system(fp32, smoother, graph, krylov_fp64):
    """Every system against the oracle's one-reduce GMRES with its own V-cycle. The systems' sizes
    (216, 729, 343, 1728, 512, 1000 rows) put odd first and last rows into the split basis's
    row pairs (krylov_fp64 = 0); krylov_fp64 = 1 keeps the FP64 basis."""
    S = systems()
    m = 30
    p = nsamg.default_params(smoother=smoother, vcycle_fp32=fp32, restart=m, use_graph=graph,
                             krylov_fp64=krylov_fp64)
    with nsamg.batch_setup([H for _, H, _ in S], p) as h:
        off = h.offsets
        b = np.concatenate([bb for _, _, bb in S])
        x = torch.zeros(h.n, dtype=torch.float64, device="cuda")
        stats = nsamg.batch_solve(h, dev(b), x, rtol=1e-8, maxit=400)
        torch.cuda.synchronize()
        xg = x.cpu().numpy()
    assert len(stats) == len(S)
    for k, (A, H, bb) in enumerate(S):
        st = stats[k]
        xs = xg[off[k]:off[k + 1]]
        ref = gmres_onereduce(A, bb, lambda v: ovcycle(H, v, oparams(p)), m=m, rtol=1e-8)
        true = np.linalg.norm(bb - A @ xs) / np.linalg.norm(bb)
        assert st["converged"] == 1 and true <= 1e-8 and abs(true - st["relres_true"]) <= 1e-12
        assert abs(st["iters"] - ref.iters) <= 1, (k, st["iters"], ref.iters)
        if not fp32:
            assert np.linalg.norm(xs - ref.x) / np.linalg.norm(ref.x) <= 1e-6
        # per-system ||S_k||_2 of the last cycle: tiny (the basis stays independent), nonzero
        assert 0.0 < st["sk_norm"] <= st["orth_loss"] < 1e-6


def test_batch_fp32v_solution_matches_fp64_oracle():
    """Mixed precision (FP32 V-cycle inside FP64 flexible GMRES): every system's x within 1e-6
    relative of the FP64 oracle's x. Both solve to rtol 1e-10, so the difference measures the
    mixed-precision error rather than the kappa * rtol band that any two solutions meeting
    rtol 1e-8 may differ by."""
    S = systems()
    m = 30
    p = nsamg.default_params(vcycle_fp32=1, restart=m)
    with nsamg.batch_setup([H for _, H, _ in S], p) as h:
        off = h.offsets
        b = np.concatenate([bb for _, _, bb in S])
        x = torch.zeros(h.n, dtype=torch.float64, device="cuda")
        stats = nsamg.batch_solve(h, dev(b), x, rtol=1e-10, maxit=400)
        torch.cuda.synchronize()
        xg = x.cpu().numpy()
    for k, (A, H, bb) in enumerate(S):
        ref = gmres_onereduce(A, bb, lambda v: ovcycle(H, v, oparams(p)), m=m, rtol=1e-10)
        xs = xg[off[k]:off[k + 1]]
        assert stats[k]["converged"] == 1
        assert np.linalg.norm(xs - ref.x) / np.linalg.norm(ref.x) <= 1e-6, k


def test_batch_stops_on_backward_error():
    """stop_nrbe = 1 in a batch: each system stops on beta(x) <= rtol (Sec. 3) like the oracle's
    one-reduce GMRES with the same stop (iterations within 1, beta(x) recomputed on the host)."""
    S = systems()
    m = 6
    p = nsamg.default_params(restart=m, stop_nrbe=1)
    with nsamg.batch_setup([H for _, H, _ in S], p) as h:
        off = h.offsets
        b = np.concatenate([bb for _, _, bb in S])
        x = torch.zeros(h.n, dtype=torch.float64, device="cuda")
        stats = nsamg.batch_solve(h, dev(b), x, rtol=1e-8, maxit=400)
        torch.cuda.synchronize()
        xg = x.cpu().numpy()
    for k, (A, H, bb) in enumerate(S):
        ref = gmres_onereduce(A, bb, lambda v: ovcycle(H, v, oparams(p)), m=m, rtol=1e-8, stop="nrbe")
        xs = xg[off[k]:off[k + 1]]
        Ad = A.toarray()
        beta = np.linalg.norm(bb - Ad @ xs) / (np.linalg.norm(bb) + np.abs(Ad).sum(axis=1).max() * np.linalg.norm(xs))
        assert stats[k]["converged"] == 1 and beta <= 1e-8
        assert stats[k]["nrbe"] == pytest.approx(beta, rel=1e-6)
        assert abs(stats[k]["iters"] - ref.iters) <= 1, (k, stats[k]["iters"], ref.iters)


def test_batch_mixed_progress_and_restarts():
    """One system starts at its solution and one has b = 0: they finish at once while the others
    keep stepping; a short restart length forces restarts in lock step."""
    S = systems()
    p = nsamg.default_params(restart=3)
    with nsamg.batch_setup([H for _, H, _ in S], p) as h:
        off = h.offsets
        bs = [bb.copy() for _, _, bb in S]
        bs[1][:] = 0.0
        x0 = np.zeros(h.n)
        A2 = S[2][0]
        x0[off[2]:off[3]] = np.linalg.solve(A2.toarray(), bs[2])
        x = dev(x0)
        stats = nsamg.batch_solve(h, dev(np.concatenate(bs)), x, rtol=1e-8, maxit=600)
        torch.cuda.synchronize()
        xg = x.cpu().numpy()
    assert stats[1]["iters"] == 0 and stats[1]["converged"] and np.all(xg[off[1]:off[2]] == 0)
    assert stats[2]["iters"] == 0 and stats[2]["converged"]
    assert stats[1]["sk_norm"] == 0.0 and stats[2]["sk_norm"] == 0.0  # no cycle ran
    for k in (0, 3, 4, 5):
        A = S[k][0]
        xs = xg[off[k]:off[k + 1]]
        assert stats[k]["converged"] and stats[k]["restarts"] >= 1
        assert np.linalg.norm(bs[k] - A @ xs) / np.linalg.norm(bs[k]) <= 1e-8


def test_batch_rejects_uneven_depth():
    S = systems()
    A = pressure3d_7pt(8, seed=1)
    H2 = build_hierarchy(A, max_levels=2, coarse_max=8)
    with pytest.raises(nsamg.NsamgError) as ei:
        nsamg.batch_setup([S[0][1], H2], nsamg.default_params())
    assert ei.value.status == -1
