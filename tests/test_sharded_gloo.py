"""The row-sharded solve of the paper's multi-rank runs, on CPU ranks (gloo): the hybrid
block-Jacobi smoother (Sec. 5.2) pinned to closed forms, and the sharded one-reduce GMRES
(oracle/sharded.py: rows of every level dealt to the ranks, one all_reduce of 2(i+1) values per
Arnoldi step) against the unsharded oracle run with the same hybrid V-cycle."""
import os
import socket

import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from oracle import kernels as K  # noqa: E402


def _poisson2d(k):
    T = sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], shape=(k, k))
    I = sp.identity(k)
    return sp.csr_matrix(sp.kron(T, I) + sp.kron(I, T))


def test_row_blocks_cover_the_rows():
    for n, p in [(10, 3), (7, 7), (5, 8), (1000, 4)]:
        off = K.row_blocks(n, p)
        assert off[0] == 0 and off[-1] == n and np.all(np.diff(off) >= 0) and off.size == p + 1
        assert np.max(np.diff(off)) == -(-n // p)


def test_local_block_keeps_exactly_the_in_block_couplings():
    A = sp.csr_matrix(sp.random(40, 40, density=0.25, random_state=3) + sp.identity(40))
    for p in (1, 3, 6):
        off = K.row_blocks(40, p)
        blk = np.searchsorted(off, np.arange(40), side="right")
        D = A.toarray()
        want = np.where(blk[:, None] == blk[None, :], D, 0.0)  # brute force over all (i, j)
        assert np.array_equal(K.local_block(A, p).toarray(), want)


def test_hybrid_poly_gs_with_one_row_per_rank_is_jacobi():
    """Every row its own rank: no coupling left inside a block, so any number of Neumann terms
    gives the Jacobi step x + D^-1 r (the zero-inner-sweep case of Sec. 5.2)."""
    A = _poisson2d(9)
    n = A.shape[0]
    rng = np.random.default_rng(0)
    b, x = rng.standard_normal(n), rng.standard_normal(n)
    got = K.poly_gs_sweep(A, b, x, terms=4, ranks=n)
    assert np.allclose(got, x + (b - A @ x) / A.diagonal(), rtol=1e-14, atol=1e-14)
    got_b = K.poly_gs_sweep(A, b, x, terms=3, backward=True, ranks=n)
    assert np.allclose(got_b, got, rtol=1e-14, atol=1e-14)


def test_hybrid_poly_gs_equals_global_on_a_block_diagonal_operator():
    """With no couplings across the rank blocks, the hybrid sweep is the global sweep, and with
    one rank it is the global sweep for any operator."""
    blocks = [_poisson2d(5) * (1.0 + q) for q in range(3)]
    A = sp.csr_matrix(sp.block_diag(blocks))
    n = A.shape[0]
    rng = np.random.default_rng(1)
    b, x = rng.standard_normal(n), rng.standard_normal(n)
    for mode in ("definition", "direct"):
        assert np.array_equal(K.poly_gs_sweep(A, b, x, 3, mode=mode, ranks=3), K.poly_gs_sweep(A, b, x, 3, mode=mode))
    B = _poisson2d(8)
    bb, xx = rng.standard_normal(64), rng.standard_normal(64)
    assert np.array_equal(K.poly_gs_sweep(B, bb, xx, 3, ranks=1), K.poly_gs_sweep(B, bb, xx, 3))


def test_hybrid_direct_sweep_solves_the_local_triangles():
    """mode='direct' with ranks: x + (D + L_loc)^-1 r, checked against a dense solve with the
    in-block lower triangle written out from the definition."""
    A = _poisson2d(6)
    n = A.shape[0]
    rng = np.random.default_rng(2)
    b, x = rng.standard_normal(n), rng.standard_normal(n)
    off = K.row_blocks(n, 4)
    blk = np.searchsorted(off, np.arange(n), side="right")
    D = A.toarray()
    M = np.tril(np.where(blk[:, None] == blk[None, :], D, 0.0))
    want = x + np.linalg.solve(M, b - A @ x)
    assert np.allclose(K.poly_gs_sweep(A, b, x, 3, mode="direct", ranks=4), want, rtol=1e-12, atol=1e-12)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem(ranks):
    from workloads import build_hierarchy, pressure3d_7pt, rhs_uniform
    A = pressure3d_7pt(14, sigma=1.0, seed=5)
    H = build_hierarchy(A, coarse_max=64, seed=5, ilu_levels=(0,), ranks=ranks)
    return A, H, rhs_uniform(A.shape[0], 5)


def _worker(rank, world, port, smoother, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import sharded
    A, H, b = _problem(world)
    p = K.SmootherParams(smoother=smoother, neumann_terms=2, ilu_terms_L=3, ilu_terms_U=3, ranks=world)
    comm = sharded.Comm()
    SH = sharded.ShardedHierarchy(H, comm, p)
    off = K.row_blocks(A.shape[0], world)
    res = sharded.gmres_onereduce_sharded(SH, b[off[rank]:off[rank + 1]], m=12, rtol=1e-8)
    xs = comm.gather(res.x, off)
    out[rank] = (xs, res.iters, res.restarts, res.converged, dict(comm.allreduce))
    dist.destroy_process_group()


def _run(world, smoother):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, smoother, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    return [out[r] for r in range(world)]


@pytest.mark.parametrize("world,smoother", [(1, K.HYBRID_ILU0), (2, K.HYBRID_ILU0), (3, K.POLY_GS), (2, K.JACOBI_L1)])
def test_sharded_gmres_matches_the_unsharded_hybrid_oracle(world, smoother):
    from oracle.gmres import gmres_onereduce
    from oracle.vcycle import vcycle
    A, H, b = _problem(world)
    p = K.SmootherParams(smoother=smoother, neumann_terms=2, ilu_terms_L=3, ilu_terms_U=3, ranks=world)
    ref = gmres_onereduce(A, b, lambda v: vcycle(H, v, p), m=12, rtol=1e-8)
    outs = _run(world, smoother)
    x0, iters, restarts, conv, red = outs[0]
    assert conv and ref.converged
    for xs, it, _, _, red_q in outs[1:]:  # every rank ends with the same solution and counts
        assert np.array_equal(xs, x0) and it == iters and red_q == red
    assert iters == ref.iters and restarts == ref.restarts
    tol = 0.0 if world == 1 else 1e-10  # one rank: the same arithmetic in the same order
    assert np.linalg.norm(x0 - ref.x) <= tol * np.linalg.norm(ref.x)
    # one reduction per Arnoldi step (its 2(i+1) inner products) plus one lagged norm when a
    # cycle runs to m columns; one true-residual norm per cycle and one for the final check
    assert red["gram"] + red.get("last_norm", 0) == iters + restarts + 1
    assert red["true_residual"] == restarts + 2 and red["norm_b"] == 1


def test_more_ranks_mean_a_weaker_smoother():
    """Splitting the hybrid smoother over more ranks drops couplings from its local triangles:
    the unsharded oracle needs at least as many iterations with 8 blocks as with 1 (the paper's
    hybrid smoothers lose a little convergence as the rank count grows)."""
    from oracle.gmres import gmres_onereduce
    from oracle.vcycle import vcycle
    its = []
    for ranks in (1, 8):
        A, H, b = _problem(ranks)
        p = K.SmootherParams(smoother=K.HYBRID_ILU0, neumann_terms=2, ilu_terms_L=3, ilu_terms_U=3, ranks=ranks)
        its.append(gmres_onereduce(A, b, lambda v: vcycle(H, v, p), m=30, rtol=1e-8).iters)
    assert its[1] >= its[0]
