"""Parity at the benchmark's full size, in its launch configuration: the 128^3 variable-coefficient
pressure Poisson system (n = 2,097,152, nnz = 14,581,760) with the same generator, seed, hierarchy
and solver parameters as bench.py (hybrid ILU(0) 3 + 3 terms, GMRES(50), autotuned layouts, one
CUDA graph per solve). The oracle's products are vectorised, so every kernel output is compared
with it element by element over the whole vector; the solve is compared with the oracle's
one-reduce GMRES (iteration counts within 1, x within 1e-6 relative), and the FP32-V-cycle solve
with the same FP64 oracle solution (within 1e-6 relative)."""
import numpy as np
import pytest

import oracle.kernels as K
from oracle.gmres import gmres_onereduce
from oracle.vcycle import vcycle as ovcycle
from workloads import build_hierarchy, pressure3d_7pt, rhs_uniform

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2112_14681_b300 import nsamg  # noqa: E402

EDGE, SEED, RESTART, RTOL = 128, 0, 50, 1e-8
HYBRID = dict(smoother=nsamg.HYBRID_ILU0, ilu_terms_L=3, ilu_terms_U=3, neumann_terms=2, pre_sweeps=1,
              post_sweeps=1, restart=RESTART)
TOL = 1e-12
_state = {}


def state():
    if not _state:
        A = pressure3d_7pt(EDGE, sigma=1.0, seed=SEED)
        H = build_hierarchy(A, theta=0.25, coarse_max=512, seed=SEED, ilu_levels=(0,))
        b = rhs_uniform(A.shape[0], SEED)
        p = nsamg.default_params(**HYBRID)
        op = K.SmootherParams(smoother=p.smoother, neumann_terms=p.neumann_terms, ilu_terms_L=p.ilu_terms_L,
                              ilu_terms_U=p.ilu_terms_U, pre_sweeps=p.pre_sweeps, post_sweeps=p.post_sweeps,
                              coarse_sweeps=p.coarse_sweeps)
        _state.update(A=A, H=H, b=b, p=p, op=op)
    return _state


def oracle_solution():
    s = state()
    if "ref" not in s:
        s["ref"] = gmres_onereduce(s["A"], s["b"], lambda v: ovcycle(s["H"], v, s["op"]), m=RESTART, rtol=RTOL)
    return s["ref"]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def test_fullsize_level0_kernels():
    """SpMV, residual, restriction, prolongation and the hybrid smoother's ILU(0) sweep on the
    finest level, whole vectors, componentwise within 1e-12 of their |.|-bounds."""
    s = state()
    A, H = s["A"], s["H"]
    lev = H.levels[0]
    n = A.shape[0]
    rng = np.random.default_rng(5)
    x, b = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    with nsamg.setup_hierarchy(H, s["p"]) as h:
        y = torch.empty(n, dtype=torch.float64, device="cuda")
        nsamg.level_spmv(h, 0, dev(x), y)
        bound = abs(A) @ np.abs(x)
        assert np.max(np.abs(host(y) - K.spmv(A, x)) / bound) <= TOL
        r = torch.empty_like(y)
        nsamg.level_residual(h, 0, dev(b), dev(x), r)
        assert np.max(np.abs(host(r) - K.residual(A, b, x)) / (bound + np.abs(b))) <= TOL
        nc = lev.R.shape[0]
        yc = torch.empty(nc, dtype=torch.float64, device="cuda")
        nsamg.level_restrict(h, 0, dev(x), yc)
        assert np.max(np.abs(host(yc) - K.restrict(lev.R, x)) / (abs(lev.R) @ np.abs(x))) <= TOL
        e = rng.uniform(-1, 1, nc)
        xt = dev(x)
        nsamg.level_prolong(h, 0, dev(e), xt)
        assert np.max(np.abs(host(xt) - K.prolong(lev.P, x, e)) / (np.abs(x) + abs(lev.P) @ np.abs(e))) <= TOL
        for x_zero in (True, False):
            x0 = np.zeros(n) if x_zero else x
            xt = dev(x0)
            nsamg.level_smooth(h, 0, dev(b), xt, backward=False, x_is_zero=x_zero)
            want = K.ilu0_sweep(lev.ilu_L, lev.ilu_U, lev.ilu_dinv, A, b, x0, 3, 3)
            assert np.max(np.abs(host(xt) - want)) <= TOL * np.max(np.abs(want))


def test_fullsize_vcycle():
    s = state()
    with nsamg.setup_hierarchy(s["H"], s["p"]) as h:
        z = torch.empty(s["A"].shape[0], dtype=torch.float64, device="cuda")
        nsamg.apply_vcycle(h, dev(s["b"]), z)
        want = ovcycle(s["H"], s["b"], s["op"])
        assert np.max(np.abs(host(z) - want)) <= 1e-11 * np.max(np.abs(want))


@pytest.mark.parametrize("i", [0, 17, RESTART - 1, 63])
@pytest.mark.parametrize("fp64", [0, 1])
def test_fullsize_gram_and_update(i, fp64):
    """The one-reduce Gram and update at i = 0, 17, 49 (the last column of GMRES(50)) and 63 (the
    largest restart) over 2^21 rows, double-FP32 and FP64 kernels."""
    n = 2 ** 21
    rng = np.random.default_rng(11 + i)
    ld = (n + 63) // 64 * 64
    Vb = np.zeros((i + 2, ld))
    Vb[: i + 1, :n] = rng.standard_normal((i + 1, n)) / np.sqrt(n)
    w = rng.standard_normal(n)
    Vt = dev(Vb.ravel())
    out = torch.empty(2 * (i + 1), dtype=torch.float64, device="cuda")
    (nsamg.gram_fp64 if fp64 else nsamg.gram)(n, i, Vt, ld, dev(w), out)
    a, sv = K.gram(Vb[:i, :n].T, Vb[i, :n], w)
    got = host(out)
    norms = np.sqrt(np.sum(Vb[: i + 1, :n] ** 2, axis=1))
    assert np.all(np.abs(got[: i + 1] - a) <= TOL * norms * np.linalg.norm(Vb[i, :n]))
    assert np.all(np.abs(got[i + 1:] - sv) <= TOL * norms * np.linalg.norm(w))
    beta = float(np.sqrt(a[i]))
    hcoef = rng.standard_normal(i + 1) * 1e-2
    ss = torch.empty(1, dtype=torch.float64, device="cuda")
    (nsamg.update_fp64 if fp64 else nsamg.update)(n, i, Vt, ld, dev(w), beta, dev(hcoef), ss)
    v_o, nxt_o = K.update(Vb[:i, :n].T, Vb[i, :n], w, beta, hcoef)
    Vg = host(Vt).reshape(i + 2, ld)
    assert np.max(np.abs(Vg[i, :n] - v_o)) <= TOL * np.max(np.abs(v_o))
    bound = np.abs(w) / beta + np.abs(Vb[:i, :n].T) @ np.abs(hcoef[:i]) + np.abs(v_o) * abs(hcoef[i])
    assert np.max(np.abs(Vg[i + 1, :n] - nxt_o) / bound) <= TOL
    assert abs(host(ss)[0] - np.dot(nxt_o, nxt_o)) <= TOL * np.dot(bound, bound)


def test_fullsize_solve_fp64_matches_oracle():
    s = state()
    ref = oracle_solution()
    with nsamg.setup_hierarchy(s["H"], s["p"]) as h:
        x = torch.zeros(s["A"].shape[0], dtype=torch.float64, device="cuda")
        st = nsamg.solve(h, dev(s["b"]), x, rtol=RTOL, maxit=500)
        xs = host(x)
    true = np.linalg.norm(s["b"] - s["A"] @ xs) / np.linalg.norm(s["b"])
    assert st["converged"] == 1 and true <= RTOL and abs(true - st["relres_true"]) <= 1e-12
    assert abs(st["iters"] - ref.iters) <= 1
    assert np.linalg.norm(xs - ref.x) / np.linalg.norm(ref.x) <= 1e-6


def test_fullsize_solve_fp32_vcycle_within_1e6_of_the_fp64_oracle():
    s = state()
    ref = oracle_solution()
    p = nsamg.default_params(**HYBRID, vcycle_fp32=1)
    with nsamg.setup_hierarchy(s["H"], p) as h:
        x = torch.zeros(s["A"].shape[0], dtype=torch.float64, device="cuda")
        st = nsamg.solve(h, dev(s["b"]), x, rtol=RTOL, maxit=500)
        xs = host(x)
    true = np.linalg.norm(s["b"] - s["A"] @ xs) / np.linalg.norm(s["b"])
    assert st["converged"] == 1 and true <= RTOL
    assert abs(st["iters"] - ref.iters) <= 1
    assert np.linalg.norm(xs - ref.x) / np.linalg.norm(ref.x) <= 1e-6


def test_fullsize_c3_graded_27pt_fp32_vcycle():
    """The 192^3 graded Q1 27-point case (n = 7,077,888, nnz = 189,119,224) with the benchmark's
    C3 settings (l1-Jacobi x2, FGMRES(30), FP32 V-cycle). The oracle cannot run 113 Arnoldi steps
    at this size in test time, so: finest-level SpMV rows sampled and recomputed by the oracle one
    by one; the FP32-V-cycle and FP64 solves both reach ||b - A x|| / ||b|| <= 1e-8 measured with
    the oracle's FP64 SpMV; their solutions agree within 1e-6."""
    from workloads.matrices import q1_27pt_graded
    A = q1_27pt_graded(192, aspect=100.0, seed=SEED)
    H = build_hierarchy(A, ilu_levels=(), coarse_max=512, seed=SEED)
    b = rhs_uniform(A.shape[0], SEED)
    n = A.shape[0]
    rng = np.random.default_rng(2)
    xr = rng.uniform(-1, 1, n)
    rows = rng.choice(n, 4096, replace=False)
    xs = {}
    for fp32 in (1, 0):
        p = nsamg.default_params(smoother=nsamg.JACOBI_L1, pre_sweeps=2, post_sweeps=2, restart=30, vcycle_fp32=fp32)
        with nsamg.setup_hierarchy(H, p) as h:
            if not fp32:
                y = torch.empty(n, dtype=torch.float64, device="cuda")
                nsamg.level_spmv(h, 0, dev(xr), y)
                yh = host(y)[rows]
                sub = A[rows]
                want = sub @ xr
                assert np.max(np.abs(yh - want) / (abs(sub) @ np.abs(xr))) <= TOL
            x = torch.zeros(n, dtype=torch.float64, device="cuda")
            st = nsamg.solve(h, dev(b), x, rtol=RTOL, maxit=2000)
            xs[fp32] = host(x)
        rel = np.linalg.norm(K.residual(A, b, xs[fp32])) / np.linalg.norm(b)
        assert st["converged"] == 1 and rel <= RTOL
    assert np.linalg.norm(xs[1] - xs[0]) / np.linalg.norm(xs[0]) <= 1e-6


def test_fullsize_c4_batched_256_systems():
    """The benchmark's batched workload as it times it: 256 seeded 7-point systems with edges drawn
    from 16..64, 4-level hierarchies, one nsamg_batch_solve, GMRES(30), FP32 and FP64 V-cycles.
    Every system's true residual is recomputed with the oracle's SpMV; three systems (smallest,
    largest, one in between) are solved by the oracle's one-reduce GMRES and compared (x within
    1e-6, iteration counts within 1 for the FP64 batch)."""
    import bench
    systems, _ = bench.build_pools(bench.BATCH_COUNT, 0)
    assert len(systems) == 256
    b = np.concatenate([bb for _, _, bb in systems])
    sizes = np.array([A.shape[0] for A, _, _ in systems])
    pick = [int(np.argmin(sizes)), int(np.argmax(sizes)), int(np.argsort(sizes)[128])]
    xs, stats = {}, {}
    for fp32 in (1, 0):
        p = nsamg.default_params(restart=bench.BATCH_RESTART, vcycle_fp32=fp32)
        with nsamg.batch_setup([H for _, H, _ in systems], p) as h:
            off = h.offsets
            x = torch.zeros(h.n, dtype=torch.float64, device="cuda")
            stats[fp32] = nsamg.batch_solve(h, dev(b), x, RTOL, bench.MAXIT)
            xs[fp32] = host(x)
        for k, (A, H, bb) in enumerate(systems):
            xk = xs[fp32][off[k]:off[k + 1]]
            assert stats[fp32][k]["converged"] == 1
            assert np.linalg.norm(K.residual(A, bb, xk)) / np.linalg.norm(bb) <= RTOL, k
    op = K.SmootherParams()  # the batch's default solve parameters: poly-GS, 2 terms, 1 + 1 sweeps
    for k in pick:
        A, H, bb = systems[k]
        ref = gmres_onereduce(A, bb, lambda v: ovcycle(H, v, op), m=bench.BATCH_RESTART, rtol=RTOL)
        for fp32 in (1, 0):
            xk = xs[fp32][off[k]:off[k + 1]]
            assert np.linalg.norm(xk - ref.x) / np.linalg.norm(ref.x) <= 1e-6, (k, fp32)
        assert abs(stats[0][k]["iters"] - ref.iters) <= 1


@pytest.mark.parametrize("name,kw", [
    ("poly_gs", dict(smoother=nsamg.POLY_GS, neumann_terms=2, pre_sweeps=1, post_sweeps=1)),
    ("l1_jacobi", dict(smoother=nsamg.JACOBI_L1, pre_sweeps=2, post_sweeps=2)),
])
def test_fullsize_other_smoothers_match_oracle(name, kw):
    """The benchmark's other FP64 smoothers on the 128^3 case: polynomial Gauss-Seidel (2 terms)
    and l1-Jacobi (2 + 2 sweeps), against the oracle's one-reduce GMRES with the same V-cycle."""
    s = state()
    p = nsamg.default_params(restart=RESTART, **kw)
    op = K.SmootherParams(smoother=p.smoother, neumann_terms=p.neumann_terms, pre_sweeps=p.pre_sweeps,
                          post_sweeps=p.post_sweeps, coarse_sweeps=p.coarse_sweeps)
    ref = gmres_onereduce(s["A"], s["b"], lambda v: ovcycle(s["H"], v, op), m=RESTART, rtol=RTOL)
    with nsamg.setup_hierarchy(s["H"], p) as h:
        x = torch.zeros(s["A"].shape[0], dtype=torch.float64, device="cuda")
        st = nsamg.solve(h, dev(s["b"]), x, rtol=RTOL, maxit=500)
        xs = host(x)
    true = np.linalg.norm(s["b"] - s["A"] @ xs) / np.linalg.norm(s["b"])
    assert st["converged"] == 1 and true <= RTOL
    assert abs(st["iters"] - ref.iters) <= 1, (st["iters"], ref.iters)
    assert np.linalg.norm(xs - ref.x) / np.linalg.norm(ref.x) <= 1e-6


def test_fullsize_hybrid_ilut_matches_oracle():
    """The benchmark's ILUT(1e-2, 5) line: finest-level ILUT factors with Ruiz-scaled U and 3 + 3
    Jacobi terms (Algorithm 2), polynomial GS below, against the oracle with the same factors."""
    import copy
    from workloads.hierarchy import Hierarchy, ilut
    s = state()
    H = s["H"]
    l0 = copy.copy(H.levels[0])
    l0.ilu_L, l0.ilu_U, l0.ilu_dr, l0.ilu_dc = ilut(l0.A, 1e-2, 5)
    l0.ilu_dinv, l0.ilu_form = None, 1
    Ht = Hierarchy(levels=[l0] + H.levels[1:], coarse_inv=H.coarse_inv, theta=H.theta, seed=H.seed, info=H.info)
    ref = gmres_onereduce(s["A"], s["b"], lambda v: ovcycle(Ht, v, s["op"]), m=RESTART, rtol=RTOL)
    with nsamg.setup_hierarchy(Ht, s["p"]) as h:
        x = torch.zeros(s["A"].shape[0], dtype=torch.float64, device="cuda")
        st = nsamg.solve(h, dev(s["b"]), x, rtol=RTOL, maxit=500)
        xs = host(x)
    true = np.linalg.norm(s["b"] - s["A"] @ xs) / np.linalg.norm(s["b"])
    assert st["converged"] == 1 and true <= RTOL
    assert abs(st["iters"] - ref.iters) <= 1, (st["iters"], ref.iters)
    assert np.linalg.norm(xs - ref.x) / np.linalg.norm(ref.x) <= 1e-6
