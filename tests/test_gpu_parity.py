"""GPU parity: every kernel of the CUDA path, called through the C ABI, against the FP64 oracle
on the same seeded inputs. Tolerances: per-kernel FP64 results within 1e-12 relative
(componentwise against |A||x| for products, norm-wise for multi-pass sweeps); solves reach
relative residual 1e-8 with iteration counts within +-1 of the oracle."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle.kernels as K
from oracle.gmres import gmres_mgs, gmres_onereduce
from oracle.vcycle import vcycle as ovcycle, level_smoother
from workloads import build_hierarchy, poisson2d_5pt, pressure3d_7pt, rhs_uniform

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2112_14681_b300 import nsamg  # noqa: E402

TOL = 1e-12


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def params_for(smoother, **kw):
    d = dict(smoother=smoother)
    if smoother == K.JACOBI_L1:
        d.update(pre_sweeps=2, post_sweeps=2)
    d.update(kw)
    return d


def oracle_params(p: nsamg.Params):
    return K.SmootherParams(smoother=p.smoother, neumann_terms=p.neumann_terms, ilu_terms_L=p.ilu_terms_L,
                            ilu_terms_U=p.ilu_terms_U, pre_sweeps=p.pre_sweeps, post_sweeps=p.post_sweeps,
                            coarse_sweeps=p.coarse_sweeps, ranks=p.ranks)


CASES = {
    # C1: 2D 5-point 32x32, 3 levels
    "c1": lambda: (poisson2d_5pt(32), dict(max_levels=3, coarse_max=64)),
    # ragged 3D variable-coefficient case: 23^3 = 12167 rows (not a multiple of any tile)
    "p23": lambda: (pressure3d_7pt(23, seed=3), dict(coarse_max=100)),
    # deeper hierarchy with a coarsest level solved by sweeps (no dense inverse)
    "p20s": lambda: (pressure3d_7pt(20, seed=5), dict(coarse_max=600, direct_max=0)),
    # 30^3 = 27000 rows: finest level above the SELL threshold, several sorting windows, ragged
    # last chunk
    "p30": lambda: (pressure3d_7pt(30, seed=8), dict(coarse_max=200)),
    # ILUT(1e-2, 5) factors with Ruiz-scaled U on every level (Algorithm 2)
    "p23t": lambda: (pressure3d_7pt(23, seed=3), dict(coarse_max=100, ilu="ilut", droptol=1e-2, lfil=5)),
    # the same with Ruiz stopped by the dep(U) test of Sec. 5.3 (eq. depU)
    "p23d": lambda: (pressure3d_7pt(23, seed=3), dict(coarse_max=100, ilu="ilut", droptol=1e-2, lfil=5,
                                                      ruiz_stop="dep")),
}

_cache = {}


def case(name):
    if name not in _cache:
        A, kw = CASES[name]()
        H = build_hierarchy(A, ilu_levels=None, **kw)
        _cache[name] = (A, H)
    return _cache[name]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    nsamg.load()
    yield


def rel_err_componentwise(y, yo, bound):
    return float(np.max(np.abs(y - yo) / np.maximum(bound, 1e-300)))


@pytest.mark.parametrize("layout", [0, -1, 1])
@pytest.mark.parametrize("name", list(CASES))
def test_level_spmv_residual_transfer(name, layout):
    A, H = case(name)
    with nsamg.setup_hierarchy(H, nsamg.default_params(spmv_group=layout)) as h:
        if layout == -1 and H.levels[0].n >= 16384:
            assert nsamg.level_group(h, 0) == 0
        assert nsamg.num_levels(h) == H.nlevels
        rng = np.random.default_rng(1)
        for l, lev in enumerate(H.levels):
            n = lev.n
            x, b = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
            bound = abs(lev.A) @ np.abs(x)
            y = torch.empty(n, dtype=torch.float64, device="cuda")
            nsamg.level_spmv(h, l, dev(x), y)
            assert rel_err_componentwise(host(y), K.spmv(lev.A, x), bound) <= TOL
            r = torch.empty_like(y)
            nsamg.level_residual(h, l, dev(b), dev(x), r)
            assert rel_err_componentwise(host(r), K.residual(lev.A, b, x), bound + np.abs(b)) <= TOL
            if l < H.nlevels - 1:
                nc = lev.R.shape[0]
                yc = torch.empty(nc, dtype=torch.float64, device="cuda")
                nsamg.level_restrict(h, l, dev(x), yc)
                assert rel_err_componentwise(host(yc), K.restrict(lev.R, x), abs(lev.R) @ np.abs(x)) <= TOL
                e = rng.uniform(-1, 1, nc)
                xt = dev(x)
                nsamg.level_prolong(h, l, dev(e), xt)
                assert rel_err_componentwise(host(xt), K.prolong(lev.P, x, e), np.abs(x) + abs(lev.P) @ np.abs(e)) <= TOL


SMOOTHERS = [(K.POLY_GS, 2), (K.POLY_GS, 1), (K.POLY_GS, 4), (K.ILU0, 3), (K.HYBRID_ILU0, 3), (K.JACOBI_L1, 1)]


@pytest.mark.parametrize("smoother,terms", SMOOTHERS)
@pytest.mark.parametrize("backward", [False, True])
@pytest.mark.parametrize("x_zero", [True, False])
@pytest.mark.parametrize("name,layout", [("p23", 0), ("p30", -1), ("p23t", 0)])
def test_smoother_sweep(smoother, terms, backward, x_zero, name, layout):
    A, H = case(name)
    kw = dict(smoother=smoother, neumann_terms=terms, ilu_terms_L=terms, ilu_terms_U=max(1, terms - 1),
              spmv_group=layout)
    p = nsamg.default_params(**kw)
    op = oracle_params(p)
    with nsamg.setup_hierarchy(H, p) as h:
        rng = np.random.default_rng(7)
        for l in range(H.nlevels - 1):
            lev = H.levels[l]
            b = rng.uniform(-1, 1, lev.n)
            x0 = np.zeros(lev.n) if x_zero else rng.uniform(-1, 1, lev.n)
            xt = dev(x0)
            nsamg.level_smooth(h, l, dev(b), xt, backward=backward, x_is_zero=x_zero)
            kind = level_smoother(H, l, op)
            if kind == "ilu":
                want = K.ilu0_sweep(lev.ilu_L, lev.ilu_U, lev.ilu_dinv, lev.A, b, x0, op.ilu_terms_L, op.ilu_terms_U)
            elif kind == "ilut":
                want = K.ilut_sweep(lev.ilu_L, lev.ilu_U, lev.ilu_dr, lev.ilu_dc, lev.A, b, x0, op.ilu_terms_L,
                                    op.ilu_terms_U)
            elif kind == "jacobi":
                want = K.l1_jacobi_sweep(lev.A, b, x0)
            else:
                want = K.poly_gs_sweep(lev.A, b, x0, op.neumann_terms, backward=backward)
            got = host(xt)
            assert np.max(np.abs(got - want)) <= TOL * max(1.0, np.max(np.abs(want))), (l, kind)


@pytest.mark.parametrize("name", list(CASES))
def test_coarse_solve(name):
    A, H = case(name)
    p = nsamg.default_params()
    with nsamg.setup_hierarchy(H, p) as h:
        lev = H.levels[-1]
        b = np.random.default_rng(3).uniform(-1, 1, lev.n)
        z = torch.empty(lev.n, dtype=torch.float64, device="cuda")
        nsamg.coarse_solve(h, dev(b), z)
        if H.coarse_inv is not None:
            want = K.coarse_direct(lev.A, b)
            kappa = np.linalg.cond(lev.A.toarray())
            assert np.max(np.abs(host(z) - want)) <= 1e-14 * kappa * np.max(np.abs(want)) + TOL
        else:
            x = np.zeros(lev.n)
            for _ in range(p.coarse_sweeps):
                x = K.poly_gs_sweep(lev.A, b, x, p.neumann_terms, backward=False)
            assert np.max(np.abs(host(z) - x)) <= TOL * np.max(np.abs(x))


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("smoother", [K.POLY_GS, K.HYBRID_ILU0, K.ILU0, K.JACOBI_L1])
def test_vcycle(name, smoother):
    A, H = case(name)
    p = nsamg.default_params(**params_for(smoother), spmv_group=-1 if name == "p30" else 0)
    with nsamg.setup_hierarchy(H, p) as h:
        r = rhs_uniform(A.shape[0], 11)
        z = torch.empty(A.shape[0], dtype=torch.float64, device="cuda")
        nsamg.apply_vcycle(h, dev(r), z)
        want = ovcycle(H, r, oracle_params(p))
        got = host(z)
        assert np.max(np.abs(got - want)) <= 1e-11 * np.max(np.abs(want))


def _gram_update_case(n, i, fp64, vscale=1.0, wscale=1.0, zero_rows=0, seed=0, aligned=False):
    """Random orthonormal V_i, an unnormalised vt, scaled (vt, w) pair; checks the Gram (step 6)
    and the update (steps 8, 12) against the oracle's gram / update componentwise: each dot
    product within TOL of ||a|| ||b|| (Cauchy-Schwarz), each updated entry within TOL of the sum
    of the absolute values of its terms."""
    rng = np.random.default_rng(n + i + seed)
    # aligned: every column start on a 16-byte boundary (the bulk-copy Gram); else an odd stride
    ld = (n + 63) // 64 * 64 if aligned else n + (7 if n > 1 else 0)
    Vb = np.zeros((i + 2, ld))
    Q, _ = np.linalg.qr(rng.standard_normal((n, i + 1))) if n >= i + 1 else (rng.standard_normal((n, i + 1)), None)
    Vb[: i + 1, :n] = Q.T[: i + 1]
    Vb[i, :n] = rng.standard_normal(n) * 3.0 * vscale  # unnormalised newest vector
    w = rng.standard_normal(n) * wscale
    if zero_rows:
        Vb[:, :zero_rows] = 0.0
        w[:zero_rows] = 0.0
    Vt = dev(Vb.ravel())
    out = torch.empty(2 * (i + 1), dtype=torch.float64, device="cuda")
    (nsamg.gram_fp64 if fp64 else nsamg.gram)(n, i, Vt, ld, dev(w), out)
    a, s = K.gram(Vb[:i, :n].T, Vb[i, :n], w)
    got = host(out)
    scale_a = np.sqrt(np.sum(Vb[: i + 1, :n] ** 2, axis=1)) * np.linalg.norm(Vb[i, :n])
    scale_s = np.sqrt(np.sum(Vb[: i + 1, :n] ** 2, axis=1)) * np.linalg.norm(w)
    assert np.all(np.abs(got[: i + 1] - a) <= TOL * scale_a)
    assert np.all(np.abs(got[i + 1:] - s) <= TOL * scale_s)
    beta = float(np.sqrt(a[i]))
    hcoef = rng.standard_normal(i + 1) * wscale / max(vscale, 1e-300)
    ss = torch.empty(1, dtype=torch.float64, device="cuda")
    (nsamg.update_fp64 if fp64 else nsamg.update)(n, i, Vt, ld, dev(w), beta, dev(hcoef), ss)
    v_o, nxt_o = K.update(Vb[:i, :n].T, Vb[i, :n], w, beta, hcoef)
    Vg = host(Vt).reshape(i + 2, ld)
    assert np.max(np.abs(Vg[i, :n] - v_o)) <= TOL * np.max(np.abs(v_o))
    bound = np.abs(w) / beta + np.abs(Vb[:i, :n].T) @ np.abs(hcoef[:i]) + np.abs(v_o) * abs(hcoef[i])
    nz = bound > 0
    assert np.all(Vg[i + 1, :n][~nz] == 0.0)
    assert np.max(np.abs(Vg[i + 1, :n] - nxt_o)[nz] / bound[nz]) <= TOL
    assert abs(host(ss)[0] - np.dot(nxt_o, nxt_o)) <= TOL * np.dot(bound, bound)


@pytest.mark.parametrize("fp64", [0, 1])
@pytest.mark.parametrize("n,i", [(1, 0), (1000, 0), (1000, 1), (4097, 3), (100003, 17), (262144, 63), (70001, 10)])
def test_gram_and_update(n, i, fp64):
    _gram_update_case(n, i, fp64)


@pytest.mark.parametrize("n,i", [(1, 0), (2, 1), (3, 2), (1000, 0), (1001, 1), (4097, 3), (100003, 17), (262147, 63),
                                 (70001, 10), (148 * 96 + 1, 40), (5000, 8), (33333, 33)])
def test_gram_and_update_aligned_columns(n, i):
    """16-byte aligned columns: the Gram runs its bulk-copy pipeline (ragged tiles, odd last rows,
    one-row tiles, empty blocks)."""
    _gram_update_case(n, i, 0, aligned=True)


@pytest.mark.parametrize("vscale,wscale", [(1e30, 1e30), (1e-30, 1e-30), (1.0, 1e25), (1.0, 1e-20), (1e-12, 1.0)])
def test_gram_and_update_outside_the_double_fp32_window(vscale, wscale):
    """vt and w far from unit scale: the double-FP32 kernels fall back to FP64 for the blocks
    (Gram) and rows (update) whose magnitudes leave [2^-50, 2^60]; results still within TOL."""
    _gram_update_case(50021, 12, 0, vscale=vscale, wscale=wscale)
    _gram_update_case(50021, 12, 0, vscale=vscale, wscale=wscale, aligned=True)


def _split_case(n, i, wscale=1.0, seed=0):
    """The solve's split-basis kernels: unnormalised columns vt_0..vt_i stored as (hi, lo) pairs by
    nsamg_split_basis; the Gram's raw products against the oracle's gram on the FP64 columns, the
    update against the oracle's update with v_j = vt_j / beta_j (coefficients c_j = h_j / beta_j),
    and the stored pair of the new column against its FP64 value."""
    rng = np.random.default_rng(7 * n + i + seed)
    ld = (n + 63) // 64 * 64
    Vb = np.zeros((i + 2, ld))
    Vb[: i + 1, :n] = rng.standard_normal((i + 1, n)) * rng.uniform(0.3, 3.0, (i + 1, 1))
    w = rng.standard_normal(n) * wscale
    Vs = torch.zeros(2 * ld * (i + 2), dtype=torch.float32, device="cuda")
    nsamg.split_basis(n, i + 1, dev(Vb.ravel()), ld, Vs, ld)
    out = torch.empty(2 * (i + 1), dtype=torch.float64, device="cuda")
    dw = dev(w)
    nsamg.gram_split(n, i, Vs, ld, dw, out)
    a, s_ = K.gram(Vb[:i, :n].T, Vb[i, :n], w)
    got = host(out)
    norms = np.sqrt(np.sum(Vb[: i + 1, :n] ** 2, axis=1))
    assert np.all(np.abs(got[: i + 1] - a) <= TOL * norms * norms[i])
    assert np.all(np.abs(got[i + 1:] - s_) <= TOL * norms * np.linalg.norm(w))
    betas = norms * rng.uniform(0.5, 2.0, i + 1)
    hcoef = rng.standard_normal(i + 1)
    c = hcoef / betas
    vin = torch.empty(n, dtype=torch.float64, device="cuda")
    ss = torch.empty(1, dtype=torch.float64, device="cuda")
    nsamg.update_split(n, i, Vs, ld, dw, float(betas[i]), dev(c), vin, ss)
    Vn = (Vb[:i, :n] / betas[:i, None]).T
    _, nxt_o = K.update(Vn, Vb[i, :n], w, float(betas[i]), hcoef)
    bound = np.abs(w) / betas[i] + np.abs(Vn) @ np.abs(hcoef[:i]) + np.abs(Vb[i, :n] / betas[i]) * abs(hcoef[i])
    g = host(vin)
    assert np.max(np.abs(g - nxt_o) / bound) <= TOL
    assert abs(host(ss)[0] - np.dot(nxt_o, nxt_o)) <= TOL * np.dot(bound, bound)
    # row-pair layout: group q of a column = (hi_2q, hi_2q+1, lo_2q, lo_2q+1)
    grp = host(Vs).reshape(i + 2, ld // 2, 2, 2)[i + 1].astype(np.float64)
    hi, lo = grp[:, 0, :].reshape(-1), grp[:, 1, :].reshape(-1)
    assert np.max(np.abs(hi[:n] + lo[:n] - g) / np.maximum(np.abs(g), 1e-300)) <= 2.0 ** -44
    assert np.all(hi[n:] == 0) and np.all(lo[n:] == 0)  # rows past n (padding) stay zero


@pytest.mark.parametrize("n,i", [(1, 0), (2, 1), (999, 0), (1001, 1), (4097, 3), (70001, 10), (100003, 17),
                                 (148 * 96 + 1, 40), (262147, 63), (33333, 30)])
def test_split_basis_gram_and_update(n, i):
    _split_case(n, i)


@pytest.mark.parametrize("wscale", [1e30, 1e-30])
def test_split_basis_w_outside_the_window(wscale):
    """w far from unit scale: the Gram's blocks and the update's rows fall back to FP64."""
    _split_case(50021, 12, wscale=wscale)


@pytest.mark.parametrize("scale", [1e-30, 1e30, 2.0 ** -100])
def test_solve_is_scale_invariant(scale):
    """b scaled by a constant: the split basis stores the residual at unit scale (the exact power of
    two goes into g_0), so the solve takes the same iterations and returns the scaled x."""
    A, H = case("p23")
    b = rhs_uniform(A.shape[0], 3)
    xs = []
    its = []
    with nsamg.setup_hierarchy(H, nsamg.default_params(smoother=K.HYBRID_ILU0)) as h:
        for f in (1.0, scale):
            x = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
            st = nsamg.solve(h, dev(b * f), x, rtol=1e-8, maxit=500)
            assert st["converged"] == 1
            xs.append(host(x) / f)
            its.append(st["iters"])
    assert its[0] == its[1]
    assert np.linalg.norm(xs[1] - xs[0]) <= 1e-10 * np.linalg.norm(xs[0])


def test_gram_and_update_with_zero_rows():
    """Exact zeros (a block of zero rows in every vector) split to (0, 0) and add nothing."""
    _gram_update_case(40000, 9, 0, zero_rows=5000)
    _gram_update_case(40000, 9, 1, zero_rows=5000)
    _gram_update_case(40000, 9, 0, zero_rows=5000, aligned=True)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("smoother", [K.POLY_GS, K.HYBRID_ILU0, K.JACOBI_L1])
@pytest.mark.parametrize("graph,krylov_fp64", [(1, 0), (0, 0), (1, 1)])
def test_solve_matches_oracle(name, smoother, graph, krylov_fp64):
    A, H = case(name)
    m = 30
    p = nsamg.default_params(**params_for(smoother), restart=m, use_graph=graph, krylov_fp64=krylov_fp64,
                             spmv_group=-1 if name == "p30" else 0)
    op = oracle_params(p)
    b = rhs_uniform(A.shape[0], 0)
    ref = gmres_onereduce(A, b, lambda v: ovcycle(H, v, op), m=m, rtol=1e-8)
    ref_mgs = gmres_mgs(A, b, lambda v: ovcycle(H, v, op), m=m, rtol=1e-8)
    with nsamg.setup_hierarchy(H, p) as h:
        x = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
        st = nsamg.solve(h, dev(b), x, rtol=1e-8, maxit=500)
        xs = host(x)
    true = np.linalg.norm(b - A @ xs) / np.linalg.norm(b)
    assert st["converged"] == 1 and st["status"] == 0
    assert true <= 1e-8 and abs(true - st["relres_true"]) <= 1e-12
    assert abs(st["iters"] - ref.iters) <= 1 and abs(st["iters"] - ref_mgs.iters) <= 1
    assert np.linalg.norm(xs - ref.x) / np.linalg.norm(ref.x) <= 1e-6


@pytest.mark.parametrize("krylov_fp64", [0, 1])
def test_solve_restarts_and_texact(krylov_fp64):
    A, H = case("c1")
    b = rhs_uniform(A.shape[0], 4)
    for t_exact in (0, 1):
        p = nsamg.default_params(restart=4, t_exact=t_exact, krylov_fp64=krylov_fp64)
        op = oracle_params(p)
        ref = gmres_onereduce(A, b, lambda v: ovcycle(H, v, op), m=4, rtol=1e-9,
                              T_mode="exact" if t_exact else "trunc")
        with nsamg.setup_hierarchy(H, p) as h:
            x = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
            st = nsamg.solve(h, dev(b), x, rtol=1e-9, maxit=500)
        assert st["converged"] and st["restarts"] >= 1
        assert abs(st["iters"] - ref.iters) <= 1
        assert np.linalg.norm(host(x) - ref.x) / np.linalg.norm(ref.x) <= 1e-6


@pytest.mark.parametrize("m", [6, 30])
@pytest.mark.parametrize("graph", [1, 0])
def test_solve_stops_on_backward_error(m, graph):
    """stop_nrbe = 1: the solve stops on beta(x) = ||r|| / (||b|| + ||A||_inf ||x||) <= rtol (Sec. 3)
    like the oracle's one-reduce GMRES with the same stop; with restarts (m = 6) it needs fewer
    steps than the relative-residual stop."""
    A, H = case("c1")
    b = rhs_uniform(A.shape[0], 0)
    p = nsamg.default_params(restart=m, stop_nrbe=1, use_graph=graph)
    ref = gmres_onereduce(A, b, lambda v: ovcycle(H, v, oracle_params(p)), m=m, rtol=1e-8, stop="nrbe")
    with nsamg.setup_hierarchy(H, p) as h:
        x = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
        st = nsamg.solve(h, dev(b), x, rtol=1e-8, maxit=500)
        xs = host(x)
    with nsamg.setup_hierarchy(H, nsamg.default_params(restart=m, use_graph=graph)) as h:
        x = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
        st_rel = nsamg.solve(h, dev(b), x, rtol=1e-8, maxit=500)
    Ad = A.toarray()
    beta = np.linalg.norm(b - Ad @ xs) / (np.linalg.norm(b) + np.abs(Ad).sum(axis=1).max() * np.linalg.norm(xs))
    assert st["converged"] == 1 and beta <= 1e-8 and st["nrbe"] == pytest.approx(beta, rel=1e-6)
    assert abs(st["iters"] - ref.iters) <= 1
    assert np.linalg.norm(xs - ref.x) / np.linalg.norm(ref.x) <= 1e-6
    assert st["iters"] <= st_rel["iters"]
    if m == 6:
        assert st["iters"] < st_rel["iters"]


def test_solve_edge_cases():
    A, H = case("p23")
    n = A.shape[0]
    b = rhs_uniform(n, 2)
    with nsamg.setup_hierarchy(H, nsamg.default_params()) as h:
        # maxit = 0: no iteration, NOT_CONVERGED, x unchanged
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        st = nsamg.solve(h, dev(b), x, rtol=1e-8, maxit=0)
        assert st["status"] == nsamg.NOT_CONVERGED and st["iters"] == 0 and float(x.abs().max()) == 0.0
        # starting from the solution: zero iterations
        xs = np.linalg.solve(A.toarray(), b)
        x = dev(xs)
        st = nsamg.solve(h, dev(b), x, rtol=1e-8, maxit=100)
        assert st["converged"] and st["iters"] == 0
        # b = 0 with x0 = 0: converged at once, x stays 0
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        st = nsamg.solve(h, torch.zeros(n, dtype=torch.float64, device="cuda"), x, rtol=1e-8, maxit=100)
        assert st["converged"] and st["iters"] == 0
        # NaN in b: reported, not hidden
        bn = b.copy()
        bn[5] = np.nan
        with pytest.raises(nsamg.NsamgError) as ei:
            nsamg.solve(h, dev(bn), torch.zeros(n, dtype=torch.float64, device="cuda"), rtol=1e-8, maxit=100)
        assert ei.value.status == -6
        # the handle still works afterwards
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        st = nsamg.solve(h, dev(b), x, rtol=1e-8, maxit=500)
        assert st["converged"]
        # host-buffer entry point gives the same x
        xh = np.zeros(n)
        st2 = nsamg.solve_host(h, b, xh, rtol=1e-8, maxit=500)
        assert st2["iters"] == st["iters"] and np.array_equal(xh, host(x))


def test_solve_is_deterministic():
    A, H = case("p23")
    b = rhs_uniform(A.shape[0], 9)
    with nsamg.setup_hierarchy(H, nsamg.default_params(smoother=K.HYBRID_ILU0)) as h:
        xs = []
        for _ in range(2):
            x = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
            nsamg.solve(h, dev(b), x, rtol=1e-10, maxit=500)
            xs.append(host(x))
    assert np.array_equal(xs[0], xs[1])


def test_setup_rejects_bad_input():
    A, H = case("c1")
    import copy
    bad = copy.deepcopy(H)
    Ab = bad.levels[0].A.copy()
    Ab.indices[3] = 10_000_000  # column out of range
    bad.levels[0].A = Ab
    with pytest.raises(nsamg.NsamgError) as ei:
        nsamg.setup_hierarchy(bad, nsamg.default_params())
    assert ei.value.status == -2
    with pytest.raises(nsamg.NsamgError) as ei:
        nsamg.setup_hierarchy(H, nsamg.default_params(restart=65))
    assert ei.value.status == -1


# ------------------------------------------------------------------------------------------------
# FP32 V-cycle inside FP64 flexible GMRES (mixed precision). Per-kernel bound from the arithmetic:
# an FP32 product sum over k entries with FP32-rounded inputs errs by at most
# gamma_{k+3} |A||x| with u = 2^-24 (rounding of A, of x, and k accumulations).
# ------------------------------------------------------------------------------------------------
U32 = 2.0 ** -24


def gamma(k):
    return k * U32 / (1 - k * U32)


@pytest.mark.parametrize("name", ["c1", "p23", "p30"])
def test_fp32_level_kernels(name):
    A, H = case(name)
    p = nsamg.default_params(vcycle_fp32=1, spmv_group=-1 if name == "p30" else 0)
    with nsamg.setup_hierarchy(H, p) as h:
        rng = np.random.default_rng(5)
        for l, lev in enumerate(H.levels):
            n = lev.n
            x, b = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
            k = int(np.diff(lev.A.indptr).max())
            bound = gamma(k + 3) * (abs(lev.A) @ np.abs(x))
            y = torch.empty(n, dtype=torch.float64, device="cuda")
            nsamg.level_spmv(h, l, dev(x), y)
            assert np.all(np.abs(host(y) - K.spmv(lev.A, x)) <= bound)
            r = torch.empty_like(y)
            nsamg.level_residual(h, l, dev(b), dev(x), r)
            assert np.all(np.abs(host(r) - K.residual(lev.A, b, x)) <= bound + gamma(k + 3) * np.abs(b))
            if l < H.nlevels - 1:
                yc = torch.empty(lev.R.shape[0], dtype=torch.float64, device="cuda")
                nsamg.level_restrict(h, l, dev(x), yc)
                kr = int(np.diff(lev.R.indptr).max())
                assert np.all(np.abs(host(yc) - K.restrict(lev.R, x)) <= gamma(kr + 3) * (abs(lev.R) @ np.abs(x)))


@pytest.mark.parametrize("smoother", [K.POLY_GS, K.HYBRID_ILU0, K.JACOBI_L1])
def test_fp32_vcycle_close_to_fp64(smoother):
    """The FP32 V-cycle is the FP64 V-cycle up to FP32 rounding: norm-wise relative difference
    below 1e-4 (a few hundred u across ~10 passes per level and the coarse solve)."""
    A, H = case("p23")
    p = nsamg.default_params(vcycle_fp32=1, **params_for(smoother))
    with nsamg.setup_hierarchy(H, p) as h:
        r = rhs_uniform(A.shape[0], 11)
        z = torch.empty(A.shape[0], dtype=torch.float64, device="cuda")
        nsamg.apply_vcycle(h, dev(r), z)
        want = ovcycle(H, r, oracle_params(p))
        got = host(z)
    assert np.linalg.norm(got - want) <= 1e-4 * np.linalg.norm(want)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("smoother", [K.POLY_GS, K.HYBRID_ILU0, K.JACOBI_L1])
def test_fp32_vcycle_solve(name, smoother):
    """Mixed precision: FP32 V-cycle in FP64 flexible GMRES reaches relative residual 1e-8 in
    FP64, with iterations within +-1 of the FP64 oracle; solved to 1e-12 both ways, x agrees
    with the FP64 oracle to 1e-6 relative."""
    A, H = case(name)
    p = nsamg.default_params(vcycle_fp32=1, restart=30, **params_for(smoother))
    op = oracle_params(p)
    b = rhs_uniform(A.shape[0], 0)
    ref = gmres_onereduce(A, b, lambda v: ovcycle(H, v, op), m=30, rtol=1e-8)
    with nsamg.setup_hierarchy(H, p) as h:
        x = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
        st = nsamg.solve(h, dev(b), x, rtol=1e-8, maxit=500)
        xs = host(x)
        assert st["converged"] and np.linalg.norm(b - A @ xs) / np.linalg.norm(b) <= 1e-8
        assert abs(st["iters"] - ref.iters) <= 1
        x2 = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
        st2 = nsamg.solve(h, dev(b), x2, rtol=1e-12, maxit=500)
    ref2 = gmres_onereduce(A, b, lambda v: ovcycle(H, v, op), m=30, rtol=1e-12)
    assert st2["converged"]
    assert np.linalg.norm(host(x2) - ref2.x) / np.linalg.norm(ref2.x) <= 1e-6


def test_c3_type_graded_27pt_fp32_vcycle():
    """Graded 27-point Q1 system (C3 structure at 20^3): l1-Jacobi V-cycle in FP32 inside FP64
    flexible GMRES reaches 1e-8 with iterations within +-1 of the FP64 oracle; at 1e-12 the
    solution agrees with the oracle's to 1e-6."""
    from workloads.matrices import q1_27pt_graded
    A = q1_27pt_graded(20, aspect=100.0, seed=1)
    H = build_hierarchy(A, ilu_levels=(), coarse_max=64)
    p = nsamg.default_params(smoother=K.JACOBI_L1, pre_sweeps=2, post_sweeps=2, restart=30, vcycle_fp32=1)
    op = oracle_params(p)
    b = rhs_uniform(A.shape[0], 3)
    ref = gmres_onereduce(A, b, lambda v: ovcycle(H, v, op), m=30, rtol=1e-8, maxit=500)
    with nsamg.setup_hierarchy(H, p) as h:
        x = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
        st = nsamg.solve(h, dev(b), x, rtol=1e-8, maxit=500)
        xs = host(x)
        assert st["converged"] and np.linalg.norm(b - A @ xs) / np.linalg.norm(b) <= 1e-8
        assert abs(st["iters"] - ref.iters) <= 1, (st["iters"], ref.iters)
        x2 = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
        nsamg.solve(h, dev(b), x2, rtol=1e-12, maxit=1000)
    ref2 = gmres_onereduce(A, b, lambda v: ovcycle(H, v, op), m=30, rtol=1e-12, maxit=1000)
    assert np.linalg.norm(host(x2) - ref2.x) / np.linalg.norm(ref2.x) <= 1e-6


@pytest.mark.parametrize("name", ["c1", "p23"])
@pytest.mark.parametrize("krylov_fp64", [1, 0])
def test_backward_error_and_orthogonality_diagnostics(name, krylov_fp64):
    """NRBE (Sec. 3: ||r|| / (||b|| + ||A||_inf ||x||)) matches the value computed from the
    returned x on the host; the loss of orthogonality of the last cycle is O(eps * kappa(B))
    (Sec. 3), with eps the precision of the basis inner products: FP64 (then also the same size
    as the oracle's loss) or double-FP32 (eps ~ 2^-45: the bound, not the oracle's value)."""
    A, H = case(name)
    b = rhs_uniform(A.shape[0], 0)
    with nsamg.setup_hierarchy(H, nsamg.default_params(krylov_fp64=krylov_fp64)) as h:
        x = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
        st = nsamg.solve(h, dev(b), x, rtol=1e-8, maxit=500)
        xs = host(x)
    r = b - A @ xs
    nrbe = np.linalg.norm(r) / (np.linalg.norm(b) + abs(A).sum(axis=1).max() * np.linalg.norm(xs))
    assert st["nrbe"] == pytest.approx(nrbe, rel=1e-6)
    eps = np.finfo(float).eps if krylov_fp64 else 2.0 ** -45
    assert 0.0 < st["orth_loss"] <= 1e3 * eps / st["relres_implicit"]
    from oracle.gmres import sk_norm
    lf = st["orth_loss"] / np.sqrt(2.0)
    assert 0.0 < st["sk_norm"] <= lf / (1.0 - lf) * (1 + 1e-12)
    if krylov_fp64:
        ref = gmres_onereduce(A, b, lambda v: ovcycle(H, v, K.SmootherParams()), m=30, rtol=1e-8)
        ref_loss = np.sqrt(2.0) * np.linalg.norm(ref.L)
        assert st["orth_loss"] == pytest.approx(ref_loss, rel=0.5, abs=1e-15)
        # ||S_k||_2 of the same cycle: the same order as the oracle's
        assert st["sk_norm"] == pytest.approx(sk_norm(ref.L), rel=0.5, abs=1e-15)


@pytest.mark.parametrize("k", [1, 2, 7, 33, 64])
@pytest.mark.parametrize("kind", ["random", "orthonormal", "dependent"])
def test_sknorm_kernel_matches_oracle(k, kind):
    """nsamg_sknorm on caller data against the oracle's definition (dense solve + 2-norm)."""
    from oracle.gmres import sk_norm
    rng = np.random.default_rng(100 + k)
    n = 300
    W = rng.standard_normal((n, k))
    if kind == "orthonormal":
        W = np.linalg.qr(W)[0]
    elif kind == "dependent" and k >= 3:
        W[:, -1] = W[:, :2] @ rng.standard_normal(2)
    W /= np.linalg.norm(W, axis=0)
    ld = 65
    Lh = np.zeros((k, ld))
    Lh[:, :k] = np.tril(W.T @ W, -1)
    Lh[:, k:] = 7.0  # beyond the k x k block: must be ignored
    Lh[np.arange(k), np.arange(k)] = 3.0  # diagonal: ignored too
    got = nsamg.sknorm(dev(Lh), k)
    want = sk_norm(np.tril(W.T @ W, -1))
    assert got == pytest.approx(want, rel=1e-10, abs=1e-14)
    if kind == "dependent" and k >= 3:
        assert got == pytest.approx(1.0, abs=1e-8)


def test_checkpoint_and_resume():
    """A stopped solve is resumed by calling solve again from the saved x (x and the true residual
    fully define the state at a restart): the resumed run reaches the tolerance, and a run that
    restarts at the same column count gives the same x."""
    A, H = case("p23")
    b = rhs_uniform(A.shape[0], 21)
    with nsamg.setup_hierarchy(H, nsamg.default_params(restart=5)) as h:
        x = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
        st1 = nsamg.solve(h, dev(b), x, rtol=1e-10, maxit=5)
        assert st1["status"] == nsamg.NOT_CONVERGED and st1["iters"] == 5
        saved = host(x).copy()
        x2 = dev(saved)
        st2 = nsamg.solve(h, dev(b), x2, rtol=1e-10, maxit=500)
        assert st2["converged"]
        x3 = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
        st3 = nsamg.solve(h, dev(b), x3, rtol=1e-10, maxit=500)
    assert st3["iters"] == st1["iters"] + st2["iters"]
    assert np.array_equal(host(x2), host(x3))


@pytest.mark.parametrize("sweeps", [0, 1, 3, 8])
def test_ilu0_fixed_point_on_gpu(sweeps):
    """GPU fixed-point ILU(0) sweeps equal the oracle's sweeps on the same pattern."""
    A = pressure3d_7pt(20, seed=11)
    got = nsamg.ilu0_fixed_point(A, sweeps)
    Ls, U = K.ilu0_fixed_point(A, sweeps)
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    want = np.asarray((Ls + U)[rows, A.indices]).ravel()
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def test_solve_with_gpu_computed_ilu0_factors():
    """Hierarchy whose finest ILU(0) factors come from 30 GPU fixed-point sweeps: the hybrid
    V-cycle solve converges like the one with host-computed factors."""
    import copy
    A, H = case("p23")
    vals = nsamg.ilu0_fixed_point(H.levels[0].A, 30)
    A0 = H.levels[0].A
    rows = np.repeat(np.arange(A0.shape[0]), np.diff(A0.indptr))
    lower = rows > A0.indices
    Lm = sp.csr_matrix((np.where(lower, vals, 0.0), A0.indices.copy(), A0.indptr.copy()), shape=A0.shape)
    Um = sp.csr_matrix((np.where(lower, 0.0, vals), A0.indices.copy(), A0.indptr.copy()), shape=A0.shape)
    Lm.eliminate_zeros()
    Um.eliminate_zeros()
    d = Um.diagonal()
    H2 = copy.copy(H)
    H2.levels = [copy.copy(l) for l in H.levels]
    H2.levels[0].ilu_L = sp.csr_matrix(Lm)
    H2.levels[0].ilu_U = sp.csr_matrix(sp.diags(1.0 / d) @ sp.triu(Um, 1))
    H2.levels[0].ilu_dinv = 1.0 / d
    np.testing.assert_allclose(H2.levels[0].ilu_dinv, H.levels[0].ilu_dinv, rtol=1e-10)
    b = rhs_uniform(A.shape[0], 5)
    p = nsamg.default_params(smoother=K.HYBRID_ILU0)
    with nsamg.setup_hierarchy(H2, p) as h2, nsamg.setup_hierarchy(H, p) as h1:
        x1 = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
        x2 = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
        s1 = nsamg.solve(h1, dev(b), x1, rtol=1e-8)
        s2 = nsamg.solve(h2, dev(b), x2, rtol=1e-8)
    assert s2["converged"] and abs(s1["iters"] - s2["iters"]) <= 1


@pytest.mark.parametrize("name", ["c1", "p23", "p20s", "p30"])
@pytest.mark.parametrize("smoother", [K.POLY_GS, K.JACOBI_L1, K.ILU0, K.HYBRID_ILU0])
@pytest.mark.parametrize("fp32", [0, 1])
def test_fused_tail_equals_separate_launches(name, smoother, fp32):
    """The V-cycle below the first level with <= 8192 rows run as one cluster kernel gives bitwise
    the same z = M^-1 r as one launch per pass, with fewer launches per Arnoldi step. The layouts
    are fixed (spmv_group = -1) so that the timed autotuner cannot pick different kernels for the
    two handles."""
    A, H = case(name)
    r = np.random.default_rng(7).uniform(-1, 1, A.shape[0])
    outs, launches = [], []
    for fuse in (0, 1, 2):
        p = nsamg.default_params(**params_for(smoother, vcycle_fp32=fp32, fuse_tail=fuse, spmv_group=-1))
        with nsamg.setup_hierarchy(H, p) as h:
            z = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
            nsamg.apply_vcycle(h, dev(r), z)
            outs.append(host(z))
            launches.append(nsamg.launches_per_step(h))
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    assert launches[1] < launches[0] and launches[2] < launches[0]


@pytest.mark.parametrize("fp32", [0, 1])
def test_fused_tail_solve_is_bitwise_unchanged(fp32):
    A, H = case("p23")
    b = rhs_uniform(A.shape[0], 4)
    res = []
    for fuse in (0, 1, 2):
        p = nsamg.default_params(smoother=nsamg.HYBRID_ILU0, vcycle_fp32=fp32, fuse_tail=fuse, spmv_group=-1)
        with nsamg.setup_hierarchy(H, p) as h:
            x = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
            st = nsamg.solve(h, dev(b), x, rtol=1e-8, maxit=300)
            assert st["status"] == 0
            res.append((st["iters"], host(x)))
    for k in (1, 2):
        assert res[0][0] == res[k][0] and np.array_equal(res[0][1], res[k][1])


def test_grid_barrier_completes_every_round():
    """The grid tail's barrier: one block per SM, 7 rounds, every block passes every round."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    passed, status = nsamg.grid_barrier_test(7)
    assert (passed, status) == (7 * sms, 0)


def test_grid_barrier_wait_runs_out_and_the_context_survives():
    """A barrier that waits for an arrival nothing makes: every block gives up after its poll limit
    (a few ms here), the kernel returns NSAMG_ERR_TIMEOUT instead of hanging, and the context then
    runs a solve as usual."""
    passed, status = nsamg.grid_barrier_test(3, missing=1, spin_limit=20000)
    assert passed == 0 and status == nsamg.ERR_TIMEOUT
    A, H = case("p23")
    b = rhs_uniform(A.shape[0], 4)
    with nsamg.setup_hierarchy(H, nsamg.default_params(fuse_tail=2)) as h:
        x = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
        st = nsamg.solve(h, dev(b), x, rtol=1e-8, maxit=300)
    assert st["status"] == 0 and st["converged"] == 1


def test_fp32_vcycle_on_unaligned_caller_arrays():
    """The FP64 <-> FP32 casts take four elements per access only when both arrays are 16-byte
    aligned; caller arrays at an odd element offset give the same z through the scalar path."""
    A, H = case("p23")
    n = A.shape[0]
    r = np.random.default_rng(3).uniform(-1, 1, n)
    with nsamg.setup_hierarchy(H, nsamg.default_params(vcycle_fp32=1, spmv_group=-1)) as h:
        z = torch.zeros(n, dtype=torch.float64, device="cuda")
        nsamg.apply_vcycle(h, dev(r), z)
        big_r = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
        big_r[1:] = dev(r)
        big_z = torch.zeros(n + 1, dtype=torch.float64, device="cuda")
        nsamg.apply_vcycle(h, big_r[1:], big_z[1:])
        assert np.array_equal(host(z), host(big_z)[1:])


def test_fp32_casts_round_to_nearest_even():
    """The FP64 -> FP32 -> FP64 casts of FP32-V-cycle handles (integer forms) against IEEE 754
    conversion (numpy): a one-level FP32 handle whose operator is the identity returns
    double(float(x)). Covers the whole exponent range, exact ties (to even), values beside them,
    the binary32 overflow boundary (FLT_MAX + half an ulp rounds to infinity), the normal/subnormal
    boundary, zeros, infinities and NaN."""
    from workloads.hierarchy import Hierarchy, Level
    rng = np.random.default_rng(17)
    f = (rng.uniform(1, 2, 4000) * 2.0 ** rng.integers(-126, 128, 4000)).astype(np.float32)
    f *= np.where(rng.random(4000) < 0.5, -1, 1).astype(np.float32)
    ulp = np.spacing(np.abs(f)).astype(np.float64)
    ties = f.astype(np.float64) + np.sign(f) * ulp / 2
    vals = np.concatenate([
        rng.uniform(-1, 1, 4000) * 2.0 ** rng.integers(-160, 160, 4000),
        ties, np.nextafter(ties, np.inf), np.nextafter(ties, -np.inf),
        [3.4028234663852886e38, 3.4028234663852886e38 * (1 + 2.0 ** -25), 3.4028235677973366e38,
         np.nextafter(3.4028235677973366e38, 0), 1.1754943508222875e-38, 1.1754942e-38, 1.4e-45, 7e-46,
         1e-40, -1e-40, 0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, -1.0, 2.0 ** 24 + 1, 16777217.0],
    ])
    n = vals.size
    I = sp.identity(n, format="csr")
    I.indices = I.indices.astype(np.int32)
    I.indptr = I.indptr.astype(np.int32)
    H = Hierarchy(levels=[Level(A=I)], coarse_inv=None)
    with nsamg.setup_hierarchy(H, nsamg.default_params(vcycle_fp32=1)) as h:
        y = torch.empty(n, dtype=torch.float64, device="cuda")
        nsamg.level_spmv(h, 0, dev(vals), y)
        got = host(y)
    with np.errstate(over="ignore"):
        want = vals.astype(np.float32).astype(np.float64)
    np.testing.assert_array_equal(got, want)


_rank_cache = {}


def ranked_case(ranks):
    """p23 with the ILU factors of every level taken from the block diagonal over `ranks` row
    blocks (the local matrices of a `ranks`-rank run)."""
    if ranks not in _rank_cache:
        A, kw = CASES["p23"]()
        _rank_cache[ranks] = (A, build_hierarchy(A, ilu_levels=None, ranks=ranks, **kw))
    return _rank_cache[ranks]


@pytest.mark.parametrize("ranks", [2, 5, 64])
@pytest.mark.parametrize("smoother", [K.POLY_GS, K.HYBRID_ILU0, K.ILU0])
def test_vcycle_with_emulated_ranks(ranks, smoother):
    """Hybrid block-Jacobi smoothing of a multi-rank run (Sec. 5.2) computed on one GPU: the
    V-cycle against the oracle's with the same row blocks, componentwise."""
    A, H = ranked_case(ranks)
    p = nsamg.default_params(**params_for(smoother), ranks=ranks)
    with nsamg.setup_hierarchy(H, p) as h:
        r = rhs_uniform(A.shape[0], 12)
        z = torch.empty(A.shape[0], dtype=torch.float64, device="cuda")
        nsamg.apply_vcycle(h, dev(r), z)
    want = ovcycle(H, r, oracle_params(p))
    assert np.max(np.abs(host(z) - want)) <= 1e-11 * np.max(np.abs(want))
    if smoother == K.ILU0:  # ILU on every smoothed level: the blocks live in the factors alone
        return
    # the blocks change the polynomial Gauss-Seidel levels: the same V-cycle without them differs
    with nsamg.setup_hierarchy(H, nsamg.default_params(**params_for(smoother))) as h1:
        z1 = torch.empty(A.shape[0], dtype=torch.float64, device="cuda")
        nsamg.apply_vcycle(h1, dev(r), z1)
    assert np.max(np.abs(host(z1) - want)) > 1e-6 * np.max(np.abs(want))


@pytest.mark.parametrize("ranks", [1, 4, 16])
def test_solve_with_emulated_ranks_matches_oracle(ranks):
    """GMRES with the hybrid V-cycle of a `ranks`-rank run: iterations and solution as the FP64
    oracle with the same blocks; more ranks never take fewer iterations here."""
    A, H = ranked_case(ranks) if ranks > 1 else case("p23")
    p = nsamg.default_params(smoother=K.HYBRID_ILU0, restart=30, ranks=ranks)
    b = rhs_uniform(A.shape[0], 13)
    ref = gmres_onereduce(A, b, lambda v: ovcycle(H, v, oracle_params(p)), m=30, rtol=1e-8)
    with nsamg.setup_hierarchy(H, p) as h:
        x = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
        st = nsamg.solve(h, dev(b), x, rtol=1e-8, maxit=500)
    assert st["converged"] == 1 and abs(st["iters"] - ref.iters) <= 1
    assert np.linalg.norm(host(x) - ref.x) <= 1e-6 * np.linalg.norm(ref.x)
