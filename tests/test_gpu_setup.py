"""GPU Ruge-Stuben setup (nsamg_amg_build) against the setup oracle, level by level: strength
flags and the PMIS splitting bit-exact, interpolation weights and Galerkin products within
1e-14 relative (the products are summed in the same order as a sequential row-by-row product, so
they also equal the host input generator's bitwise), fixed-point ILU(0) factors and the coarse
inverse within their rounding bounds; a solve on the GPU-built hierarchy converges."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle.setup as OS
from workloads import build_hierarchy, pressure3d_7pt, q1_27pt_graded, rhs_uniform

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2112_14681_b300 import nsamg  # noqa: E402


def zero_rowsum(n, seed, density=0.01):
    rng = np.random.default_rng(seed)
    B = sp.random(n, n, density=density, random_state=rng, format="csr")
    B.data = -np.where(rng.random(B.nnz) < 0.3, rng.uniform(0.01, 0.05, B.nnz), rng.uniform(0.5, 1.0, B.nnz))
    B.setdiag(0.0)
    B.eliminate_zeros()
    chain = sp.diags([-np.ones(n - 1), -np.ones(n - 1)], [-1, 1], format="csr")
    B = sp.csr_matrix(B + chain)
    A = sp.csr_matrix(B - sp.diags(np.asarray(B.sum(axis=1)).ravel()) + 1e-3 * sp.eye(n))
    A.sort_indices()
    return A


CASES = {
    # 3D variable-coefficient 7-point, ragged size (7^3 * 8 + ...): several levels
    "p21": lambda: (pressure3d_7pt(21, seed=4), dict(coarse_max=100, seed=3), "abs"),
    # Q1 27-point graded stiffness, sign-aware strength: rows of 100+ entries on level 1
    "q12": lambda: (q1_27pt_graded(12), dict(coarse_max=100, seed=1, strength_mode=1), "neg"),
    # random nonsymmetric with weak couplings
    "z3000": lambda: (zero_rowsum(3000, 2), dict(coarse_max=50, seed=9), "abs"),
}
_built = {}


def built(name):
    if name not in _built:
        A, kw, mode = CASES[name]()
        A = sp.csr_matrix(A)
        A.sort_indices()
        opt = nsamg.amg_default_options(ilu_levels=0b11, ilu_sweeps=4, direct_max=512, **kw)
        g = nsamg.amg_build(A, opt)
        _built[name] = (A, kw, mode, g, g.export())
    return _built[name]


def rel_close(got, want, rtol):
    scale = max(np.max(np.abs(want)), 1e-300)
    return np.max(np.abs(got - want)) <= rtol * scale


@pytest.mark.parametrize("name", list(CASES))
def test_levels_match_the_oracle(name):
    A, kw, mode, g, H = built(name)
    seed = kw["seed"]
    assert H.nlevels >= 3
    for l, lev in enumerate(H.levels[:-1]):
        Al = lev.A
        # strength flags and PMIS splitting: bit-exact (decisions taken in float64 on both sides)
        cf, strong = g.splitting(l)
        s_or = OS.strength(Al, 0.25, mode)
        assert np.array_equal(strong, s_or), l
        cf_or, nc_or = OS.pmis(Al, s_or, seed + 7919 * (l + 1))
        assert np.array_equal(cf, cf_or), l
        assert g.level_info(l)["nc"] == nc_or == lev.P.shape[1]
        # interpolation: same pattern, weights within rounding of the closed form
        P_or = OS.bamg_direct(Al, s_or, cf_or, nc_or)
        assert np.array_equal(lev.P.indptr, P_or.indptr) and np.array_equal(lev.P.indices, P_or.indices)
        assert rel_close(lev.P.data, P_or.data, 1e-14)
        # restriction is the exact transpose; the Galerkin product within 1e-14 of scipy's
        R_or, Ac_or = OS.galerkin(Al, lev.P)
        assert np.array_equal(lev.R.indptr, R_or.indptr) and np.array_equal(lev.R.indices, R_or.indices)
        assert np.array_equal(lev.R.data, R_or.data)
        Ac = H.levels[l + 1].A
        assert abs(Ac - Ac_or).max() <= 1e-14 * abs(Ac_or).max(), l
        # the GPU keeps entries that cancel to zero, scipy may drop them: never fewer entries
        assert Ac.nnz >= Ac_or.nnz


@pytest.mark.parametrize("name", list(CASES))
def test_ilu_factors_and_coarse_inverse(name):
    A, kw, mode, g, H = built(name)
    for l in (0, 1):
        lev = H.levels[l]
        Ls, Us, dinv = OS.ilu0_factors(lev.A, 4)
        assert np.array_equal(lev.ilu_L.indptr, Ls.indptr) and np.array_equal(lev.ilu_L.indices, Ls.indices)
        assert np.array_equal(lev.ilu_U.indptr, Us.indptr) and np.array_equal(lev.ilu_U.indices, Us.indices)
        assert rel_close(lev.ilu_L.data, Ls.data, 1e-12) and rel_close(lev.ilu_U.data, Us.data, 1e-12)
        assert rel_close(lev.ilu_dinv, dinv, 1e-12)
    assert H.levels[2].ilu_L is None
    Ac = H.levels[-1].A
    want = OS.coarse_inverse(Ac)
    cond = np.linalg.cond(Ac.toarray())
    assert np.max(np.abs(H.coarse_inv - want)) <= 64 * np.finfo(float).eps * cond * np.max(np.abs(want))


def test_gpu_setup_equals_the_host_generator_bitwise():
    """Same splitting, same P, and the same coarse operators bit for bit as the C++ host setup
    (both sum each product entry in the order of the left operand's row, without fused
    multiply-adds)."""
    A = pressure3d_7pt(24, seed=7)
    Hh = build_hierarchy(A, theta=0.25, coarse_max=100, seed=5, ilu_levels=())
    with nsamg.amg_build(A, nsamg.amg_default_options(coarse_max=100, seed=5, ilu_levels=0)) as g:
        H = g.export()
    assert H.nlevels == Hh.nlevels
    for a, b in zip(H.levels, Hh.levels):
        assert np.array_equal(a.A.indptr, b.A.indptr) and np.array_equal(a.A.indices, b.A.indices)
        assert np.array_equal(a.A.data, b.A.data)
        if b.P is not None:
            assert np.array_equal(a.P.indices, b.P.indices) and np.array_equal(a.P.data, b.P.data)


def test_solve_on_the_gpu_built_hierarchy():
    A = pressure3d_7pt(32, seed=2)
    b = rhs_uniform(A.shape[0], 3)
    p = nsamg.default_params(smoother=nsamg.HYBRID_ILU0)
    with nsamg.amg_build(A, nsamg.amg_default_options(coarse_max=512, ilu_sweeps=3)) as g:
        h = g.setup_solver(p)
    x = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
    st = nsamg.solve(h, torch.from_numpy(b).cuda(), x, rtol=1e-8, maxit=300)
    torch.cuda.synchronize()
    assert st["converged"]
    xh = x.cpu().numpy()
    assert np.linalg.norm(b - A @ xh) / np.linalg.norm(b) <= 1e-8
    Hh = build_hierarchy(A, theta=0.25, coarse_max=512, seed=0, ilu_levels=(0,))
    with nsamg.setup_hierarchy(Hh, p) as h2:
        x2 = torch.zeros_like(x)
        st2 = nsamg.solve(h2, torch.from_numpy(b).cuda(), x2, rtol=1e-8, maxit=300)
    assert abs(st["iters"] - st2["iters"]) <= 2
    h.close()


def test_bad_inputs():
    with pytest.raises(nsamg.NsamgError) as e:
        nsamg.amg_build(pressure3d_7pt(6), nsamg.amg_default_options(theta=2.0))
    assert e.value.status == -1
    # exactly singular coarsest operator (no coarsening: 2 rows <= coarse_max)
    S = sp.csr_matrix(np.ones((2, 2)))
    with pytest.raises(nsamg.NsamgError) as e:
        nsamg.amg_build(S, nsamg.amg_default_options())
    assert e.value.status == -2
    # missing diagonal: rejected before any upload
    B = sp.csr_matrix(np.array([[0.0, 1.0], [1.0, 2.0]]))
    B.eliminate_zeros()
    with pytest.raises(nsamg.NsamgError) as e:
        nsamg.amg_build(B, nsamg.amg_default_options())
    assert e.value.status == -2


def test_no_coarsening_when_small():
    A = pressure3d_7pt(6, seed=1)
    with nsamg.amg_build(A, nsamg.amg_default_options(coarse_max=1000)) as g:
        H = g.export()
        assert H.nlevels == 1 and H.levels[0].P is None
        assert np.allclose(H.coarse_inv @ A.toarray(), np.eye(A.shape[0]), atol=1e-10)


@pytest.mark.parametrize("name", ["p21", "z3000"])
def test_mm_ext_levels_match_the_oracle(name):
    """MM-ext interpolation (Sec. 5.1) on every level against the oracle's matrix formula; the
    Galerkin products of the MM-ext hierarchy as before."""
    A, kw, mode, _, _ = built(name)
    opt = nsamg.amg_default_options(ilu_levels=0, direct_max=512, interp=1, **kw)
    with nsamg.amg_build(A, opt) as g:
        H = g.export()
        splits = [g.splitting(l) for l in range(H.nlevels - 1)]
    assert H.nlevels >= 3
    for l, lev in enumerate(H.levels[:-1]):
        cf, strong = splits[l]
        s_or = OS.strength(lev.A, 0.25, mode)
        assert np.array_equal(strong, s_or)
        cf_or, nc = OS.pmis(lev.A, s_or, kw["seed"] + 7919 * (l + 1))
        assert np.array_equal(cf, cf_or)
        P_or = OS.mm_ext(lev.A, s_or, cf_or, nc)
        # each weight is a sum of up to k = (row length of A) products of mixed sign, summed in
        # another order by the oracle: |difference| <= 2 k eps max|P| (rounding of both sides)
        k = int(np.diff(lev.A.indptr).max())
        assert abs(lev.P - P_or).max() <= 2 * k * np.finfo(float).eps * abs(P_or).max(), l
        assert lev.P.nnz >= P_or.nnz
        _, Ac_or = OS.galerkin(lev.A, lev.P)
        # componentwise: |difference| <= 2 k eps (|R| |A| |P|), k the longest chain of products
        R = sp.csr_matrix(lev.P.T)
        bound = (abs(R) @ abs(lev.A) @ abs(lev.P)).toarray()
        kk = int(np.diff(R.indptr).max() + np.diff(lev.A.indptr).max() + np.diff(lev.P.indptr).max())
        D = abs(H.levels[l + 1].A - Ac_or).toarray()
        assert np.all(D <= 2 * kk * np.finfo(float).eps * bound), l


def test_solve_on_mm_ext_hierarchy():
    A = pressure3d_7pt(32, seed=2)
    b = rhs_uniform(A.shape[0], 3)
    p = nsamg.default_params(smoother=nsamg.HYBRID_ILU0)
    its = {}
    for interp in (0, 1):
        with nsamg.amg_build(A, nsamg.amg_default_options(coarse_max=512, interp=interp)) as g:
            with g.setup_solver(p) as h:
                x = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
                st = nsamg.solve(h, torch.from_numpy(b).cuda(), x, rtol=1e-8, maxit=300)
                torch.cuda.synchronize()
                assert st["converged"]
                assert np.linalg.norm(b - A @ x.cpu().numpy()) / np.linalg.norm(b) <= 1e-8
                its[interp] = st["iters"]
    assert its[1] <= its[0] + 2


def test_setup_edge_cases():
    # a 1 x 1 operator: no coarsening, the coarse inverse is 1 / a
    one = sp.csr_matrix(np.array([[4.0]]))
    with nsamg.amg_build(one, nsamg.amg_default_options()) as g:
        H = g.export()
        assert H.nlevels == 1 and np.allclose(H.coarse_inv, [[0.25]])
    # max_levels = 1 stops before any coarsening
    A = pressure3d_7pt(10, seed=1)
    with nsamg.amg_build(A, nsamg.amg_default_options(max_levels=1, direct_max=0)) as g:
        assert g.nlevels == 1 and g.export().coarse_inv is None
    # positive couplings only, sign-aware strength: nothing is strong, every point would stay C,
    # so coarsening stops (no level is added)
    B = sp.csr_matrix(sp.diags([np.ones(999), 4 * np.ones(1000), np.ones(999)], [-1, 0, 1]))
    B.sort_indices()
    with nsamg.amg_build(B, nsamg.amg_default_options(strength_mode=1, coarse_max=10, direct_max=0)) as g:
        assert g.nlevels == 1
    # zero fixed-point sweeps: the factors are the initial guess l = a_ij / a_jj, u = a_ij
    with nsamg.amg_build(A, nsamg.amg_default_options(coarse_max=100, ilu_sweeps=0)) as g:
        lev = g.export().levels[0]
        Ls, Us, dinv = OS.ilu0_factors(lev.A, 0)
        assert rel_close(lev.ilu_L.data, Ls.data, 1e-15) and rel_close(lev.ilu_U.data, Us.data, 1e-15)
    # an unknown interpolation choice is rejected
    with pytest.raises(nsamg.NsamgError) as e:
        nsamg.amg_build(A, nsamg.amg_default_options(interp=2))
    assert e.value.status == -1


@pytest.mark.parametrize("smoother", ["hybrid_ilu0", "poly_gs", "jacobi_l1", "ilu0"])
def test_device_built_handle_equals_the_host_built_handle(smoother):
    """nsamg_amg_setup_solver forms D^-1, the l1 diagonal, the scaled triangles, the plain SELL
    copies and the transfers from the device hierarchy with kernels; with the threads per row
    fixed, the solve is bit for bit the one on the same hierarchy exported and set up on the
    host (same arrays, same kernels)."""
    A = pressure3d_7pt(32, seed=2)  # 32768 rows: level 0 gets its plain SELL copies
    b = torch.from_numpy(rhs_uniform(A.shape[0], 3)).cuda()
    sm = {"hybrid_ilu0": nsamg.HYBRID_ILU0, "poly_gs": nsamg.POLY_GS, "jacobi_l1": nsamg.JACOBI_L1,
          "ilu0": nsamg.ILU0}[smoother]
    p = nsamg.default_params(smoother=sm, spmv_group=1)
    with nsamg.amg_build(A, nsamg.amg_default_options(coarse_max=512, ilu_levels=0b111, ilu_sweeps=3)) as g:
        H = g.export()
        xs, sts = [], []
        for make in (lambda: g.setup_solver(p), lambda: nsamg.setup_hierarchy(H, p)):
            with make() as h:
                x = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
                sts.append(nsamg.solve(h, b, x, rtol=1e-8, maxit=300))
                torch.cuda.synchronize()
                xs.append(x.cpu().numpy())
    assert sts[0]["converged"] and sts[0]["iters"] == sts[1]["iters"]
    assert np.array_equal(xs[0], xs[1])
    assert sts[0]["nrbe"] == sts[1]["nrbe"]  # same ||A||_inf


@pytest.mark.parametrize("fp32", [0, 1])
def test_device_built_handle_tuned(fp32):
    """Default (tuned) thread shapes and the FP32 V-cycle: the device-built handle converges to
    the tolerance in the host-built handle's iteration count (+-1: the tuner may pick another
    shape on each handle, which changes rounding only)."""
    A = pressure3d_7pt(32, seed=5)
    bn = rhs_uniform(A.shape[0], 1)
    b = torch.from_numpy(bn).cuda()
    p = nsamg.default_params(smoother=nsamg.HYBRID_ILU0, vcycle_fp32=fp32)
    its = []
    with nsamg.amg_build(A, nsamg.amg_default_options(coarse_max=512)) as g:
        H = g.export()
        for make in (lambda: g.setup_solver(p), lambda: nsamg.setup_hierarchy(H, p)):
            with make() as h:
                x = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
                st = nsamg.solve(h, b, x, rtol=1e-8, maxit=300)
                torch.cuda.synchronize()
                assert st["converged"]
                assert np.linalg.norm(bn - A @ x.cpu().numpy()) / np.linalg.norm(bn) <= 1e-8
                its.append(st["iters"])
    assert abs(its[0] - its[1]) <= 1
