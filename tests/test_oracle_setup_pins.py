"""Pins of the setup oracle (oracle/setup.py, Sec. 5.1) against the mathematics (no GPU needed).

Expected values come from published generator outputs, hand-derived rows, an equivalent
sequential characterisation of PMIS, the constrained least-squares problem of eq. (bamgdir)
solved as a KKT system, dense products and invariants (constants interpolated exactly, zero
row sums kept by the Galerkin product). Planted mistakes at the end check that the pins bite.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle.setup as OS
from workloads import build_hierarchy, poisson2d_5pt, pressure3d_7pt


def lap1d(n):
    return sp.csr_matrix(sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]))


def aniso2d(m, eps):
    T = lap1d(m)
    I = sp.eye(m)
    A = sp.csr_matrix(sp.kron(I, T) + eps * sp.kron(T, I))
    A.sort_indices()
    return A


def zero_rowsum(n, seed, density=0.15, weak_frac=0.3):
    """Random nonsymmetric matrix with negative off-diagonals of mixed strength and a_ii equal to
    minus the off-diagonal row sum (zero row sums)."""
    rng = np.random.default_rng(seed)
    B = sp.random(n, n, density=density, random_state=rng, format="csr")
    B.data = -np.where(rng.random(B.nnz) < weak_frac, rng.uniform(0.01, 0.05, B.nnz), rng.uniform(0.5, 1.0, B.nnz))
    B.setdiag(0.0)
    B.eliminate_zeros()
    # a chain keeps every row connected
    chain = sp.diags([-np.ones(n - 1), -np.ones(n - 1)], [-1, 1], format="csr")
    B = sp.csr_matrix(B + chain)
    A = sp.csr_matrix(B - sp.diags(np.asarray(B.sum(axis=1)).ravel()))
    A.sort_indices()
    return A


# ---- SplitMix64 (the PMIS random numbers) --------------------------------------------------

def _check_splitmix(mod):
    # Published first outputs of SplitMix64 from the state 1234567 (reference implementation).
    st, outs = 1234567, []
    for _ in range(3):
        st, o = mod.splitmix64_next(st)
        outs.append(o)
    assert outs == [6457827717110365317, 3203168211198807973, 9817491932198370423]


def test_splitmix64_published_values():
    _check_splitmix(OS)


def test_pmis_uniforms_are_uniform_and_distinct():
    u = OS.pmis_uniforms(12345, 20000)
    assert u.min() >= 0.0 and u.max() < 1.0 and np.unique(u).size == u.size
    assert abs(u.mean() - 0.5) < 0.01 and abs(u.var() - 1 / 12) < 0.005
    assert not np.array_equal(u, OS.pmis_uniforms(12346, 20000))


# ---- strength of connection (Sec. 5.1) -----------------------------------------------------

def _strength_row():
    # row 0: diag 4, then -1 (the largest), -0.2 (below 0.25), -0.25 (exactly theta * max),
    # +0.5 (positive coupling) and an explicit zero
    A = sp.csr_matrix((np.array([4.0, -1.0, -0.2, -0.25, 0.5, 0.0]), np.array([0, 1, 2, 3, 4, 5]),
                       np.array([0, 6] + [6] * 5)), shape=(6, 6))
    return A


def _check_strength(mod):
    A = _strength_row()
    s_abs = mod.strength(A, 0.25, "abs")
    assert s_abs.tolist() == [False, True, False, True, True, False]
    s_neg = mod.strength(A, 0.25, "neg")
    assert s_neg.tolist() == [False, True, False, True, False, False]
    # only positive off-diagonals: nothing is strong in the sign-aware form
    B = sp.csr_matrix(np.array([[2.0, 1.0], [1.0, 2.0]]))
    assert not mod.strength(B, 0.25, "neg").any()
    assert mod.strength(B, 0.25, "abs").tolist() == [False, True, True, False]


def test_strength_hand_row():
    _check_strength(OS)


# ---- PMIS (Sec. 5.1) -----------------------------------------------------------------------

def pmis_greedy(A, s, seed):
    """Sequential characterisation of PMIS before promotion: visit the points in decreasing
    (lambda_i, i); an undecided point becomes C and every undecided point that strongly depends
    on it becomes F. Points that influence no one are F from the start. With the weights fixed,
    the parallel rounds reach the same splitting (a point is selected exactly when every
    higher-weighted neighbour has been decided)."""
    n = A.shape[0]
    S = OS.strength_matrix(A, s)
    ST = sp.csr_matrix(S.T)
    infl = np.diff(ST.indptr)
    lam = infl + OS.pmis_uniforms(seed, n)
    st = np.where(infl == 0, 2, 0)
    for v in sorted(range(n), key=lambda i: (lam[i], i), reverse=True):
        if st[v] != 0:
            continue
        st[v] = 1
        for i in ST.indices[ST.indptr[v]:ST.indptr[v + 1]]:
            if st[i] == 0:
                st[i] = 2
    return st


def weak_columns(n, seed, frac=0.2):
    """zero_rowsum with a random fifth of the columns made weak in every row: those points
    influence no one and must start as F."""
    A = zero_rowsum(n, seed).tolil()
    rng = np.random.default_rng(seed + 100)
    cols = rng.choice(n, int(frac * n), replace=False)
    A = sp.csr_matrix(A)
    rows = np.repeat(np.arange(n), np.diff(A.indptr))
    hit = np.isin(A.indices, cols) & (A.indices != rows)
    A.data[hit] *= 1e-3
    A = sp.csr_matrix(A - sp.diags(np.asarray(A.sum(axis=1)).ravel()))
    A.sort_indices()
    return A


def _check_pmis(mod):
    cases = [(zero_rowsum(300, 1), 0.25, 11), (weak_columns(300, 3), 0.25, 16), (zero_rowsum(500, 2, density=0.02), 0.25, 12),
             (aniso2d(20, 0.001), 0.25, 13), (sp.csr_matrix(poisson2d_5pt(16)), 0.25, 15), (lap1d(97), 0.25, 14)]
    for A, theta, seed in cases:
        s = mod.strength(A, theta, "abs")
        cf, nc = mod.pmis(A, s, seed, promote=False)
        st = pmis_greedy(A, s, seed)
        assert np.array_equal(cf >= 0, st == 1)
        assert nc == int((st == 1).sum()) and np.array_equal(cf[cf >= 0], np.arange(nc))
        # after promotion every F-point has a strong C-neighbour
        cf2, _ = mod.pmis(A, s, seed)
        S = OS.strength_matrix(A, s)
        for i in np.flatnonzero(cf2 < 0):
            assert np.any(cf2[S.indices[S.indptr[i]:S.indptr[i + 1]]] >= 0), i
        assert np.all(cf2[cf >= 0] >= 0)  # promotion only adds C-points
        # a promoted point influences no one (so the order of promotion cannot matter)
        infl = np.diff(sp.csr_matrix(S.T).indptr)
        assert np.all(infl[(cf2 >= 0) & (cf < 0)] == 0)


def test_pmis_equals_sequential_characterisation():
    _check_pmis(OS)


def test_pmis_on_a_chain_alternates():
    # 1D Laplacian, all couplings strong: no two neighbours are both C before promotion, every
    # F-point is next to a C-point, so between n/3 and n/2 points are C.
    A = lap1d(64)
    s = OS.strength(A, 0.25)
    cf, nc = OS.pmis(A, s, 3, promote=False)
    c = cf >= 0
    assert not np.any(c[1:] & c[:-1])
    left = np.concatenate([[False], c[:-1]])
    right = np.concatenate([c[1:], [False]])
    assert np.all(c | left | right)  # every F-point has a C-neighbour (all couplings strong)
    assert 22 <= nc <= 32


# ---- BAMG-direct interpolation (Sec. 5.1, eq. bamgdir) --------------------------------------

def _bamg_row():
    # row 0: a_00 = 4; strong C-neighbours 1, 2 (-1 each); strong F-neighbour 3 (-1);
    # weak neighbour 4 (-0.2 < 0.25 * 1). Points 1, 2 are C, 0, 3, 4 are F.
    # By hand: denominator 4 - 0.2 = 3.8, beta = -1, n_C = 2,
    # w = -(-1 + (-1)/2) / 3.8 = 1.5 / 3.8 for both C-neighbours.
    A = sp.csr_matrix(np.array([[4.0, -1.0, -1.0, -1.0, -0.2],
                                [-1.0, 2.0, 0, 0, 0], [-1.0, 0, 2.0, 0, 0],
                                [-1.0, -1.0, 0, 2.0, 0], [-1.0, 0, -1.0, 0, 2.0]]))
    cf = np.array([-1, 0, 1, -1, -1])
    return A, cf


def _check_bamg(mod):
    A, cf = _bamg_row()
    s = mod.strength(A, 0.25)
    P = mod.bamg_direct(A, s, cf, 2).toarray()
    assert np.allclose(P[0], [1.5 / 3.8, 1.5 / 3.8], rtol=0, atol=1e-15)
    assert np.array_equal(P[1], [1.0, 0.0]) and np.array_equal(P[2], [0.0, 1.0])
    # zero-row-sum operators: every row of P sums to one (f = 1 interpolated exactly)
    for A in (zero_rowsum(400, 5), zero_rowsum(300, 6, weak_frac=0.0)):
        s = mod.strength(A, 0.25)
        cf, nc = mod.pmis(A, s, 7)
        P = mod.bamg_direct(A, s, cf, nc)
        assert np.allclose(np.asarray(P.sum(axis=1)).ravel(), 1.0, rtol=0, atol=1e-13)
        Pd = P.toarray()
        assert np.array_equal(Pd[cf >= 0], np.eye(nc)[cf[cf >= 0]])
    # no weak couplings and zero row sum: the closed form is the minimiser of
    # || a_ii w + a_{i,C} ||_2 subject to sum(w) = 1, solved here as a KKT system
    A = zero_rowsum(300, 6, weak_frac=0.0)
    s = mod.strength(A, 0.0)  # theta = 0: every nonzero off-diagonal is strong
    cf, nc = mod.pmis(A, s, 8)
    P = mod.bamg_direct(A, s, cf, nc).tocsr()
    checked = 0
    for i in np.flatnonzero(cf < 0)[:40]:
        lo, hi = A.indptr[i], A.indptr[i + 1]
        cols, vals = A.indices[lo:hi], A.data[lo:hi]
        aii = vals[cols == i][0]
        cmask = (cols != i) & (cf[cols] >= 0)
        aC = vals[cmask]
        k = aC.size
        K = np.zeros((k + 1, k + 1))
        K[:k, :k] = aii * aii * np.eye(k)
        K[:k, k] = K[k, :k] = 1.0
        rhs = np.concatenate([-aii * aC, [1.0]])
        w = np.linalg.solve(K, rhs)[:k]
        got = P[i, cf[cols[cmask]]].toarray().ravel()
        assert np.allclose(got, w, rtol=1e-12, atol=1e-14)
        checked += 1
    assert checked >= 20


def test_bamg_direct_pins():
    _check_bamg(OS)


# ---- MM-ext interpolation (Sec. 5.1) --------------------------------------------------------

def _check_mmext(mod):
    for A in (zero_rowsum(300, 5), zero_rowsum(250, 11, density=0.05)):
        s = mod.strength(A, 0.25)
        cf, nc = mod.pmis(A, s, 3)
        P = mod.mm_ext(A, s, cf, nc).toarray()
        # constants interpolated exactly on zero-row-sum operators
        assert np.allclose(P.sum(axis=1), 1.0, rtol=0, atol=1e-13)
        assert np.array_equal(P[cf >= 0], np.eye(nc)[cf[cf >= 0]])
        # element form of the extended weights, derived by hand from the matrix product:
        # w_ij = -(a^s_ij + sum_{k in F^s_i} a_ik a^s_kj / beta_k) / (a_ii + gamma_i), j in C
        n = A.shape[0]
        beta, gamma, strongC, strongF = np.zeros(n), np.zeros(n), {}, {}
        for i in range(n):
            sc, sf = {}, {}
            for p in range(A.indptr[i], A.indptr[i + 1]):
                j, a = A.indices[p], A.data[p]
                if j == i:
                    continue
                if not s[p]:
                    gamma[i] += a
                elif cf[j] >= 0:
                    sc[j] = a
                    beta[i] += a
                else:
                    sf[j] = a
            strongC[i], strongF[i] = sc, sf
        Ad = A.diagonal()
        for i in np.flatnonzero(cf < 0)[:60]:
            w = np.zeros(nc)
            for j, a in strongC[i].items():
                w[cf[j]] += a
            for k, aik in strongF[i].items():
                if beta[k] != 0.0:
                    for j, akj in strongC[k].items():
                        w[cf[j]] += aik * akj / beta[k]
            w = -w / (Ad[i] + gamma[i])
            assert np.allclose(P[i], w, rtol=1e-12, atol=1e-15), i
        # rows without strong F-neighbours reduce to direct interpolation
        P0 = mod.bamg_direct(A, s, cf, nc).toarray()
        rows = [i for i in np.flatnonzero(cf < 0) if not strongF[i]]
        assert np.allclose(P[rows], P0[rows], rtol=1e-12, atol=1e-15)


def test_mm_ext_pins():
    _check_mmext(OS)


# ---- Galerkin product and the coarse inverse (Sec. 5, eq. A_k) ------------------------------

def _check_galerkin(mod):
    A = zero_rowsum(400, 9)
    s = mod.strength(A, 0.25)
    cf, nc = mod.pmis(A, s, 10)
    P = mod.bamg_direct(A, s, cf, nc)
    R, Ac = mod.galerkin(A, P)
    Pd = P.toarray()
    assert np.array_equal(R.toarray(), Pd.T)
    assert np.allclose(Ac.toarray(), Pd.T @ A.toarray() @ Pd, rtol=0, atol=1e-12)
    # A 1 = 0 and P 1 = 1 give A_c 1 = P^T A P 1 = 0
    assert np.allclose(Ac @ np.ones(nc), 0.0, atol=1e-12)
    # symmetric A gives a symmetric A_c
    B = sp.csr_matrix(pressure3d_7pt(8, seed=3))
    sB = mod.strength(B, 0.25)
    cfB, ncB = mod.pmis(B, sB, 1)
    _, AcB = mod.galerkin(B, mod.bamg_direct(B, sB, cfB, ncB))
    assert abs(AcB - AcB.T).max() <= 1e-12 * abs(AcB).max()


def test_galerkin_pins():
    _check_galerkin(OS)


def test_coarse_inverse():
    A = sp.csr_matrix(pressure3d_7pt(6, seed=1))
    X = OS.coarse_inverse(A)
    assert np.allclose(A @ X, np.eye(A.shape[0]), atol=1e-12)


def test_ilu0_factors_form_on_a_tridiagonal():
    # no fill-in: the sweeps reach the exact LU once they have crossed the dependency chain
    # (u_ii needs l_{i,i-1}, which needs u_{i-1,i-1}: two sweeps per row), and the LDU form then
    # reproduces A
    A = lap1d(12)
    Ls, Us, dinv = OS.ilu0_factors(A, 2 * 12)
    n = A.shape[0]
    M = (sp.eye(n) + Ls) @ sp.diags(1.0 / dinv) @ (sp.eye(n) + Us)
    assert np.allclose(M.toarray(), A.toarray(), rtol=0, atol=1e-13)
    assert Ls.nnz == n - 1 and Us.nnz == n - 1


def test_setup_levels_and_stop_rules():
    A = sp.csr_matrix(pressure3d_7pt(14, seed=2))
    levels, cinv = OS.setup(A, coarse_max=64, direct_max=512, seed=4, ilu_levels=(0, 1))
    ns = [lev["A"].shape[0] for lev in levels]
    assert all(b < 0.9 * a for a, b in zip(ns, ns[1:])) and ns[-1] <= 64 < ns[-2]
    for lev, nxt in zip(levels, levels[1:]):
        Pd = lev["P"].toarray()
        assert np.allclose(nxt["A"].toarray(), Pd.T @ lev["A"].toarray() @ Pd, atol=1e-11)
    assert "ilu" in levels[0] and "ilu" in levels[1] and cinv is not None
    assert np.allclose(levels[-1]["A"] @ cinv, np.eye(ns[-1]), atol=1e-10)


def test_setup_matches_the_host_input_generator():
    """The restatement and the host generator (C++, built for the solve-phase inputs) agree on
    every level: splitting, P and A_c (the generator's ILU is exact, so factors are not compared)."""
    A = sp.csr_matrix(pressure3d_7pt(12, seed=5))
    H = build_hierarchy(A, theta=0.25, coarse_max=64, seed=6, ilu_levels=())
    levels, _ = OS.setup(A, coarse_max=64, seed=6, ilu_levels=())
    assert len(levels) == H.nlevels
    for lev, hl in zip(levels, H.levels):
        assert lev["A"].shape == hl.A.shape and np.array_equal(lev["A"].indices, hl.A.indices)
        assert np.allclose(lev["A"].data, hl.A.data, rtol=1e-14, atol=0)
        if hl.P is not None:
            assert np.array_equal(lev["P"].indices, hl.P.indices)
            assert np.allclose(lev["P"].data, hl.P.data, rtol=1e-14, atol=0)


# ---- planted mistakes ----------------------------------------------------------------------

SETUP_MUTANTS = [
    ("(meas >= thr)", "(meas > thr)", _check_strength),                               # strict threshold
    ("meas = np.abs(vals) if mode", "meas = vals if mode", _check_strength),          # sign of the measure
    ("new_c[i] = not np.any(rank[js] > rank[i])", "new_c[i] = not np.any(rank[js] < rank[i])", _check_pmis),
    ("lam = infl + pmis_uniforms(seed, n)", "lam = pmis_uniforms(seed, n)", _check_pmis),  # weights without |S^T_i|
    ("st[infl == 0] = F", "st[infl == 0] = UNDEC", _check_pmis),
    ("js = S.indices[S.indptr[i]:S.indptr[i + 1]]\n            if np.any(new_c[js])",
     "js = ST.indices[ST.indptr[i]:ST.indptr[i + 1]]\n            if np.any(new_c[js])", _check_pmis),  # transposed S
    ("beta / len(strong_c)) / den", "beta) / den", _check_bamg),                      # beta not spread
    ("den = aii + weak", "den = aii", _check_bamg),                                    # weak not lumped
    ("elif not s[p]:\n                weak += a", "elif not s[p]:\n                weak -= a", _check_bamg),
    ("M1 = sp.diags(1.0 / (d_FF + gamma)) @ (As_FF + sp.diags(beta))", "M1 = sp.diags(1.0 / (d_FF + gamma)) @ As_FF",
     _check_mmext),                                                                    # D_beta dropped
    ("M1 = sp.diags(1.0 / (d_FF + gamma)) @", "M1 = sp.diags(1.0 / d_FF) @", _check_mmext),  # D_gamma dropped
    ("Ac = sp.csr_matrix(R @ sp.csr_matrix(A @ P))", "Ac = sp.csr_matrix(P.T @ sp.csr_matrix(A.T @ P))", _check_galerkin),
    ("z = ((z ^ (z >> 27)) * 0x94D049BB133111EB)", "z = ((z ^ (z >> 26)) * 0x94D049BB133111EB)", _check_splitmix),
]


def _mutated_setup(old, new):
    import importlib
    import inspect
    import types
    mod = importlib.import_module("oracle.setup")
    src = inspect.getsource(mod)
    assert src.count(old) == 1, old
    ns = dict(mod.__dict__)
    exec(compile(src.replace(old, new), mod.__file__, "exec"), ns)
    m = types.SimpleNamespace(**ns)
    return m


@pytest.mark.parametrize("old,new,pin", SETUP_MUTANTS, ids=[m[1].split("\n")[0][:40] for m in SETUP_MUTANTS])
def test_planted_setup_mistake_is_caught(old, new, pin):
    with pytest.raises(AssertionError):
        pin(_mutated_setup(old, new))
