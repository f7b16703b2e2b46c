"""Input generation: the host setup library's parallel Q1 assembly and symmetric permutation give
bitwise the matrix of the plain scipy construction (Kronecker products, CSR sums, fancy indexing)."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import reverse_cuthill_mckee

from workloads.matrices import _TAG_PERM, _fe1d, _finish, _graded_coords, _rng, q1_27pt_graded


def _scipy_q1(e, aspect, seed):
    hx = np.full(e + 1, 1.0 / (e + 1))
    hz = np.diff(_graded_coords(e, aspect, 1.1))
    Kx, Mx = _fe1d(hx)
    Kz, Mz = _fe1d(hz)
    A = sp.kron(sp.kron(Mz, Mx), Kx, format="csr")
    A = A + sp.kron(sp.kron(Mz, Kx), Mx, format="csr")
    A = _finish(A + sp.kron(sp.kron(Kz, Mx), Mx, format="csr"))
    perm = _rng(seed, _TAG_PERM).permutation(A.shape[0])
    A = _finish(A[perm, :][:, perm])
    rcm = reverse_cuthill_mckee(A, symmetric_mode=True)
    return _finish(A[rcm, :][:, rcm])


@pytest.mark.parametrize("e,seed", [(1, 0), (2, 0), (7, 3), (12, 1)])
def test_q1_generator_matches_scipy_construction(e, seed):
    want = _scipy_q1(e, 100.0, seed)
    got = q1_27pt_graded(e, aspect=100.0, seed=seed)
    assert np.array_equal(got.indptr, want.indptr)
    assert np.array_equal(got.indices, want.indices)
    assert np.array_equal(got.data, want.data)
    assert got.nnz == (3 * e - 2) ** 3 and abs(got - got.T).max() == 0.0
