"""Every SELL-32 launch shape (K chunks per warp, U entries staged per round) on the three SELL
layouts: sorted with a permutation (ragged rows), plain with chunk offsets loaded (chunks of two
widths), plain with uniform chunks (7-point operator). All shapes sum each row in the order of
its stored entries, with padded entries adding exact zeros, so y = A x and r = b - A x are
bitwise the same for every shape and for CSR with one thread per row, in FP64 and in the FP32
copies; and within rounding of the product formed on the host."""
import numpy as np
import pytest
import scipy.sparse as sp

from workloads import pressure3d_7pt
from workloads.hierarchy import Hierarchy, Level

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2112_14681_b300 import nsamg  # noqa: E402

SHAPES = [11, 21, 41, 14, 22, 18]


def ragged(n=40000, seed=3):
    """Diagonal plus 0..40 random off-diagonal entries per row within a band of +-6000."""
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for i in range(n):
        k = int(rng.integers(0, 41))
        c = np.unique(np.clip(i + rng.integers(-6000, 6001, size=k), 0, n - 1))
        c = c[c != i]
        rows.append(np.full(c.size + 1, i))
        cols.append(np.concatenate([c, [i]]))
    r, c = np.concatenate(rows), np.concatenate(cols)
    v = rng.uniform(-1.0, 1.0, r.size)
    A = sp.csr_matrix((v, (r, c)), shape=(n, n))
    A.setdiag(np.abs(A).sum(axis=1).A.ravel() + 1.0)
    A.sort_indices()
    return A


def two_widths(n=40000, seed=5):
    """Rows of even chunks have 5 entries, rows of odd chunks 7: no padding inside a chunk, 17%
    padding if every chunk were as wide as the widest."""
    rng = np.random.default_rng(seed)
    offs5, offs7 = [-200, -1, 0, 1, 200], [-400, -200, -1, 0, 1, 200, 400]
    rows, cols = [], []
    for i in range(n):
        offs = offs7 if (i // 32) % 2 else offs5
        c = np.array([i + o for o in offs])
        c = np.where(c < 0, c + n, np.where(c >= n, c - n, c))
        rows.append(np.full(len(c), i))
        cols.append(c)
    r, c = np.concatenate(rows), np.concatenate(cols)
    A = sp.csr_matrix((rng.uniform(0.1, 1.0, r.size), (r, c)), shape=(n, n))
    A.setdiag(8.0)
    A.sort_indices()
    assert np.all(np.diff(A.indptr) == np.where((np.arange(n) // 32) % 2, 7, 5))
    return A


MATS = {"ragged": ragged, "two_widths": two_widths, "p34": lambda: pressure3d_7pt(34, seed=1)}
_cache = {}


def mat(name):
    if name not in _cache:
        _cache[name] = MATS[name]()
    return _cache[name]


def run(A, fp32, **kw):
    H = Hierarchy(levels=[Level(A=A)])
    rng = np.random.default_rng(11)
    x = torch.from_numpy(rng.uniform(-1, 1, A.shape[0])).cuda()
    b = torch.from_numpy(rng.uniform(-1, 1, A.shape[0])).cuda()
    y, r = torch.empty_like(x), torch.empty_like(x)
    with nsamg.setup_hierarchy(H, nsamg.default_params(vcycle_fp32=fp32, **kw)) as h:
        nsamg.level_spmv(h, 0, x, y)
        nsamg.level_residual(h, 0, b, x, r)
        torch.cuda.synchronize()
        group = nsamg.level_group(h, 0)
    return x.cpu().numpy(), b.cpu().numpy(), y.cpu().numpy(), r.cpu().numpy(), group


@pytest.mark.parametrize("fp32", [0, 1])
@pytest.mark.parametrize("name", list(MATS))
def test_every_sell_shape_is_bitwise_the_csr_result(name, fp32):
    A = mat(name)
    x, b, y_ref, r_ref, g = run(A, fp32, spmv_group=1)
    assert g == 1
    for shape in SHAPES:
        _, _, y, r, g = run(A, fp32, spmv_group=-1, sell_shape=shape)
        assert g == 0, shape  # the SELL copy was used
        assert np.array_equal(y, y_ref), shape
        assert np.array_equal(r, r_ref), shape
    # against the host product: FP64 within a few ulps of |A| |x|; FP32 within the FP32 rounding
    # of the matrix, the vector and each partial sum
    scale = abs(A) @ np.abs(x)
    k = int(np.diff(A.indptr).max())
    eps = np.finfo(np.float32 if fp32 else np.float64).eps
    assert np.all(np.abs(y_ref - A @ x) <= (k + 2) * eps * scale)


def test_bad_sell_shape_is_rejected():
    H = Hierarchy(levels=[Level(A=pressure3d_7pt(8))])
    with pytest.raises(nsamg.NsamgError) as e:
        nsamg.setup_hierarchy(H, nsamg.default_params(spmv_group=-1, sell_shape=12))
    assert e.value.status == -1
