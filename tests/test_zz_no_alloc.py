"""Allocation-free Gram entry point (nsamg_gram_noalloc) against the allocating one (nsamg_gram).

Some callers may not allocate device memory (their framework's allocator owns the budget, or the
call sits on a path that must not enter the CUDA allocator). This file is named so pytest
collects it last; it must also pass on its own in a fresh process.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2112_14681_b300 import nsamg  # noqa: E402

TOL = 1e-12


@pytest.mark.parametrize("n,i", [(1000, 0), (262147, 9), (2_000_003, 63)])
def test_gram_noalloc_matches_gram_twice(n, i):
    nsamg.load()
    rng = np.random.default_rng(n + i)
    ld = n + 5
    V = torch.from_numpy(rng.standard_normal((i + 1) * ld)).cuda()
    w = torch.from_numpy(rng.standard_normal(n)).cuda()
    ref = torch.empty(2 * (i + 1), dtype=torch.float64, device="cuda")
    nsamg.gram(n, i, V, ld, w, ref)
    torch.cuda.synchronize()
    Vh = V.cpu().numpy().reshape(i + 1, ld)[:, :n]
    scale = np.linalg.norm(Vh, axis=1) * np.concatenate([np.full(i + 1, np.linalg.norm(Vh[i]))])
    scale_w = np.linalg.norm(Vh, axis=1) * np.linalg.norm(w.cpu().numpy())
    bound = np.concatenate([scale, scale_w])
    for _ in range(2):  # two calls in a row share the fixed scratch
        out = torch.full((2 * (i + 1),), np.nan, dtype=torch.float64, device="cuda")
        nsamg.gram_noalloc(n, i, V, ld, w, out)
        torch.cuda.synchronize()
        d = np.abs(out.cpu().numpy() - ref.cpu().numpy())
        assert np.all(d <= TOL * bound)


def test_gram_noalloc_rejects_too_many_columns():
    nsamg.load()
    V = torch.zeros(65 * 10, dtype=torch.float64, device="cuda")
    w = torch.zeros(10, dtype=torch.float64, device="cuda")
    out = torch.zeros(130, dtype=torch.float64, device="cuda")
    with pytest.raises(nsamg.NsamgError) as ei:
        nsamg.gram_noalloc(10, 64, V, 10, w, out)
    assert ei.value.status == -1 and "63" in str(ei.value)
