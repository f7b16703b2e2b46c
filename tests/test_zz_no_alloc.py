"""Allocation-free Gram entry point (nsamg_gram_noalloc) against the allocating one (nsamg_gram)
and against FP64 products on the host.

Some callers may not allocate device memory: their framework's allocator owns the budget, or the
call sits on a path that must not enter the CUDA allocator. This file is named so pytest collects
it last; the subprocess case also runs it in a fresh process where nothing else has run.
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2112_14681_b300 import nsamg  # noqa: E402

TOL = 1e-12
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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
    wh = w.cpu().numpy()
    norms = np.linalg.norm(Vh, axis=1)
    bound = np.concatenate([norms * norms[i], norms * np.linalg.norm(wh)])
    host = np.concatenate([Vh @ Vh[i], Vh @ wh])  # FP64 products on the host
    for _ in range(2):  # two calls in a row share the fixed scratch
        out = torch.full((2 * (i + 1),), np.nan, dtype=torch.float64, device="cuda")
        nsamg.gram_noalloc(n, i, V, ld, w, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.abs(got - ref.cpu().numpy()) <= TOL * bound)
        assert np.all(np.abs(got - host) <= TOL * bound)


def test_gram_noalloc_rejects_too_many_columns():
    nsamg.load()
    V = torch.zeros(65 * 10, dtype=torch.float64, device="cuda")
    w = torch.zeros(10, dtype=torch.float64, device="cuda")
    out = torch.zeros(130, dtype=torch.float64, device="cuda")
    with pytest.raises(nsamg.NsamgError) as ei:
        nsamg.gram_noalloc(10, 64, V, 10, w, out)
    assert ei.value.status == -1 and "63" in str(ei.value)


_FRESH = textwrap.dedent("""
    import sys
    import numpy as np
    import torch
    sys.path.insert(0, {root!r})
    from paper_2112_14681_b300 import nsamg
    nsamg.load()
    rng = np.random.default_rng(3)
    cases = [(300001, 5), (4097, 0), (1_000_003, 31), (77, 2)]
    bufs = []
    for n, i in cases:
        ld = n + 3
        V = torch.from_numpy(rng.standard_normal((i + 1) * ld)).cuda()
        w = torch.from_numpy(rng.standard_normal(n)).cuda()
        out = torch.empty(2 * (i + 1), dtype=torch.float64, device="cuda")
        bufs.append((n, i, ld, V, w, out))
    torch.cuda.synchronize()
    # the first Gram call of the process is the allocation-free one (it also loads the module)
    n, i, ld, V, w, out = bufs[0]
    nsamg.gram_noalloc(n, i, V, ld, w, out)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for n, i, ld, V, w, out in bufs + bufs:
        nsamg.gram_noalloc(n, i, V, ld, w, out)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, "device memory changed during gram_noalloc"
        Vh = V.cpu().numpy().reshape(i + 1, ld)[:, :n]
        wh = w.cpu().numpy()
        nr = np.linalg.norm(Vh, axis=1)
        bound = np.concatenate([nr * nr[i], nr * np.linalg.norm(wh)])
        host = np.concatenate([Vh @ Vh[i], Vh @ wh])
        assert np.all(np.abs(out.cpu().numpy() - host) <= 1e-12 * bound)
    # positive control: the allocating entry point's first call takes its scratch from cudaMalloc
    n, i, ld, V, w, out = bufs[0]
    nsamg.gram(n, i, V, ld, w, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] < free0, "nsamg_gram's first call allocated nothing"
    print("fresh-process no-alloc ok")
""")


def test_gram_noalloc_in_a_fresh_process_allocates_nothing():
    """In a new process whose first Gram call is nsamg_gram_noalloc: after that call, free device
    memory stays exactly the same over calls with other sizes, and every result matches host FP64
    products; then nsamg_gram's first call lowers it (its scratch is allocated)."""
    r = subprocess.run([sys.executable, "-c", _FRESH.format(root=ROOT)], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "fresh-process no-alloc ok" in r.stdout
