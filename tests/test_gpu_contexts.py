"""Solver contexts (nsamg_context_create): a context shares its parent's matrices and tuned
kernel shapes, so its solves are bitwise the parent's, also when two contexts solve at the same
time from two host threads; destroying a context leaves the parent usable."""
import threading

import numpy as np
import pytest

from workloads import build_hierarchy, pressure3d_7pt, rhs_uniform

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2112_14681_b300 import nsamg  # noqa: E402


@pytest.mark.parametrize("fp32", [0, 1])
def test_context_solves_equal_the_parent_also_concurrently(fp32):
    A = pressure3d_7pt(24, seed=3)
    n = A.shape[0]
    H = build_hierarchy(A, theta=0.25, coarse_max=100, seed=1, ilu_levels=(0,))
    p = nsamg.default_params(smoother=nsamg.HYBRID_ILU0, vcycle_fp32=fp32)
    rhs = [rhs_uniform(n, k) for k in range(4)]
    with nsamg.setup_hierarchy(H, p) as h:
        ref = []
        for b in rhs:
            x = np.zeros(n)
            st = nsamg.solve_host(h, b, x, 1e-8, 300)
            assert st["converged"]
            assert np.linalg.norm(b - A @ x) <= 1e-8 * np.linalg.norm(b)
            ref.append(x)
        c1, c2 = h.context(), h.context()
        x = np.zeros(n)
        nsamg.solve_host(c1, rhs[0], x, 1e-8, 300)
        assert np.array_equal(x, ref[0])
        # two host threads, one context each, solving at the same time
        out, errors = {}, []

        def work(ctx, ks):
            try:
                for k in ks:
                    xk = np.zeros(n)
                    nsamg.solve_host(ctx, rhs[k], xk, 1e-8, 300)
                    out[k] = xk
            except Exception as e:  # reported below
                errors.append(e)

        ts = [threading.Thread(target=work, args=(c1, [0, 2])), threading.Thread(target=work, args=(c2, [1, 3]))]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        assert not errors, errors
        for k in range(4):
            assert np.array_equal(out[k], ref[k]), k
        # device buffers on a context; then the parent after its contexts are gone
        xd = torch.zeros(n, dtype=torch.float64, device="cuda")
        nsamg.solve(c2, torch.from_numpy(rhs[3]).cuda(), xd, 1e-8, 300)
        torch.cuda.synchronize()
        assert np.array_equal(xd.cpu().numpy(), ref[3])
        with pytest.raises(nsamg.NsamgError) as e:
            c1.context()  # a context of a context
        assert e.value.status == -1
        c1.close()
        c2.close()
        x = np.zeros(n)
        nsamg.solve_host(h, rhs[1], x, 1e-8, 300)
        assert np.array_equal(x, ref[1])
        c3 = h.context()
    assert c3._h is None  # closing the parent closed its live context first


def test_context_of_a_batch_handle_is_rejected():
    hs = [build_hierarchy(pressure3d_7pt(e, seed=e), max_levels=3, coarse_max=8, direct_max=10_000,
                          ilu_levels=None, seed=e) for e in (6, 7)]
    with nsamg.batch_setup(hs, nsamg.default_params()) as hb:
        with pytest.raises(nsamg.NsamgError) as e:
            hb.context()
        assert e.value.status == -1
