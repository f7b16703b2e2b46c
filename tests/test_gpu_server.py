"""Request server: continuous batching on resident hierarchies. Each result must be the same
alone and in the mix (bitwise: every context runs the same deterministic kernels), every request
converges, admission and cancellation behave as documented."""
import time

import numpy as np
import pytest

from workloads import build_hierarchy, pressure3d_7pt, rhs_uniform

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2112_14681_b300 import nsamg  # noqa: E402

EDGES = [10, 14, 18]
_h = None


def hierarchies():
    global _h
    if _h is None:
        _h = []
        for k, e in enumerate(EDGES):
            A = pressure3d_7pt(e, seed=300 + k)
            _h.append((A, build_hierarchy(A, coarse_max=64, seed=k)))
    return _h


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("fp32", [0, 1])
def test_same_result_alone_and_in_the_mix(fp32):
    Hs = hierarchies()
    p = nsamg.default_params(smoother=nsamg.HYBRID_ILU0, vcycle_fp32=fp32)
    handles = [nsamg.setup_hierarchy(H, p) for _, H in Hs]
    reqs = [(k % 3, rhs_uniform(Hs[k % 3][0].shape[0], 500 + k)) for k in range(9)]
    try:
        # alone: one slot, one request at a time
        alone = []
        with nsamg.Server(1 << 34, 1) as srv:
            for hk, b in reqs:
                x = torch.zeros(b.size, dtype=torch.float64, device="cuda")
                st = srv.wait(srv.submit(handles[hk], dev(b), x))
                torch.cuda.synchronize()
                alone.append((st, x.cpu().numpy()))
        # in the mix: 4 slots, everything submitted at once
        with nsamg.Server(1 << 34, 4) as srv:
            xs, ts = [], []
            for hk, b in reqs:
                x = torch.zeros(b.size, dtype=torch.float64, device="cuda")
                xs.append(x)
                ts.append(srv.submit(handles[hk], dev(b), x))
            mixed = [srv.wait(t) for t in ts]
            torch.cuda.synchronize()
            assert srv.info()["contexts"] >= 2
        for k, (hk, b) in enumerate(reqs):
            A = Hs[hk][0]
            st_a, x_a = alone[k]
            x_m = xs[k].cpu().numpy()
            assert st_a["converged"] and mixed[k]["converged"]
            assert np.linalg.norm(b - A @ x_m) / np.linalg.norm(b) <= 1e-8
            assert np.array_equal(x_a, x_m) and st_a["iters"] == mixed[k]["iters"]
            assert mixed[k]["t_submit"] <= mixed[k]["t_start"] <= mixed[k]["t_done"]
    finally:
        for h in handles:
            h.close()


def test_server_matches_direct_solve():
    A, H = hierarchies()[1]
    b = rhs_uniform(A.shape[0], 7)
    with nsamg.setup_hierarchy(H, nsamg.default_params()) as h:
        x1 = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
        st1 = nsamg.solve(h, dev(b), x1)
        with nsamg.Server(1 << 34, 2) as srv:
            x2 = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
            st2 = srv.wait(srv.submit(h, dev(b), x2))
        torch.cuda.synchronize()
        assert np.array_equal(x1.cpu().numpy(), x2.cpu().numpy()) and st1["iters"] == st2["iters"]


def test_admission_budget_and_cancel():
    Hs = hierarchies()
    p = nsamg.default_params()
    handles = [nsamg.setup_hierarchy(H, p) for _, H in Hs]
    try:
        b = dev(rhs_uniform(Hs[0][0].shape[0], 1))
        # a budget no context fits: rejected, not queued forever
        with nsamg.Server(1024, 2) as srv:
            x = torch.zeros(b.numel(), dtype=torch.float64, device="cuda")
            t = srv.submit(handles[0], b, x)
            with pytest.raises(nsamg.NsamgError) as ei:
                srv.wait(t)
            assert ei.value.status == nsamg.ERR_ADMISSION
        # one slot: the third request is cancelled while it waits in the queue
        with nsamg.Server(1 << 34, 1) as srv:
            xs = [torch.zeros(b.numel(), dtype=torch.float64, device="cuda") for _ in range(3)]
            ts = [srv.submit(handles[0], b, xs[k]) for k in range(3)]
            srv.cancel(ts[2])
            assert srv.wait(ts[0])["converged"] and srv.wait(ts[1])["converged"]
            with pytest.raises(nsamg.NsamgError):
                srv.wait(ts[2])
            torch.cuda.synchronize()
            assert float(xs[2].abs().max()) == 0.0
        # a budget that holds one context at a time: alternating hierarchies evict and re-create
        sizes = [h_ctx_bytes(handles[k]) for k in range(2)]
        with nsamg.Server(max(sizes) + min(sizes) // 2, 2) as srv:
            out = []
            for k in range(4):
                hk = k % 2
                bb = rhs_uniform(Hs[hk][0].shape[0], 40 + k)
                x = torch.zeros(bb.size, dtype=torch.float64, device="cuda")
                out.append((hk, bb, x, srv.submit(handles[hk], dev(bb), x)))
            for hk, bb, x, t in out:
                st = srv.wait(t)
                torch.cuda.synchronize()
                A = Hs[hk][0]
                assert st["converged"] and np.linalg.norm(bb - A @ x.cpu().numpy()) / np.linalg.norm(bb) <= 1e-8
            assert srv.info()["contexts"] == 1
    finally:
        for h in handles:
            h.close()


def h_ctx_bytes(h):
    """Context size as the server estimates it: run one request alone and read the accounting."""
    with nsamg.Server(1 << 36, 1) as srv:
        n = h.n
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        srv.wait(srv.submit(h, torch.ones(n, dtype=torch.float64, device="cuda"), x))
        return srv.info()["bytes_in_use"]
