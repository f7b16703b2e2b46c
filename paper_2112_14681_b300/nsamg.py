"""ctypes binding of libnsamg.so (argument marshalling only).

Names follow the C ABI without the `nsamg_` prefix. Device vectors are torch CUDA float64
tensors (contiguous); host matrices are scipy.sparse CSR matrices (float64, int32 indices,
sorted columns). Errors raise NsamgError with the library's message.
"""
from __future__ import annotations

import ctypes
import os
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnsamg.so")

OK, NOT_CONVERGED, PENDING = 0, 1, 2
POLY_GS, JACOBI_L1, ILU0, HYBRID_ILU0 = 0, 1, 2, 3
MAX_RESTART = 64


class NsamgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"nsamg status {status}: {msg}")
        self.status = status


class Csr(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int32), ("ncols", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("rowptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class LevelDesc(ctypes.Structure):
    _fields_ = [("A", Csr), ("P", Csr), ("R", Csr), ("ilu_L", Csr), ("ilu_U", Csr), ("ilu_dinv", ctypes.c_void_p),
                ("ilu_form", ctypes.c_int32), ("ilu_dr", ctypes.c_void_p), ("ilu_dc", ctypes.c_void_p)]


class HierarchyDesc(ctypes.Structure):
    _fields_ = [("nlevels", ctypes.c_int32), ("levels", ctypes.POINTER(LevelDesc)), ("coarse_inv", ctypes.c_void_p)]


class Params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("smoother", "neumann_terms", "ilu_terms_L", "ilu_terms_U", "pre_sweeps",
                                               "post_sweeps", "coarse_sweeps", "restart", "vcycle_fp32", "t_exact",
                                               "use_graph", "spmv_group", "fuse_tail", "sell_shape", "krylov_fp64",
                                               "stop_nrbe", "ranks")]


class AmgOptions(ctypes.Structure):
    _fields_ = [("theta", ctypes.c_double), ("strength_mode", ctypes.c_int32), ("max_levels", ctypes.c_int32),
                ("coarse_max", ctypes.c_int32), ("direct_max", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("ilu_levels", ctypes.c_uint64), ("ilu_sweeps", ctypes.c_int32), ("interp", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("restarts", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("status", ctypes.c_int32), ("relres_true", ctypes.c_double), ("relres_implicit", ctypes.c_double),
                ("bnorm", ctypes.c_double), ("nrbe", ctypes.c_double), ("orth_loss", ctypes.c_double),
                ("sk_norm", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = [
    "nsamg_default_params", "nsamg_setup_hierarchy", "nsamg_solve", "nsamg_solve_host", "nsamg_apply_vcycle",
    "nsamg_num_levels", "nsamg_level_size", "nsamg_level_group", "nsamg_level_spmv", "nsamg_level_residual",
    "nsamg_level_smooth", "nsamg_level_restrict", "nsamg_level_prolong", "nsamg_coarse_solve", "nsamg_gram",
    "nsamg_update", "nsamg_gram_fp64", "nsamg_update_fp64", "nsamg_split_basis", "nsamg_gram_split",
    "nsamg_update_split", "nsamg_destroy", "nsamg_context_create", "nsamg_status_str", "nsamg_last_error",
    "nsamg_launches_per_step", "nsamg_fma_probe", "nsamg_grid_barrier_test",
    "nsamg_gram_noalloc", "nsamg_batch_setup", "nsamg_batch_solve", "nsamg_batch_count", "nsamg_batch_offsets",
    "nsamg_server_create", "nsamg_server_submit", "nsamg_server_poll", "nsamg_server_wait", "nsamg_server_cancel",
    "nsamg_server_info", "nsamg_server_destroy", "nsamg_ilu0_fixed_point",
    "nsamg_sknorm", "nsamg_amg_default_options", "nsamg_amg_build", "nsamg_amg_num_levels", "nsamg_amg_level_info",
    "nsamg_amg_level_splitting", "nsamg_amg_export", "nsamg_amg_setup_solver", "nsamg_amg_destroy",
]

_lib = None


def load(path: str = LIB_PATH):
    """Load libnsamg.so; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2112_14681_b300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    sig = {
        "nsamg_default_params": (None, [ctypes.POINTER(Params)]),
        "nsamg_setup_hierarchy": (i32, [ctypes.POINTER(HierarchyDesc), ctypes.POINTER(Params), vp, ctypes.POINTER(vp)]),
        "nsamg_solve": (i32, [vp, vp, vp, f64, i32, ctypes.POINTER(Stats)]),
        "nsamg_solve_host": (i32, [vp, vp, vp, f64, i32, ctypes.POINTER(Stats)]),
        "nsamg_apply_vcycle": (i32, [vp, vp, vp]),
        "nsamg_num_levels": (i32, [vp]),
        "nsamg_level_size": (i32, [vp, i32]),
        "nsamg_level_group": (i32, [vp, i32]),
        "nsamg_level_spmv": (i32, [vp, i32, vp, vp]),
        "nsamg_level_residual": (i32, [vp, i32, vp, vp, vp]),
        "nsamg_level_smooth": (i32, [vp, i32, i32, i32, vp, vp]),
        "nsamg_level_restrict": (i32, [vp, i32, vp, vp]),
        "nsamg_level_prolong": (i32, [vp, i32, vp, vp]),
        "nsamg_coarse_solve": (i32, [vp, vp, vp]),
        "nsamg_gram": (i32, [i64, i32, vp, i64, vp, vp, vp]),
        "nsamg_update": (i32, [i64, i32, vp, i64, vp, f64, vp, vp, vp]),
        "nsamg_gram_fp64": (i32, [i64, i32, vp, i64, vp, vp, vp]),
        "nsamg_split_basis": (i32, [i64, i32, vp, i64, vp, i64, vp]),
        "nsamg_gram_split": (i32, [i64, i32, vp, i64, vp, vp, vp]),
        "nsamg_update_split": (i32, [i64, i32, vp, i64, vp, f64, vp, vp, vp, vp]),
        "nsamg_update_fp64": (i32, [i64, i32, vp, i64, vp, f64, vp, vp, vp]),
        "nsamg_gram_noalloc": (i32, [i64, i32, vp, i64, vp, vp, vp]),
        "nsamg_batch_setup": (i32, [ctypes.POINTER(HierarchyDesc), i32, ctypes.POINTER(Params), vp, ctypes.POINTER(vp)]),
        "nsamg_batch_solve": (i32, [vp, vp, vp, f64, i32, ctypes.POINTER(Stats)]),
        "nsamg_batch_count": (i32, [vp]),
        "nsamg_batch_offsets": (i32, [vp, ctypes.POINTER(ctypes.c_int64)]),
        "nsamg_server_create": (i32, [ctypes.c_size_t, i32, ctypes.POINTER(vp)]),
        "nsamg_server_submit": (i32, [vp, vp, vp, vp, f64, i32, vp, ctypes.POINTER(ctypes.c_uint64)]),
        "nsamg_server_poll": (i32, [vp, ctypes.c_uint64, ctypes.POINTER(Stats), ctypes.POINTER(f64)]),
        "nsamg_server_wait": (i32, [vp, ctypes.c_uint64, ctypes.POINTER(Stats), ctypes.POINTER(f64)]),
        "nsamg_server_cancel": (i32, [vp, ctypes.c_uint64]),
        "nsamg_server_info": (i32, [vp, ctypes.POINTER(ctypes.c_int64)]),
        "nsamg_server_destroy": (None, [vp]),
        "nsamg_ilu0_fixed_point": (i32, [ctypes.POINTER(Csr), i32, vp, vp]),
        "nsamg_sknorm": (i32, [vp, i32, i32, vp, vp]),
        "nsamg_amg_default_options": (None, [ctypes.POINTER(AmgOptions)]),
        "nsamg_amg_build": (i32, [ctypes.POINTER(Csr), ctypes.POINTER(AmgOptions), vp, ctypes.POINTER(vp)]),
        "nsamg_amg_num_levels": (i32, [vp]),
        "nsamg_amg_level_info": (i32, [vp, i32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
        "nsamg_amg_level_splitting": (i32, [vp, i32, vp, vp]),
        "nsamg_amg_export": (i32, [vp, ctypes.POINTER(HierarchyDesc)]),
        "nsamg_amg_setup_solver": (i32, [vp, ctypes.POINTER(Params), vp, ctypes.POINTER(vp)]),
        "nsamg_amg_destroy": (None, [vp]),
        "nsamg_destroy": (None, [vp]),
        "nsamg_context_create": (i32, [vp, ctypes.POINTER(vp)]),
        "nsamg_launches_per_step": (i32, [vp]),
        "nsamg_fma_probe": (i32, [i32, i64, i32, vp, vp, ctypes.POINTER(f64)]),
        "nsamg_grid_barrier_test": (i32, [i32, i32, ctypes.c_uint, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "nsamg_status_str": (ctypes.c_char_p, [i32]),
        "nsamg_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int, allow=(OK,)) -> int:
    if rc in allow:
        return rc
    lib = load()
    raise NsamgError(rc, lib.nsamg_last_error().decode())


def _ptr(t) -> int:
    """Device pointer of a contiguous torch CUDA tensor (or an int address)."""
    if isinstance(t, int):
        return t
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def default_params(**overrides) -> Params:
    p = Params()
    load().nsamg_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, int(v))
    return p


def _csr_desc(M, keep: list) -> Csr:
    c = Csr()
    if M is None:
        return c
    M = M.tocsr()
    if not M.has_sorted_indices:  # the ABI requires sorted columns; sort a copy
        M = M.copy()
        M.sort_indices()
    rp = np.ascontiguousarray(M.indptr, dtype=np.int32)
    ci = np.ascontiguousarray(M.indices, dtype=np.int32)
    v = np.ascontiguousarray(M.data, dtype=np.float64)
    keep += [rp, ci, v]
    c.nrows, c.ncols, c.nnz = M.shape[0], M.shape[1], M.nnz
    c.rowptr, c.col, c.val = rp.ctypes.data, ci.ctypes.data, v.ctypes.data
    return c


def _hierarchy_desc(hierarchy, keep: list) -> HierarchyDesc:
    levels = hierarchy.levels
    arr = (LevelDesc * len(levels))()
    keep.append(arr)
    for l, lev in enumerate(levels):
        arr[l].A = _csr_desc(lev.A, keep)
        arr[l].P = _csr_desc(lev.P, keep)
        arr[l].R = _csr_desc(lev.R, keep)
        arr[l].ilu_L = _csr_desc(lev.ilu_L, keep)
        arr[l].ilu_U = _csr_desc(lev.ilu_U, keep)
        if lev.ilu_dinv is not None:
            d = np.ascontiguousarray(lev.ilu_dinv, dtype=np.float64)
            keep.append(d)
            arr[l].ilu_dinv = d.ctypes.data
        arr[l].ilu_form = int(getattr(lev, "ilu_form", 0))
        for fld in ("ilu_dr", "ilu_dc"):
            vec = getattr(lev, fld, None)
            if vec is not None:
                d = np.ascontiguousarray(vec, dtype=np.float64)
                keep.append(d)
                setattr(arr[l], fld, d.ctypes.data)
    desc = HierarchyDesc()
    desc.nlevels = len(levels)
    desc.levels = arr
    if hierarchy.coarse_inv is not None:
        ci = np.ascontiguousarray(hierarchy.coarse_inv, dtype=np.float64)
        keep.append(ci)
        desc.coarse_inv = ci.ctypes.data
    return desc


class Handle:
    """Owns an nsamg handle (device hierarchy + GMRES workspace)."""

    def __init__(self, hierarchy, params: Params | None = None, stream=None, _batch=None):
        lib = load()
        keep: list = []
        self.params = params or default_params()
        sptr = None if stream is None else ctypes.c_void_p(stream)
        h = ctypes.c_void_p()
        if _batch is not None:  # list of hierarchies -> one batch handle
            descs = (HierarchyDesc * len(_batch))()
            for k, hier in enumerate(_batch):
                descs[k] = _hierarchy_desc(hier, keep)
            _check(lib.nsamg_batch_setup(descs, len(_batch), ctypes.byref(self.params), sptr, ctypes.byref(h)))
            self._h = h
            self.count = len(_batch)
            off = (ctypes.c_int64 * (self.count + 1))()
            _check(lib.nsamg_batch_offsets(h, off))
            self.offsets = np.array(off[:], dtype=np.int64)
            self.n = int(self.offsets[-1])
            return
        levels = hierarchy.levels
        desc = _hierarchy_desc(hierarchy, keep)
        _check(lib.nsamg_setup_hierarchy(ctypes.byref(desc), ctypes.byref(self.params), sptr, ctypes.byref(h)))
        self._h = h
        self.n = levels[0].A.shape[0]

    def context(self) -> "Handle":
        """A second solver context on this hierarchy (nsamg_context_create). It keeps this handle
        alive while it exists, and closing this handle closes its contexts first (they use its
        matrices)."""
        c = Handle.__new__(Handle)
        c.params = self.params
        hp = ctypes.c_void_p()
        _check(load().nsamg_context_create(self._h, ctypes.byref(hp)))
        c._h = hp
        c.n = self.n
        c._parent = self
        if not hasattr(self, "_contexts"):
            self._contexts = weakref.WeakSet()
        self._contexts.add(c)
        return c

    def close(self):
        for c in list(getattr(self, "_contexts", ())):
            c.close()
        if getattr(self, "_h", None):
            load().nsamg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def setup_hierarchy(hierarchy, params: Params | None = None, stream=None) -> Handle:
    return Handle(hierarchy, params, stream)


def batch_setup(hierarchies, params: Params | None = None, stream=None) -> Handle:
    """Block-diagonal batch of independent systems (same depth); see nsamg_batch_setup."""
    return Handle(None, params, stream, _batch=list(hierarchies))


def batch_solve(h: Handle, b, x, rtol: float = 1e-8, maxit: int = 1000) -> list:
    """b, x: concatenated device vectors (system s at rows offsets[s]:offsets[s+1])."""
    st = (Stats * h.count)()
    rc = load().nsamg_batch_solve(h._h, _ptr(b), _ptr(x), float(rtol), int(maxit), st)
    _check(rc, (OK, NOT_CONVERGED))
    return [s.as_dict() for s in st]


def solve(h: Handle, b, x, rtol: float = 1e-8, maxit: int = 1000) -> dict:
    st = Stats()
    rc = load().nsamg_solve(h._h, _ptr(b), _ptr(x), float(rtol), int(maxit), ctypes.byref(st))
    _check(rc, (OK, NOT_CONVERGED))
    return st.as_dict()


def solve_host(h: Handle, b: np.ndarray, x: np.ndarray, rtol: float = 1e-8, maxit: int = 1000) -> dict:
    """b, x: host float64 arrays (pinned torch CPU tensors or numpy); x is updated in place."""
    st = Stats()

    def hptr(a):
        if isinstance(a, np.ndarray):
            assert a.dtype == np.float64 and a.flags.c_contiguous
            return a.ctypes.data
        return a.data_ptr()
    rc = load().nsamg_solve_host(h._h, hptr(b), hptr(x), float(rtol), int(maxit), ctypes.byref(st))
    _check(rc, (OK, NOT_CONVERGED))
    return st.as_dict()


def apply_vcycle(h: Handle, r, z) -> None:
    _check(load().nsamg_apply_vcycle(h._h, _ptr(r), _ptr(z)))


def num_levels(h: Handle) -> int:
    return _check(load().nsamg_num_levels(h._h), allow=range(0, 1 << 30))


def level_size(h: Handle, level: int) -> int:
    return _check(load().nsamg_level_size(h._h, level), allow=range(0, 1 << 31))


def level_group(h: Handle, level: int) -> int:
    return _check(load().nsamg_level_group(h._h, level), allow=range(0, 33))


def launches_per_step(h: Handle) -> int:
    return _check(load().nsamg_launches_per_step(h._h), allow=range(0, 1 << 30))


def solve_launches(h: Handle, stats: dict) -> int:
    """Kernel launches of a finished solve: initial residual + iters * per_step + 2 per cycle
    (x-update, residual) + the final ||S_k||_2 kernel."""
    return 2 + stats["iters"] * launches_per_step(h) + 2 * (stats["restarts"] + 1)


def level_spmv(h: Handle, level: int, x, y) -> None:
    _check(load().nsamg_level_spmv(h._h, level, _ptr(x), _ptr(y)))


def level_residual(h: Handle, level: int, b, x, r) -> None:
    _check(load().nsamg_level_residual(h._h, level, _ptr(b), _ptr(x), _ptr(r)))


def level_smooth(h: Handle, level: int, b, x, backward: bool = False, x_is_zero: bool = False) -> None:
    _check(load().nsamg_level_smooth(h._h, level, int(backward), int(x_is_zero), _ptr(b), _ptr(x)))


def level_restrict(h: Handle, level: int, r, y) -> None:
    _check(load().nsamg_level_restrict(h._h, level, _ptr(r), _ptr(y)))


def level_prolong(h: Handle, level: int, e, x) -> None:
    _check(load().nsamg_level_prolong(h._h, level, _ptr(e), _ptr(x)))


def coarse_solve(h: Handle, b, z) -> None:
    _check(load().nsamg_coarse_solve(h._h, _ptr(b), _ptr(z)))


def gram(n: int, i: int, V, ldv: int, w, out, stream=None) -> None:
    _check(load().nsamg_gram(int(n), int(i), _ptr(V), int(ldv), _ptr(w), _ptr(out), stream))


def gram_noalloc(n: int, i: int, V, ldv: int, w, out, stream=None) -> None:
    """Same as gram() but never allocates device memory: the scratch is a fixed array inside the
    library (room for i <= 63). For callers whose device memory is owned by another allocator or
    who must stay out of the CUDA allocator; overlapping calls race on the shared array."""
    _check(load().nsamg_gram_noalloc(int(n), int(i), _ptr(V), int(ldv), _ptr(w), _ptr(out), stream))


def update(n: int, i: int, V, ldv: int, w, beta: float, h, sumsq, stream=None) -> None:
    _check(load().nsamg_update(int(n), int(i), _ptr(V), int(ldv), _ptr(w), float(beta), _ptr(h), _ptr(sumsq), stream))


def split_basis(n: int, ncols: int, V, ldv: int, Vs, lds: int, stream=None) -> None:
    """FP64 columns -> (hi, lo) float pairs (the layout of a solve's basis); Vs: any contiguous
    device buffer of at least 8 * lds * ncols bytes (e.g. a float32 tensor of 2 * lds * ncols)."""
    _check(load().nsamg_split_basis(int(n), int(ncols), _ptr(V), int(ldv), _ptr(Vs), int(lds), stream))


def gram_split(n: int, i: int, Vs, lds: int, w, out, stream=None) -> None:
    """Raw products vt_j . vt_i and vt_j . w (j <= i) on the split basis (a solve's Gram kernel)."""
    _check(load().nsamg_gram_split(int(n), int(i), _ptr(Vs), int(lds), _ptr(w), _ptr(out), stream))


def update_split(n: int, i: int, Vs, lds: int, w, beta_i: float, c, vin, sumsq, stream=None) -> None:
    """Column i+1 = w / beta_i - sum_j c_j vt_j on the split basis (a solve's update kernel)."""
    _check(load().nsamg_update_split(int(n), int(i), _ptr(Vs), int(lds), _ptr(w), float(beta_i), _ptr(c),
                                     None if vin is None else _ptr(vin), _ptr(sumsq), stream))


def gram_fp64(n: int, i: int, V, ldv: int, w, out, stream=None) -> None:
    """gram() with every product and sum in FP64."""
    _check(load().nsamg_gram_fp64(int(n), int(i), _ptr(V), int(ldv), _ptr(w), _ptr(out), stream))


def update_fp64(n: int, i: int, V, ldv: int, w, beta: float, h, sumsq, stream=None) -> None:
    """update() with every product and sum in FP64."""
    _check(load().nsamg_update_fp64(int(n), int(i), _ptr(V), int(ldv), _ptr(w), float(beta), _ptr(h), _ptr(sumsq),
                                    stream))


def grid_barrier_test(rounds: int, missing: int = 0, spin_limit: int = 1 << 20) -> tuple:
    """(barriers completed summed over blocks, status) of nsamg_grid_barrier_test: one block per
    SM runs `rounds` bounded grid barriers, each expecting `missing` arrivals more than the grid
    has (missing > 0: every wait gives up after `spin_limit` polls, status NSAMG_ERR_TIMEOUT)."""
    passed, status = ctypes.c_int(), ctypes.c_int()
    _check(load().nsamg_grid_barrier_test(int(rounds), int(missing), int(spin_limit), ctypes.byref(passed),
                                          ctypes.byref(status)))
    return passed.value, status.value


def fma_rate(fp64: bool, iters: int = 1 << 16, blocks_per_sm: int = 8, reps: int = 5) -> float:
    """FMA/s of the current device in FP64 or FP32 (nsamg_fma_probe, best of `reps` launches
    timed with CUDA events after one warm-up launch)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks = sms * blocks_per_sm
    sink = torch.empty(blocks * 256, dtype=torch.float64 if fp64 else torch.float32, device="cuda")
    s = torch.cuda.current_stream()
    cnt = ctypes.c_double()
    lib = load()
    _check(lib.nsamg_fma_probe(int(bool(fp64)), int(iters), blocks, _ptr(sink), s.cuda_stream, ctypes.byref(cnt)))
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        _check(lib.nsamg_fma_probe(int(bool(fp64)), int(iters), blocks, _ptr(sink), s.cuda_stream, None))
        e1.record(s)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) * 1e-3)
    return cnt.value / best


def sknorm(L, k: int | None = None, out=None, stream=None) -> float:
    """||S_k||_2 of the strictly lower part of the device matrix L (torch, row-major)."""
    import torch
    k = int(L.shape[0] if k is None else k)
    if out is None:
        out = torch.zeros(1, dtype=torch.float64, device=L.device)
    _check(load().nsamg_sknorm(_ptr(L), int(L.stride(0)), k, _ptr(out), stream))
    return float(out.cpu()[0])


def ilu0_fixed_point(A, sweeps: int, stream=None) -> np.ndarray:
    """ILU(0) values on A's pattern after `sweeps` fixed-point sweeps on the GPU
    (strictly lower entries: L_s; the others: U with its diagonal)."""
    keep: list = []
    c = _csr_desc(A, keep)
    out = np.empty(A.nnz, np.float64)
    _check(load().nsamg_ilu0_fixed_point(ctypes.byref(c), int(sweeps), out.ctypes.data, stream))
    return out


def amg_default_options(**overrides) -> AmgOptions:
    o = AmgOptions()
    load().nsamg_amg_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, float(v) if k == "theta" else int(v))
    return o


def _csr_from_desc(c: Csr):
    """Copy a host CSR described by the library into a scipy matrix (None when absent)."""
    import scipy.sparse as sp
    if c.nrows == 0:
        return None
    n, nnz = int(c.nrows), int(c.nnz)
    rp = np.ctypeslib.as_array(ctypes.cast(c.rowptr, ctypes.POINTER(ctypes.c_int32)), (n + 1,)).copy()
    if nnz:
        ci = np.ctypeslib.as_array(ctypes.cast(c.col, ctypes.POINTER(ctypes.c_int32)), (nnz,)).copy()
        v = np.ctypeslib.as_array(ctypes.cast(c.val, ctypes.POINTER(ctypes.c_double)), (nnz,)).copy()
    else:
        ci, v = np.zeros(0, np.int32), np.zeros(0)
    M = sp.csr_matrix((v, ci, rp), shape=(n, int(c.ncols)))
    M.has_sorted_indices = True
    return M


class ExportedLevel:
    """One level of a GPU-built hierarchy copied to the host (the attributes setup_hierarchy reads)."""

    def __init__(self, d: LevelDesc):
        self.A, self.P, self.R = _csr_from_desc(d.A), _csr_from_desc(d.P), _csr_from_desc(d.R)
        self.ilu_L, self.ilu_U = _csr_from_desc(d.ilu_L), _csr_from_desc(d.ilu_U)
        n = self.A.shape[0]
        self.ilu_dinv = (np.ctypeslib.as_array(ctypes.cast(d.ilu_dinv, ctypes.POINTER(ctypes.c_double)), (n,)).copy()
                         if d.ilu_dinv else None)
        self.ilu_form, self.ilu_dr, self.ilu_dc = 0, None, None

    @property
    def n(self) -> int:
        return self.A.shape[0]


class ExportedHierarchy:
    def __init__(self, levels, coarse_inv):
        self.levels, self.coarse_inv = levels, coarse_inv

    @property
    def nlevels(self) -> int:
        return len(self.levels)


class GpuHierarchy:
    """Ruge-Stuben hierarchy of A built on the GPU (nsamg_amg_build)."""

    def __init__(self, A, options: AmgOptions | None = None, stream=None):
        lib = load()
        keep: list = []
        self.options = options or amg_default_options()
        c = _csr_desc(A, keep)
        g = ctypes.c_void_p()
        _check(lib.nsamg_amg_build(ctypes.byref(c), ctypes.byref(self.options),
                                   None if stream is None else ctypes.c_void_p(stream), ctypes.byref(g)))
        self._g = g

    @property
    def nlevels(self) -> int:
        return int(load().nsamg_amg_num_levels(self._g))

    def level_info(self, l: int) -> dict:
        n, nc, rounds = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        nnz = ctypes.c_int64()
        _check(load().nsamg_amg_level_info(self._g, int(l), ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(nc),
                                           ctypes.byref(rounds)))
        return {"n": n.value, "nnz": nnz.value, "nc": nc.value, "pmis_rounds": rounds.value}

    def splitting(self, l: int):
        """(cf, strong): coarse index or -1 per point; strength flag per entry of A_l."""
        info = self.level_info(l)
        cf = np.empty(info["n"], np.int32)
        strong = np.empty(max(info["nnz"], 1), np.uint8)
        _check(load().nsamg_amg_level_splitting(self._g, int(l), cf.ctypes.data, strong.ctypes.data))
        return cf, strong[:info["nnz"]].astype(bool)

    def export(self) -> ExportedHierarchy:
        d = HierarchyDesc()
        _check(load().nsamg_amg_export(self._g, ctypes.byref(d)))
        levels = [ExportedLevel(d.levels[l]) for l in range(d.nlevels)]
        cinv = None
        if d.coarse_inv:
            nc = levels[-1].n
            cinv = np.ctypeslib.as_array(ctypes.cast(d.coarse_inv, ctypes.POINTER(ctypes.c_double)), (nc, nc)).copy()
        return ExportedHierarchy(levels, cinv)

    def setup_solver(self, params: Params | None = None, stream=None) -> Handle:
        h = Handle.__new__(Handle)
        h.params = params or default_params()
        hp = ctypes.c_void_p()
        _check(load().nsamg_amg_setup_solver(self._g, ctypes.byref(h.params),
                                             None if stream is None else ctypes.c_void_p(stream), ctypes.byref(hp)))
        h._h = hp
        h.n = self.level_info(0)["n"]
        return h

    def close(self):
        if getattr(self, "_g", None):
            load().nsamg_amg_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def amg_build(A, options: AmgOptions | None = None, stream=None) -> GpuHierarchy:
    return GpuHierarchy(A, options, stream)


def status_str(s: int) -> str:
    return load().nsamg_status_str(int(s)).decode()


ERR_TIMEOUT = -5
ERR_ADMISSION = -7


class Server:
    """Continuous-batching request server (see nsamg_server_create). Device arrays passed to
    submit() must stay alive until the request completes; the object keeps references."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.nsamg_server_create(int(hbm_budget_bytes), int(max_slots), ctypes.byref(h)))
        self._s = h
        self._keep: dict = {}

    def submit(self, handle: Handle, b, x, rtol: float = 1e-8, maxit: int = 1000, ready_stream=None) -> int:
        """ready_stream: cudaStream_t (int) on which b and x were produced; None = legacy default."""
        t = ctypes.c_uint64()
        rs = None if not ready_stream else ctypes.c_void_p(ready_stream)
        _check(load().nsamg_server_submit(self._s, handle._h, _ptr(b), _ptr(x), float(rtol), int(maxit), rs,
                                          ctypes.byref(t)))
        self._keep[t.value] = (b, x)
        return t.value

    def _result(self, fn, ticket: int):
        st = Stats()
        times = (ctypes.c_double * 3)()
        rc = fn(self._s, ctypes.c_uint64(ticket), ctypes.byref(st), times)
        if rc == PENDING:
            return None
        self._keep.pop(ticket, None)
        _check(rc, (OK, NOT_CONVERGED))
        d = st.as_dict()
        d["t_submit"], d["t_start"], d["t_done"] = times[0], times[1], times[2]
        return d

    def poll(self, ticket: int):
        """None while pending, else the stats dict (with server-clock times)."""
        return self._result(load().nsamg_server_poll, ticket)

    def wait(self, ticket: int) -> dict:
        return self._result(load().nsamg_server_wait, ticket)

    def cancel(self, ticket: int) -> None:
        _check(load().nsamg_server_cancel(self._s, ctypes.c_uint64(ticket)))

    def info(self) -> dict:
        out = (ctypes.c_int64 * 4)()
        _check(load().nsamg_server_info(self._s, out))
        return {"bytes_in_use": out[0], "contexts": out[1], "running": out[2], "queued": out[3]}

    def close(self):
        if getattr(self, "_s", None):
            load().nsamg_server_destroy(self._s)
            self._s = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
