"""The C-ABI library loads and exports every symbol include/nsamg.h declares (no GPU calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "nsamg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nsamg_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("nsamg_setup_hierarchy", "nsamg_solve", "nsamg_apply_vcycle", "nsamg_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2112_14681_b300 import build, nsamg
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(nsamg.EXPORTS) <= set(declared_functions())


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2112_14681_b300 import nsamg
    saved = nsamg._lib
    nsamg._lib = None
    try:
        with pytest.raises(ImportError):
            nsamg.load(str(tmp_path / "missing.so"))
    finally:
        nsamg._lib = saved


def test_status_strings_and_defaults():
    from paper_2112_14681_b300 import nsamg
    nsamg.load()
    assert nsamg.status_str(0) == "ok"
    assert nsamg.status_str(-6) == "non-finite value"
    p = nsamg.default_params()
    assert (p.smoother, p.neumann_terms, p.restart, p.use_graph) == (nsamg.POLY_GS, 2, 30, 1)


def _struct_fields(name):
    src = open(os.path.join(ROOT, "include", "nsamg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", src).group(1)
    return re.findall(r"\b(?:int32_t|int64_t|uint64_t|double|float)\s+(\w+)\s*;", body)


@pytest.mark.parametrize("cname,pyname", [("nsamg_params", "Params"), ("nsamg_stats", "Stats")])
def test_binding_structs_match_the_header(cname, pyname):
    """The ctypes mirrors list the header's fields in the header's order (a field added to one
    side only would shift every later field across the ABI)."""
    from paper_2112_14681_b300 import nsamg
    assert [f[0] for f in getattr(nsamg, pyname)._fields_] == _struct_fields(cname)


@pytest.mark.parametrize("bad", [dict(smoother=9), dict(neumann_terms=0), dict(ilu_terms_L=0), dict(ilu_terms_U=0),
                                 dict(pre_sweeps=-1), dict(post_sweeps=-1), dict(coarse_sweeps=0), dict(restart=0),
                                 dict(restart=65), dict(vcycle_fp32=2), dict(t_exact=2), dict(use_graph=2),
                                 dict(spmv_group=3), dict(spmv_group=64), dict(spmv_group=-2), dict(sell_shape=12),
                                 dict(fuse_tail=3), dict(fuse_tail=-1), dict(ranks=0), dict(ranks=-2), dict(ranks=(1 << 20) + 1), dict(krylov_fp64=2), dict(krylov_fp64=-1),
                                 dict(stop_nrbe=2)])
def test_params_are_rejected_before_any_device_work(bad):
    """nsamg_setup_hierarchy validates every parameter first: INVALID_ARG with a message, no device
    needed (this runs on CPU)."""
    from paper_2112_14681_b300 import nsamg
    from workloads import pressure3d_7pt
    from workloads.hierarchy import Hierarchy, Level
    H = Hierarchy(levels=[Level(A=pressure3d_7pt(4))])
    with pytest.raises(nsamg.NsamgError) as e:
        nsamg.setup_hierarchy(H, nsamg.default_params(**bad))
    assert e.value.status == -1
    assert nsamg.load().nsamg_last_error()


@pytest.mark.parametrize("vs,lds", [(0x1008, 1000), (0x1000, 999), (0x1000, 998)])
def test_split_basis_layout_is_checked_before_any_device_work(vs, lds):
    """The row-pair split layout needs 16-byte aligned columns (an even leading dimension) and
    room for the last row pair: the three split-basis entry points reject anything else with
    INVALID_ARG before touching memory (the pointers here are never dereferenced)."""
    import ctypes
    from paper_2112_14681_b300 import nsamg
    lib = nsamg.load()
    n, p, w = 999, ctypes.c_void_p(vs), ctypes.c_void_p(0x2000)
    assert lib.nsamg_split_basis(n, 1, ctypes.c_void_p(0x3000), n, p, lds, None) == -1
    assert lib.nsamg_gram_split(n, 0, p, lds, w, ctypes.c_void_p(0x4000), None) == -1
    assert lib.nsamg_update_split(n, 0, p, lds, w, 1.0, ctypes.c_void_p(0x5000), None, ctypes.c_void_p(0x6000),
                                  None) == -1
    assert lib.nsamg_last_error()
