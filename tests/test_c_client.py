"""The C ABI is usable from plain C: tests/c/abi_smoke.c compiles against include/nsamg.h and
links libnsamg.so (CPU check); on a GPU it builds a two-level hierarchy by hand and solves."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _build(tmp_path):
    from paper_2112_14681_b300 import build
    lib = build.build()
    exe = str(tmp_path / "abi_smoke")
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-Wall", "-Werror", os.path.join(ROOT, "tests", "c", "abi_smoke.c"),
                           "-I", os.path.join(ROOT, "include"), "-L", os.path.dirname(lib), "-lnsamg", "-lm",
                           "-Wl,-rpath," + os.path.dirname(lib), "-o", exe])
    return exe


def test_c_client_compiles_and_links(tmp_path):
    assert os.path.exists(_build(tmp_path))


@pytest.mark.gpu
def test_c_client_solves(tmp_path):
    exe = _build(tmp_path)
    res = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert res.returncode == 0, res.stdout + res.stderr
    assert "relres=" in res.stdout
