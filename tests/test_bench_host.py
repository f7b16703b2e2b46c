"""Host-side measurement logic of bench.py, without a GPU: the nvidia-smi clock record and its
throttle reasons, DRAM traffic taken only while the kernel sources match the committed counters,
the two-floor kernel roofline, and the seeded arrival trace and queue summary of the serving
comparison."""
import hashlib
import json
import os
import shutil

import numpy as np
import pytest

import bench


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.lines = lines
    return s.summary()


def test_clock_summary_median_max_and_active_reasons():
    # index, clocks.sm, clocks.max.sm, power.draw, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    lines = ["0, 2032, 2032, 640.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
             "0, 1980, 2032, 1100.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
             "0, 2010, 2032, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"]
    got = _sampler(lines)
    assert got["sm_mhz"] == 2010.0 and got["sm_max_mhz"] == 2032.0 and got["samples"] == 3
    assert got["reasons"] == ["sw_power_cap"]
    hot = _sampler(["0, 1500, 2032, 700, 0x48, Active, Not Active, Active, Not Active"])
    assert hot["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_skips_malformed_lines():
    got = _sampler(["", "0, [N/A], 2032, 1, 0x0, Not Active, Not Active, Not Active, Not Active", "garbage",
                    "0, 2032, 2032, 1, 0x0, Not Active, Not Active, Not Active, Not Active"])
    assert got["samples"] == 1 and got["sm_mhz"] == 2032.0 and got["reasons"] == []
    empty = _sampler([])
    assert empty["sm_mhz"] is None and empty["samples"] == 0


def _fake_root(tmp_path, sha_matches: bool):
    csrc = tmp_path / "paper_2112_14681_b300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    for name in ("kernels.cuh", "gmres.cuh"):
        (csrc / name).write_bytes(f"// {name}\n".encode())
    src = b"".join((csrc / n).read_bytes() for n in ("kernels.cuh", "gmres.cuh"))
    sha = hashlib.sha256(src).hexdigest()[:16]
    d = {"source_sha": sha if sha_matches else "0" * 16, "spmv_l0": {"traffic_bytes_per_launch": 1234}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(d))
    return tmp_path


@pytest.mark.parametrize("sha_matches", [True, False])
def test_traffic_only_while_the_kernel_sources_match(tmp_path, monkeypatch, sha_matches):
    monkeypatch.setattr(bench, "ROOT", str(_fake_root(tmp_path, sha_matches)))
    assert bench.measured_traffic("spmv_l0") == (1234 if sha_matches else None)
    assert bench.measured_traffic("no_such_kernel") is None


def test_traffic_goes_null_when_a_kernel_source_changes(tmp_path, monkeypatch):
    root = _fake_root(tmp_path, True)
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.measured_traffic("spmv_l0") == 1234
    with open(root / "paper_2112_14681_b300" / "csrc" / "gmres.cuh", "a") as f:
        f.write("// changed\n")
    assert bench.measured_traffic("spmv_l0") is None


def test_committed_traffic_file_is_well_formed():
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        d = json.load(f)
    assert len(d["source_sha"]) == 16
    for key, v in d.items():
        if isinstance(v, dict) and "traffic_bytes_per_launch" in v:
            assert v["traffic_bytes_per_launch"] > 0, key


def test_kernel_roofline_takes_the_larger_floor():
    # 100 MB at 5000 GB/s = 20 us; 1e6 FP64 FMAs at 5e11/s = 2 us: HBM bound
    r = bench.kernel_roofline(25e-6, 100_000_000, 1_000_000, 5000.0, 5e11)
    assert r["bound"] == "hbm"
    assert r["GBps"] == pytest.approx(4000.0) and r["frac_hbm"] == pytest.approx(0.8)
    assert r["frac_of_bound"] == pytest.approx(0.8)
    # the same bytes with 2e7 FMAs: 40 us of FP64 work, FP64 bound
    r = bench.kernel_roofline(50e-6, 100_000_000, 20_000_000, 5000.0, 5e11)
    assert r["bound"] == "fp64" and r["frac_of_bound"] == pytest.approx(0.8)
    assert r["frac_hbm"] == pytest.approx(0.4)


def test_arrivals_are_seeded_poisson():
    t, which = bench._arrivals(20000, 65.0, 12)
    t2, which2 = bench._arrivals(20000, 65.0, 12)
    assert np.array_equal(t, t2) and np.array_equal(which, which2)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert np.mean(gaps) == pytest.approx(1 / 65.0, rel=0.03)  # exponential gaps, mean 1 / rate
    assert np.std(gaps) == pytest.approx(1 / 65.0, rel=0.05)
    assert which.min() >= 0 and which.max() < 12


def test_queue_summary_shows_growth_by_quarter():
    flat = bench._queue_summary([1, 2, 1, 2, 1, 2, 1, 2])
    assert flat["mean_by_quarter"] == [1.5, 1.5, 1.5, 1.5] and flat["max"] == 2.0
    growing = bench._queue_summary(list(range(40)))
    q = growing["mean_by_quarter"]
    assert all(b > a for a, b in zip(q, q[1:])) and growing["p50"] == pytest.approx(19.5)
    assert bench._queue_summary([]) == {"max": 0.0, "p50": 0.0, "mean_by_quarter": []}
