"""bench.py's roofline bookkeeping, on the host.

The committed DRAM traffic of the level-0 smoother step is reported only while
the kernel's sources hash to the value recorded beside it (and only for the
workload it was captured on); per-class and solve-phase figures are
algorithmic bytes / time / the HBM peak, with coarse classes that move less
than the L2 holds labelled as L2-resident.
"""
import hashlib
import os
import shutil
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

SOURCES = ("sparse.cu", "spmv.cuh", "internal.cuh")


def _args(workload="lshape", N=None):
    return types.SimpleNamespace(workload=workload, N=N)


def _fake_root(tmp_path, traffic, digest=None):
    csrc = tmp_path / "paper_2001_11533_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in SOURCES:
        shutil.copy(os.path.join(ROOT, "paper_2001_11533_gb300", "csrc", f), csrc / f)
    if digest is None:
        digest = hashlib.sha256(b"".join((csrc / f).read_bytes() for f in SOURCES)).hexdigest()
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "k_cheb_step_level0_lshape1025.md").write_text(
        f"# summary\n\ntraffic_bytes_per_launch: {traffic}\nsource_sha256: {digest}\n(hash note)\n")
    return csrc


def test_captured_traffic_follows_the_kernel_source(tmp_path, monkeypatch):
    csrc = _fake_root(tmp_path, 45510656)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.captured_traffic(_args()) == 45510656.0
    assert bench.captured_traffic(_args(N=1025)) == 45510656.0
    # another workload or grid: the capture does not describe it
    assert bench.captured_traffic(_args("cube")) is None
    assert bench.captured_traffic(_args(N=513)) is None
    # any change to the kernel's sources voids the capture
    with open(csrc / "spmv.cuh", "a") as f:
        f.write("\n// edited after the capture\n")
    assert bench.captured_traffic(_args()) is None


def test_captured_traffic_absent_or_stale_profile(tmp_path, monkeypatch):
    _fake_root(tmp_path, 1000, digest="0" * 64)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.captured_traffic(_args()) is None
    os.remove(tmp_path / "profiles" / "k_cheb_step_level0_lshape1025.md")
    assert bench.captured_traffic(_args()) is None


def test_kernel_table_fractions_and_residency(monkeypatch):
    monkeypatch.setattr(bench, "hbm_peak", lambda: (5000.0, "measured"))
    classes = {
        # 10 launches of 51.7 MB in 0.15 ms: 15 us each, 3446.7 GB/s
        "cheb_step_l0": {"launches": 10, "ms": 0.15, "bytes": 10 * 51.7e6},
        # a coarse class moving 7 MB per launch: L2-resident
        "cheb_step_coarse": {"launches": 40, "ms": 0.30, "bytes": 40 * 7e6},
        # a coarse class moving more than 32 MB per launch streams from HBM
        "cg_spmv_coarse": {"launches": 2, "ms": 0.05, "bytes": 2 * 40e6},
        "restrict_l0": {"launches": 0, "ms": 0.0, "bytes": 0.0},
    }
    t = bench.kernel_table(classes)
    assert "restrict_l0" not in t
    assert list(t) == ["cheb_step_coarse", "cheb_step_l0", "cg_spmv_coarse"]  # by time
    c = t["cheb_step_l0"]
    assert c["avg_us"] == pytest.approx(15.0)
    assert c["achieved_GBs"] == pytest.approx(517e6 / 0.15e-3 / 1e9, abs=0.1)
    assert c["frac_of_hbm"] == pytest.approx(517e6 / 0.15e-3 / 1e9 / 5000.0, abs=1e-4)
    assert c["mb_per_launch"] == pytest.approx(51.7)
    assert c["share"] == pytest.approx(0.15 / 0.50, abs=1e-4)
    assert c["residency"] == "hbm"
    assert t["cheb_step_coarse"]["residency"] == "l2-resident"
    assert t["cg_spmv_coarse"]["residency"] == "hbm"
    assert sum(v["share"] for v in t.values()) == pytest.approx(1.0, abs=1e-3)


def test_solve_phase_and_roofline_arithmetic(monkeypatch):
    monkeypatch.setattr(bench, "hbm_peak", lambda: (6000.0, "measured"))
    sp = bench.solve_phase({"alg_bytes": 2.4e11, "t_solve_s": 0.1, "hessian_applies": 5})
    assert sp["bytes_per_hessian_apply"] == pytest.approx(4.8e10)
    assert sp["achieved_GBs"] == pytest.approx(2400.0)
    assert sp["frac"] == pytest.approx(0.4)
    assert bench.solve_phase({"alg_bytes": 0.0, "t_solve_s": 0.1, "hessian_applies": 5}) is None
    r = bench.roofline_from({"kstats": {"launches": 4, "ms": 0.06, "bytes": 4 * 51.7e6}}, _args("cube"),
                            traffic="captured")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6000.0
    assert r["avg_us"] == pytest.approx(15.0)
    assert r["frac"] == pytest.approx(r["achieved"] / 6000.0, abs=1e-4)
    assert r["traffic"] is None  # no capture for this workload
    assert bench.roofline_from({"kstats": {"launches": 0, "ms": 0.0, "bytes": 0.0}}, _args()) is None
